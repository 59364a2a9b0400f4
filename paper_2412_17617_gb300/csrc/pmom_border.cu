// Bordered low-rank evaluation of candidates that differ little from a reference map.
//
// A single-pixel change removes or adds a handful of RWG basis functions (the pixel's inner BF,
// its inter-pixel BFs to metal neighbours and a pixel-port BF), so a candidate's impedance
// matrix is the reference's Z_sub(f) = A with k_r rows/columns deleted (set R) and k_a bordered
// on (set Ad).  With G = A^-1 (reference inverse, FP64) and T = S \ R the kept set:
//
//   H     = (A_TT)^-1 = G_TT - G_TR G_RR^-1 G_RT                  (inverse of a principal block)
//   H V_T = Xs[T] - G_TR G_RR^-1 Xs[R],      Xs = G V (reference port solutions)
//   H B_T = W[T]  - G_TR G_RR^-1 W[R],       W  = G B,  B = Z(f)[S, Ad]
//   C     = D - E_T H B_T,                   D  = Z(f)[Ad, Ad],  E = Z(f)[Ad, S]
//   x_T   = H V_T + H B_T C^-1 E_T H V_T,    x_Ad = -C^-1 E_T H V_T
//
// and only the port rows of x_T are needed for Y (Eq. 6-7).  Per (candidate, frequency) task the
// cost is O(n^2 k_a) for W plus O(n k (k + P)) for the reductions, against O(n^3) for a new LU;
// per frequency the reference costs one FP64 LU and n solves (the inverse), shared by the batch.
//
//   ref_lu_kernel  : gather A = Z(f)[S, S] (complex64 promoted exactly) and factor it in FP64
//   ref_inv_kernel : G = A^-1, four columns per CTA through the LU factors
//   border_kernel  : persistent; one (candidate, frequency) task per CTA at a time
#include "pmom_eval_kernels.cuh"

namespace pmom {
namespace {

constexpr int kBK = kBorderK;   // BFs removed / added per candidate at most
// The reference inverse is refined further than a candidate's port solutions: the bordered
// formulas subtract quantities of the reference's size to get a candidate's, so the inverse's
// error reaches the candidate's S relative to the reference's (for a candidate with |S21| of
// 1e-5 against a reference with 0.1, four orders of magnitude).  Refinement goes on until the
// backward error reaches kEtaInverse or stops improving; it is accepted at kEtaTarget.
constexpr double kEtaInverse = 1e-14;
constexpr int kInvCols = 4;     // inverse columns per CTA (the solve's right-hand-side width)
constexpr int kInvLd = 5;       // row stride of the mixed route's shared solution and correction

// Reference-state bits per frequency: kRefSingular (the reference matrix has a zero pivot),
// kRefFailed (the single-precision reference could not be refined: redo it in FP64), kRefRedone
// (set by the FP64 factorization of a failed frequency, read by the FP64 inverse).
constexpr uint32_t kRefSingular = 1u, kRefFailed = 2u, kRefRedone = 4u;

// gated: only the frequencies whose single-precision reference failed are factored (FP64 fallback)
template <typename ZT, int NB>
__global__ void __launch_bounds__(kThreads, 1)
ref_lu_kernel(const ZT* __restrict__ Z, int M, const int32_t* __restrict__ ref_idx, const int32_t* __restrict__ ref_n,
              double2* __restrict__ LU, int ldn, int* __restrict__ piv, uint32_t* __restrict__ ref_flags, int gated) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double s_val[kWarps + 1];
  __shared__ int s_row[kWarps + 1];
  const int f = blockIdx.x, tid = threadIdx.x;
  if (gated && !(ref_flags[f] & (kRefSingular | kRefFailed))) return;
  const int n = *ref_n;
  constexpr bool large = NB != Cfg<double2>::NB;
  size_t u_off, idx_off, tc_off;
  smem_layout<double2>(n, 0, large, &u_off, &idx_off, &tc_off);
  double2* Pn = reinterpret_cast<double2*>(smem);
  double2* Ut = reinterpret_cast<double2*>(smem + u_off);
  int* s_idx = reinterpret_cast<int*>(smem + idx_off);
  for (int i = tid; i < n; i += kThreads) s_idx[i] = ref_idx[i];
  gsync();
  const ZT* Zf = Z + static_cast<size_t>(f) * M * M;
  double2* A = LU + static_cast<size_t>(f) * n * ldn;
  for (int i = 0; i < n; ++i) {
    const ZT* zrow = Zf + static_cast<size_t>(s_idx[i]) * M;
    for (int j = tid; j < n; j += kThreads) A[static_cast<size_t>(i) * ldn + j] = zload<ZT, double2>(zrow + s_idx[j]);
  }
  gsync();
  const bool singular = lu_factor<double2, NB>(A, ldn, n, piv + static_cast<size_t>(f) * n, Pn, Ut, s_val, s_row, nullptr);
  gsync();
  lu_invert_diag<double2>(A, ldn, n, large ? Pn : Ut);   // the form lu_solve reads
  if (tid == 0) ref_flags[f] = (singular ? kRefSingular : 0u) | (gated ? kRefRedone : 0u);
}

__global__ void __launch_bounds__(kThreads)
ref_inv_kernel(const double2* __restrict__ LU, int ldn, const int* __restrict__ piv, const int32_t* __restrict__ ref_n,
               int nblk, double2* __restrict__ G, const uint32_t* __restrict__ ref_flags, int gated) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = *ref_n;
  const int f = blockIdx.x / nblk, j0 = (blockIdx.x % nblk) * kInvCols;
  if (j0 >= n) return;
  if (gated && !(ref_flags[f] & kRefRedone)) return;
  const int tid = threadIdx.x;
  double2* W = reinterpret_cast<double2*>(smem);                                  // n x 4
  double2* D = reinterpret_cast<double2*>(smem + static_cast<size_t>(n) * kInvCols * sizeof(double2));   // 32 x 33
  for (int e = tid; e < n * kInvCols; e += kThreads) {
    const int i = e / kInvCols, c = e % kInvCols;
    W[e] = make_double2(i == j0 + c ? 1.0 : 0.0, 0.0);
  }
  gsync();
  const double2* A = LU + static_cast<size_t>(f) * n * ldn;
  lu_solve<double2>(A, ldn, n, piv + static_cast<size_t>(f) * n, W, kInvCols, D);
  double2* Gf = G + static_cast<size_t>(f) * n * ldn;
  for (int e = tid; e < n * kInvCols; e += kThreads) {
    const int i = e / kInvCols, c = e % kInvCols;
    if (j0 + c < n) Gf[static_cast<size_t>(i) * ldn + j0 + c] = W[e];
  }
}

__device__ __forceinline__ float4 split_df(double2 v) {
  const float hx = static_cast<float>(v.x), hy = static_cast<float>(v.y);
  return make_float4(hx, static_cast<float>(v.x - hx), hy, static_cast<float>(v.y - hy));
}

// Reference inverse from the single-precision factors kept by the factor-only evaluation launch
// (workspace slot f: LU, pivots and the exact complex64 copy of Z_sub), four columns per task:
// X = LU^-1 e_j, then iterative refinement with the float-float residual e_j - Z_sub X until the
// normwise backward error reaches kEtaInverse (or stops improving; accepted at kEtaTarget).  X
// stays in shared memory as float-float pairs (re_hi, re_lo, im_hi, im_lo): the residual reads it
// as it is and each float correction is added in float-float, so the refinement does no FP64
// work, and the converged columns go to G in the same form.  Columns whose refinement stalls mark
// their frequency kRefFailed; the gated FP64 kernels then recompute that frequency.
__global__ void __launch_bounds__(kThreads) ref_inv_mixed_kernel(RefInvArgs r) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double s_red[2 * kWarps], s_norm[2];
  __shared__ float s_xmax[kWarps];
  __shared__ int s_task, s_flag;
  const int n = *r.ref_n, ldn = r.ldn, lda = r.lda;
  const int nblk = (n + kInvCols - 1) / kInvCols, ntasks = r.F * nblk;
  const int tid = gtid();
  // X and W rows kInvLd apart (odd): the four columns of consecutive rows fall in distinct banks
  float4* X = reinterpret_cast<float4*>(smem);                                                  // n x kInvLd
  float2* W = reinterpret_cast<float2*>(smem + static_cast<size_t>(n) * kInvLd * sizeof(float4));   // n x kInvLd
  float2* D = reinterpret_cast<float2*>(smem + static_cast<size_t>(n) * kInvLd * (sizeof(float4) + sizeof(float2)));
  const Slot sl = slot_layout(r.ncap, lda, r.P, sizeof(float2));
  double lone[kMaxPorts] = {1.0, 1.0, 1.0, 1.0};
  for (;;) {
    if (tid == 0) {
      const int tt = atomicAdd(r.task_counter, 1);
      s_task = tt;
      // a frequency whose factorization or another column block failed is left to the FP64
      // fallback (read once: other CTAs may set the flag meanwhile)
      s_flag = tt < ntasks ? static_cast<int>(r.ref_flags[tt / nblk] & (kRefSingular | kRefFailed)) : 0;
    }
    gsync();
    const int t = s_task, skip = s_flag;
    gsync();
    if (t >= ntasks) break;
    const int f = t / nblk, j0 = (t % nblk) * kInvCols;
    if (skip) continue;
    const unsigned char* ws = static_cast<const unsigned char*>(r.work) + r.slot_bytes * f;
    const float2* A = reinterpret_cast<const float2*>(ws + sl.a_off);
    const float2* Zs = reinterpret_cast<const float2*>(ws + sl.zs_off);
    const int* piv = reinterpret_cast<const int*>(ws + sl.piv_off);
    for (int e = tid; e < n * kInvCols; e += kThreads) {
      const int i = e / kInvCols, c = e % kInvCols;
      W[i * kInvLd + c] = make_float2(i == j0 + c ? 1.f : 0.f, 0.f);
    }
    gsync();
    lu_solve<float2>(A, lda, n, piv, W, kInvCols, D, kInvLd);
    for (int e = tid; e < n * kInvCols; e += kThreads) {
      const int o = (e / kInvCols) * kInvLd + e % kInvCols;
      X[o] = make_float4(W[o].x, 0.f, W[o].y, 0.f);
    }
    gsync();
    bool converged = false;
    double rprev = 0.0;
    for (int it = 0; it <= kMaxRefine; ++it) {
      float xmax = 0.f;
      for (int e = tid; e < n * kInvCols; e += kThreads) {
        const int o = (e / kInvCols) * kInvLd + e % kInvCols;
        xmax = fmaxf(xmax, fabsf(X[o].x) + fabsf(X[o].z));
      }
      residual_df<kInvCols, true>(Zs, lda, n, X, kInvCols, lone, nullptr, s_red, s_norm, j0, W, 3, 1, 1, nullptr,
                                  kInvLd);
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) xmax = fmaxf(xmax, __shfl_down_sync(0xffffffffu, xmax, d));
      if ((tid & 31) == 0) s_xmax[tid >> 5] = xmax;
      gsync();
      if (tid == 0) {
        float m = 0.f;
        for (int w = 0; w < kWarps; ++w) m = fmaxf(m, s_xmax[w]);
        const double rn = s_norm[0], zn = s_norm[1];
        const double eta = rn / (zn * static_cast<double>(m) + 1.0);
        int flag = 0;
        if (eta <= kEtaInverse) flag = 1;
        else if ((it > 0 && rn > 0.5 * rprev) || it == kMaxRefine) flag = eta <= kEtaTarget ? 1 : 2;
        s_flag = flag;
        s_norm[0] = rn;
      }
      gsync();
      const int flag = s_flag;
      rprev = s_norm[0];
      if (flag != 0) {
        converged = flag == 1;
        break;
      }
      lu_solve<float2>(A, lda, n, piv, W, kInvCols, D, kInvLd);
      for (int e = tid; e < n * kInvCols; e += kThreads) {   // X += correction, in float-float
        const int o = (e / kInvCols) * kInvLd + e % kInvCols;
        float4 x = X[o];
        dd_add(x.x, x.y, W[o].x, 0.f);
        dd_add(x.z, x.w, W[o].y, 0.f);
        X[o] = x;
      }
      gsync();
    }
    if (!converged) {
      if (tid == 0) atomicOr(&r.ref_flags[f], kRefFailed);
    } else {   // the bordered update reads G as float-float pairs
      float4* Gq = reinterpret_cast<float4*>(r.G) + static_cast<size_t>(f) * n * ldn;
      for (int e = tid; e < n * kInvCols; e += kThreads) {
        const int i = e / kInvCols, c = e % kInvCols;
        Gq[static_cast<size_t>(i) * ldn + j0 + c] = X[i * kInvLd + c];
      }
    }
    gsync();
  }
}

// The FP64 fallback writes G(f) as doubles; the float-float route converts the frequencies it
// redid in place.
__global__ void ref_g_to_df_kernel(double2* __restrict__ G, const int32_t* __restrict__ ref_n, int ldn,
                                   const uint32_t* __restrict__ ref_flags) {
  const int f = blockIdx.y;
  if (!(ref_flags[f] & kRefRedone)) return;
  const int n = *ref_n;
  double2* Gf = G + static_cast<size_t>(f) * n * ldn;
  const size_t total = static_cast<size_t>(n) * ldn;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<size_t>(gridDim.x) * blockDim.x)
    *reinterpret_cast<float4*>(&Gf[e]) = split_df(Gf[e]);
}

__device__ __forceinline__ bool in_sorted(const int32_t* a, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int x = a[mid];
    if (x == v) return true;
    if (x < v) lo = mid + 1; else hi = mid;
  }
  return false;
}

// Solve the k x k system Am X = Bm (nr right-hand sides, row-major, leading dims kBK / ldb) by
// Gaussian elimination with partial pivoting, in place (X overwrites Bm).  One thread.  Returns
// false if a pivot is exactly zero.
__device__ bool small_solve(double2* Am, int k, double2* Bm, int nr, int ldb) {
  for (int c = 0; c < k; ++c) {
    int p = c;
    double best = cabs2(Am[c * kBK + c]);
    for (int r = c + 1; r < k; ++r)
      if (cabs2(Am[r * kBK + c]) > best) { best = cabs2(Am[r * kBK + c]); p = r; }
    if (best == 0.0) return false;
    if (p != c) {
      for (int j = 0; j < k; ++j) { const double2 t = Am[c * kBK + j]; Am[c * kBK + j] = Am[p * kBK + j]; Am[p * kBK + j] = t; }
      for (int j = 0; j < nr; ++j) { const double2 t = Bm[c * ldb + j]; Bm[c * ldb + j] = Bm[p * ldb + j]; Bm[p * ldb + j] = t; }
    }
    const double2 inv = cinv(Am[c * kBK + c]);
    for (int r = c + 1; r < k; ++r) {
      const double2 l = cmul(Am[r * kBK + c], inv);
      for (int j = c + 1; j < k; ++j) Am[r * kBK + j] = cfms(l, Am[c * kBK + j], Am[r * kBK + j]);
      for (int j = 0; j < nr; ++j) Bm[r * ldb + j] = cfms(l, Bm[c * ldb + j], Bm[r * ldb + j]);
    }
  }
  for (int c = k - 1; c >= 0; --c) {
    const double2 inv = cinv(Am[c * kBK + c]);
    for (int j = 0; j < nr; ++j) {
      double2 v = Bm[c * ldb + j];
      for (int t = c + 1; t < k; ++t) v = cfms(Am[c * kBK + t], Bm[t * ldb + j], v);
      Bm[c * ldb + j] = cmul(v, inv);
    }
  }
  return true;
}

// SMEM_B: the added columns B = Z(f)[S, Ad] are staged in shared memory (q-major, so the lanes of
// a warp read consecutive rows); otherwise they stay in the slot's global scratch.
// DF (complex64 databases only): W = G B in float-float arithmetic on the FP32 pipe -- B's
// entries are exact floats and each G entry is split into two floats -- instead of FP64 (the
// FP64 pipe runs at 1/64 of the FP32 rate); partial sums carry about 2^-44 relative error.
template <typename ZT, bool SMEM_B, bool DF>
__global__ void __launch_bounds__(kThreads) border_kernel(BorderArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_task, s_kr, s_ka, s_bad;
  __shared__ int s_R[kBK], s_A[kBK];
  __shared__ double2 s_GRR[kBK * kBK], s_Z[kBK * (kMaxPorts + kBK)];   // G_RR, then [Z1 | Z2]
  __shared__ double2 s_HVp[kMaxPorts * kMaxPorts], s_GpR[kMaxPorts * kBK], s_HBp[kMaxPorts * kBK];
  __shared__ double2 s_U[kBK * (kMaxPorts + kBK)];                     // [E_T H V_T | E_T H B_T]
  __shared__ double2 s_C[kBK * kBK], s_D[kBK * kBK];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int M = a.M, P = a.P, n = *a.ref_n, ldn = a.ldn;
  static_assert(!DF || std::is_same<ZT, float2>::value, "float-float W needs exact float database entries");
  using BT = typename std::conditional<DF, float2, double2>::type;
  BT* s_B = reinterpret_cast<BT*>(smem);   // kBK x n (SMEM_B)
  int32_t* s_ref = reinterpret_cast<int32_t*>(smem + (SMEM_B ? static_cast<size_t>(kBK) * n * sizeof(BT) : 0));
  for (int i = tid; i < n; i += kThreads) s_ref[i] = a.ref_idx[i];
  const int NQ = kMaxPorts + kBK;
  double2* ws = a.work + a.slot_elems * blockIdx.x;
  BT* Bm = SMEM_B ? s_B : reinterpret_cast<BT*>(ws);  // kBK x n : Z(f)[S, Ad], column q of B is row q
  double2* Wm = ws + static_cast<size_t>(n) * kBK;     // n x kBK : G B
  double2* Em = Wm + static_cast<size_t>(n) * kBK;     // kBK x n : Z(f)[Ad, S]
  double2* Qm = Em + static_cast<size_t>(kBK) * n;     // n x NQ  : [H V_T | H B_T] rows over T (0 on R)
  double lp[kMaxPorts];
#pragma unroll
  for (int p = 0; p < kMaxPorts; ++p) lp[p] = a.port_len[p];
  const int ntasks = a.B * a.F;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(a.task_counter, 1);
    __syncthreads();
    const int t = s_task;
    if (t >= ntasks) break;
    const int f = t / a.B, b = t % a.B;
    double2* Y = a.S + (static_cast<size_t>(b) * a.F + f) * P * P;
    const int N = a.n_act[b];
    const double2 nan2 = make_double2(__longlong_as_double(0x7ff8000000000000ll), 0.0);
    if (N <= 0 || (a.ref_flags[f] & kRefSingular)) {   // bad pixel state (flagged by the activation) or singular reference
      if (tid < P * P) Y[tid] = nan2;
      if (tid == 0 && N > 0) atomicOr(&a.flags[b], kFlagSingular);
      __syncthreads();
      continue;
    }
    const int32_t* cidx = a.idx + static_cast<size_t>(b) * M;
    if (tid == 0) { s_kr = 0; s_ka = 0; s_bad = 0; }
    __syncthreads();
    // R: reference positions whose BF the candidate lacks; Ad: candidate BFs the reference lacks
    for (int i = tid; i < n; i += kThreads)
      if (!in_sorted(cidx, N, s_ref[i])) {
        const int k = atomicAdd(&s_kr, 1);
        if (k < kBK) s_R[k] = i;
      }
    for (int j = tid; j < N; j += kThreads) {
      const int v = cidx[j];
      if (!in_sorted(s_ref, n, v)) {
        const int k = atomicAdd(&s_ka, 1);
        if (k < kBK) s_A[k] = v;
      }
    }
    __syncthreads();
    const int kr = s_kr, ka = s_ka;
    if (kr > kBK || ka > kBK) {   // change too large for the bordered update
      if (tid < P * P) Y[tid] = nan2;
      if (tid == 0) atomicOr(&a.flags[b], kFlagFar);
      __syncthreads();
      continue;
    }
    if (tid == 0) {   // deterministic order (the atomics above fill the lists in any order)
      for (int i = 1; i < kr; ++i)
        for (int j = i; j > 0 && s_R[j - 1] > s_R[j]; --j) { const int x = s_R[j]; s_R[j] = s_R[j - 1]; s_R[j - 1] = x; }
      for (int i = 1; i < ka; ++i)
        for (int j = i; j > 0 && s_A[j - 1] > s_A[j]; --j) { const int x = s_A[j]; s_A[j] = s_A[j - 1]; s_A[j - 1] = x; }
    }
    __syncthreads();
    // G(f): double2, or (DF) float-float pairs (re_hi, re_lo, im_hi, im_lo) read back as doubles
    const double2* Gf = static_cast<const double2*>(a.G) + static_cast<size_t>(f) * n * ldn;
    const float4* Gq = static_cast<const float4*>(a.G) + static_cast<size_t>(f) * n * ldn;
    auto gv = [&](size_t off) -> double2 {
      if constexpr (DF) {
        const float4 v = Gq[off];
        return make_double2(static_cast<double>(v.x) + static_cast<double>(v.y),
                            static_cast<double>(v.z) + static_cast<double>(v.w));
      } else {
        return Gf[off];
      }
    };
    const ZT* Zf = static_cast<const ZT*>(a.Z) + static_cast<size_t>(f) * M * M;
    // small blocks of G: G_RR, G[ports, R], and the right-hand sides [Xs[R] | W[R]] come later
    for (int e = tid; e < kr * kr; e += kThreads) {
      const int r = e / kr, q = e % kr;
      s_GRR[r * kBK + q] = gv(static_cast<size_t>(s_R[r]) * ldn + s_R[q]);
    }
    for (int e = tid; e < P * kr; e += kThreads) {
      const int p = e / kr, r = e % kr;
      s_GpR[p * kBK + r] = gv(static_cast<size_t>(3 * p + 1) * ldn + s_R[r]);
    }
    // additions: B = Z(f)[S, Ad], E = Z(f)[Ad, S], D = Z(f)[Ad, Ad]
    for (int e = tid; e < n * ka; e += kThreads) {
      const int j = e / ka, q = e % ka;
      Bm[static_cast<size_t>(q) * n + j] = zload<ZT, BT>(Zf + static_cast<size_t>(s_ref[j]) * M + s_A[q]);
    }
    for (int e = tid; e < ka * n; e += kThreads) {
      const int q = e / n, j = e % n;
      Em[static_cast<size_t>(q) * n + j] = zload<ZT, double2>(Zf + static_cast<size_t>(s_A[q]) * M + s_ref[j]);
    }
    for (int e = tid; e < ka * ka; e += kThreads) {
      const int q = e / ka, r = e % ka;
      s_D[q * kBK + r] = zload<ZT, double2>(Zf + static_cast<size_t>(s_A[q]) * M + s_A[r]);
    }
    __syncthreads();
    // W = G B: one warp per row of G, lanes over the columns
    if (ka > 0) {
      if constexpr (DF) {
        for (int i = warp; i < n; i += kWarps) {
          float rh[kBK], rl[kBK], ih[kBK], il[kBK];
#pragma unroll
          for (int q = 0; q < kBK; ++q) rh[q] = rl[q] = ih[q] = il[q] = 0.f;
          const float4* grow = Gq + static_cast<size_t>(i) * ldn;
          for (int j = lane; j < n; j += 32) {
            const float4 g = grow[j];
            const float gxh = g.x, gxl = g.y, gyh = g.z, gyl = g.w;
#pragma unroll
            for (int q = 0; q < kBK; ++q)
              if (q < ka) {
                const float2 bq = Bm[static_cast<size_t>(q) * n + j];
                df_mac(bq.x, gxh, gxl, rh[q], rl[q]);
                df_mac(-bq.y, gyh, gyl, rh[q], rl[q]);
                df_mac(bq.y, gxh, gxl, ih[q], il[q]);
                df_mac(bq.x, gyh, gyl, ih[q], il[q]);
              }
          }
#pragma unroll
          for (int q = 0; q < kBK; ++q) {
            if (q >= ka) break;
            float xh = rh[q], xl = rl[q], yh = ih[q], yl = il[q];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
              const float oxh = __shfl_down_sync(0xffffffffu, xh, d), oxl = __shfl_down_sync(0xffffffffu, xl, d);
              const float oyh = __shfl_down_sync(0xffffffffu, yh, d), oyl = __shfl_down_sync(0xffffffffu, yl, d);
              dd_add(xh, xl, oxh, oxl);
              dd_add(yh, yl, oyh, oyl);
            }
            if (lane == 0)
              Wm[static_cast<size_t>(i) * kBK + q] =
                  make_double2(static_cast<double>(xh) + static_cast<double>(xl), static_cast<double>(yh) + static_cast<double>(yl));
          }
        }
      } else {
        for (int i = warp; i < n; i += kWarps) {
          double2 acc[kBK];
#pragma unroll
          for (int q = 0; q < kBK; ++q) acc[q] = make_double2(0.0, 0.0);
          const double2* grow = Gf + static_cast<size_t>(i) * ldn;
          int j = lane;
          for (; j + 32 < n; j += 64) {   // two column steps in flight
            const double2 g0 = grow[j], g1 = grow[j + 32];
#pragma unroll
            for (int q = 0; q < kBK; ++q)
              if (q < ka) {
                acc[q] = cfma(g0, Bm[static_cast<size_t>(q) * n + j], acc[q]);
                acc[q] = cfma(g1, Bm[static_cast<size_t>(q) * n + j + 32], acc[q]);
              }
          }
          if (j < n) {
            const double2 g0 = grow[j];
#pragma unroll
            for (int q = 0; q < kBK; ++q)
              if (q < ka) acc[q] = cfma(g0, Bm[static_cast<size_t>(q) * n + j], acc[q]);
          }
#pragma unroll
          for (int q = 0; q < kBK; ++q) {
            if (q >= ka) break;
            double2 v = acc[q];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
              v.x += __shfl_down_sync(0xffffffffu, v.x, d);
              v.y += __shfl_down_sync(0xffffffffu, v.y, d);
            }
            if (lane == 0) Wm[static_cast<size_t>(i) * kBK + q] = v;
          }
        }
      }
    }
    __syncthreads();
    // [Z1 | Z2] = G_RR^-1 [Xs[R] | W[R]]   (Xs[r][p] = G[r][port p] l_p)
    if (tid == 0) {
      for (int e = 0; e < kBK * NQ; ++e) s_Z[e] = make_double2(0.0, 0.0);
      for (int r = 0; r < kr; ++r) {
        const size_t row = static_cast<size_t>(s_R[r]) * ldn;
        for (int p = 0; p < P; ++p) {
          const double2 g = gv(row + 3 * p + 1);
          s_Z[r * NQ + p] = make_double2(g.x * lp[p], g.y * lp[p]);
        }
        for (int q = 0; q < ka; ++q) s_Z[r * NQ + kMaxPorts + q] = Wm[static_cast<size_t>(s_R[r]) * kBK + q];
      }
      if (kr > 0 && !small_solve(s_GRR, kr, s_Z, NQ, NQ)) s_bad = 1;
      // port rows: HVp = Xs[ports] - G[ports, R] Z1,  (H B_T)[ports] = W[ports] - G[ports, R] Z2
      for (int p = 0; p < P; ++p) {
        const size_t row = static_cast<size_t>(3 * p + 1) * ldn;
        for (int q = 0; q < P; ++q) {
          const double2 g = gv(row + 3 * q + 1);
          double2 v = make_double2(g.x * lp[q], g.y * lp[q]);
          for (int r = 0; r < kr; ++r) v = cfms(s_GpR[p * kBK + r], s_Z[r * NQ + q], v);
          s_HVp[p * kMaxPorts + q] = v;
        }
        for (int q = 0; q < ka; ++q) {
          double2 v = Wm[static_cast<size_t>(3 * p + 1) * kBK + q];
          for (int r = 0; r < kr; ++r) v = cfms(s_GpR[p * kBK + r], s_Z[r * NQ + kMaxPorts + q], v);
          s_HBp[p * kBK + q] = v;
        }
      }
    }
    __syncthreads();
    if (ka > 0 && !s_bad) {
      // Q rows over T: [H V_T | H B_T][t] = [Xs[t] | W[t]] - G[t, R] [Z1 | Z2]; zero on R
      for (int e = tid; e < n * (P + ka); e += kThreads) {
        const int i = e / (P + ka), c = e % (P + ka);
        const int q = c < P ? c : kMaxPorts + (c - P);
        bool inR = false;
        for (int r = 0; r < kr; ++r) inR |= s_R[r] == i;
        double2 v = make_double2(0.0, 0.0);
        if (!inR) {
          const size_t row = static_cast<size_t>(i) * ldn;
          if (c < P) {
            const double2 g = gv(row + 3 * c + 1);
            v = make_double2(g.x * lp[c], g.y * lp[c]);
          } else {
            v = Wm[static_cast<size_t>(i) * kBK + (c - P)];
          }
          for (int r = 0; r < kr; ++r) v = cfms(gv(row + s_R[r]), s_Z[r * NQ + q], v);
        }
        Qm[static_cast<size_t>(i) * NQ + q] = v;
      }
      __syncthreads();
      // [E_T H V_T | E_T H B_T]: one warp per output, lanes over the rows (R rows are zero in Q)
      for (int o = warp; o < ka * (P + ka); o += kWarps) {
        const int q = o / (P + ka), c = o % (P + ka);
        const int cq = c < P ? c : kMaxPorts + (c - P);
        double2 v = make_double2(0.0, 0.0);
        const double2* erow = Em + static_cast<size_t>(q) * n;
        for (int j = lane; j < n; j += 32) v = cfma(erow[j], Qm[static_cast<size_t>(j) * NQ + cq], v);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          v.x += __shfl_down_sync(0xffffffffu, v.x, d);
          v.y += __shfl_down_sync(0xffffffffu, v.y, d);
        }
        if (lane == 0) s_U[q * NQ + cq] = v;
      }
      __syncthreads();
      if (tid == 0) {
        // C = D - E_T H B_T; y = C^-1 E_T H V_T; x_ports = HVp + (H B_T)[ports] y
        for (int q = 0; q < ka; ++q)
          for (int r = 0; r < ka; ++r) {
            const double2 d = s_D[q * kBK + r], u = s_U[q * NQ + kMaxPorts + r];
            s_C[q * kBK + r] = make_double2(d.x - u.x, d.y - u.y);
          }
        if (!small_solve(s_C, ka, s_U, P, NQ)) s_bad = 1;
        for (int p = 0; p < P; ++p)
          for (int q = 0; q < P; ++q) {
            double2 v = s_HVp[p * kMaxPorts + q];
            for (int r = 0; r < ka; ++r) v = cfma(s_HBp[p * kBK + r], s_U[r * NQ + q], v);
            s_HVp[p * kMaxPorts + q] = v;
          }
      }
      __syncthreads();
    }
    // Y_ij = l_i x_i^(j) (Eq. 7) into the S slot; ys_kernel converts it
    if (tid < P * P) {
      const int i = tid / P, j = tid % P;
      const double2 x = s_HVp[i * kMaxPorts + j];
      Y[tid] = s_bad ? nan2 : make_double2(lp[i] * x.x, lp[i] * x.y);
    }
    if (tid == 0 && s_bad) atomicOr(&a.flags[b], kFlagSingular);
    __syncthreads();
  }
}

template <typename ZT, int NB>
cudaError_t launch_ref_lu_t(const void* Z, int M, const int32_t* ref_idx, const int32_t* ref_n, int n, int F,
                            double2* LU, int ldn, int* piv, uint32_t* ref_flags, int gated, cudaStream_t s) {
  size_t u_off, idx_off, tc_off;
  const size_t smem = smem_layout<double2>(n, 0, NB != Cfg<double2>::NB, &u_off, &idx_off, &tc_off);
  auto k = ref_lu_kernel<ZT, NB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<F, kThreads, smem, s>>>(static_cast<const ZT*>(Z), M, ref_idx, ref_n, LU, ldn, piv, ref_flags, gated);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ref_factor(const void* Z, int z_c128, int M, const int32_t* ref_idx, const int32_t* ref_n, int n,
                              int F, double2* LU, int ldn, int* piv, uint32_t* ref_flags, int gated, cudaStream_t s) {
  const bool large = needs_large_layout<double2>(n, false);
  if (z_c128)
    return large ? launch_ref_lu_t<double2, Cfg<double2>::NBL>(Z, M, ref_idx, ref_n, n, F, LU, ldn, piv, ref_flags, gated, s)
                 : launch_ref_lu_t<double2, Cfg<double2>::NB>(Z, M, ref_idx, ref_n, n, F, LU, ldn, piv, ref_flags, gated, s);
  return large ? launch_ref_lu_t<float2, Cfg<double2>::NBL>(Z, M, ref_idx, ref_n, n, F, LU, ldn, piv, ref_flags, gated, s)
               : launch_ref_lu_t<float2, Cfg<double2>::NB>(Z, M, ref_idx, ref_n, n, F, LU, ldn, piv, ref_flags, gated, s);
}

cudaError_t launch_ref_inverse(const double2* LU, int ldn, const int* piv, const int32_t* ref_n, int n, int F,
                               double2* G, const uint32_t* ref_flags, int gated, cudaStream_t s) {
  const int nblk = (n + kInvCols - 1) / kInvCols;
  const size_t smem = static_cast<size_t>(n) * kInvCols * sizeof(double2) + 32 * 33 * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(ref_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  ref_inv_kernel<<<F * nblk, kThreads, smem, s>>>(LU, ldn, piv, ref_n, nblk, G, ref_flags, gated);
  return cudaGetLastError();
}

cudaError_t launch_ref_g_to_df(double2* G, const int32_t* ref_n, int ldn, const uint32_t* ref_flags, int F,
                               cudaStream_t s) {
  ref_g_to_df_kernel<<<dim3(64, F), 256, 0, s>>>(G, ref_n, ldn, ref_flags);
  return cudaGetLastError();
}

size_t ref_inverse_mixed_smem(int n) {
  return static_cast<size_t>(n) * kInvLd * (sizeof(float4) + sizeof(float2)) + 32 * 33 * sizeof(float2);
}

bool ref_inverse_mixed_fits(int n) { return ref_inverse_mixed_smem(n) + 4096 <= static_cast<size_t>(optin_smem()); }

int ref_inverse_mixed_slots(int num_sms, int n) {
  const size_t smem = ref_inverse_mixed_smem(n);
  int per_sm = 0;
  if (cudaFuncSetAttribute(ref_inv_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ref_inv_mixed_kernel, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms;
}

cudaError_t launch_ref_inverse_mixed(const RefInvArgs& r, int nslots, int n, cudaStream_t s) {
  const size_t smem = ref_inverse_mixed_smem(n);
  cudaError_t e = cudaFuncSetAttribute(ref_inv_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  ref_inv_mixed_kernel<<<nslots, kThreads, smem, s>>>(r);
  return cudaGetLastError();
}

size_t border_slot_elems(int n) {
  return static_cast<size_t>(n) * (3 * kBK + kMaxPorts + kBK) + 64;
}

namespace {
size_t border_smem(int n, bool smem_b, bool df) {
  return static_cast<size_t>(n) * sizeof(int32_t) +
         (smem_b ? static_cast<size_t>(kBK) * n * (df ? sizeof(float2) : sizeof(double2)) : 0);
}
bool border_smem_b(int n, bool df) { return border_smem(n, true, df) + 16384 <= static_cast<size_t>(optin_smem()); }

template <typename ZT, bool SMEM_B, bool DF>
int border_slots_t(int num_sms, int n) {
  const size_t smem = border_smem(n, SMEM_B, DF);
  auto k = border_kernel<ZT, SMEM_B, DF>;
  int per_sm = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return per_sm * num_sms;
}

template <typename ZT, bool SMEM_B, bool DF>
cudaError_t launch_border_t(const BorderArgs& a, int nslots, int n, cudaStream_t s) {
  const size_t smem = border_smem(n, SMEM_B, DF);
  auto k = border_kernel<ZT, SMEM_B, DF>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k<<<nslots, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

int border_slots(int num_sms, int n, int z_c128, int df) {
  const bool d = df && !z_c128;
  if (d) return border_smem_b(n, true) ? border_slots_t<float2, true, true>(num_sms, n) : border_slots_t<float2, false, true>(num_sms, n);
  return border_smem_b(n, false) ? border_slots_t<float2, true, false>(num_sms, n) : border_slots_t<float2, false, false>(num_sms, n);
}

cudaError_t launch_border(const BorderArgs& a, int nslots, int n, int df, cudaStream_t s) {
  if (a.z_c128) {
    return border_smem_b(n, false) ? launch_border_t<double2, true, false>(a, nslots, n, s)
                                   : launch_border_t<double2, false, false>(a, nslots, n, s);
  }
  if (df)
    return border_smem_b(n, true) ? launch_border_t<float2, true, true>(a, nslots, n, s)
                                  : launch_border_t<float2, false, true>(a, nslots, n, s);
  return border_smem_b(n, false) ? launch_border_t<float2, true, false>(a, nslots, n, s)
                                 : launch_border_t<float2, false, false>(a, nslots, n, s);
}

}  // namespace pmom
