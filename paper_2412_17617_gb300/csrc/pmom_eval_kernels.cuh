// Candidate-evaluation kernels for sm_103a (device code shared by the default and the
// large-support-set translation units).
//
//   activate_kernel : pixel map -> active-BF indices I (Eq. 3, ascending) by a block-wide ballot scan
//   eval_kernel     : persistent; one CTA per (frequency, candidate) task at a time, frequency-major
//                     so the parent Z(f) being read stays resident in L2.  Per task:
//                       gather Z_sub = Z(f)[I, I]                           (Eq. 4-5)
//                       blocked right-looking LU, partial pivoting          (Eq. 2)
//                       forward/back substitution for the P port excitations
//                       [mixed] iterative refinement: residual V - Z_sub x in double from the
//                               exact stored Z entries, correction with the single-precision LU
//                       Y_ij = l_i x_i^(j), S = (1 + Z0 Y)^-1 (1 - Z0 Y)   (Eq. 6-7)
//   fom_kernel      : FoM of Eq. (8)-(9) per candidate, frequencies summed in order.
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor maps are encoded through the runtime's driver entry point)

#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "pmom_internal.h"
#include "pmom_tc.cuh"

namespace pmom {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// The evaluation kernel runs up to two independent task groups of kThreads threads per CTA: a
// kernel that allocates tensor memory gets one CTA per SM, and two groups keep two tasks in flight
// per SM (one overlapping the other's latency-bound phases).  Each group synchronises on its own
// named barrier and owns a shared-memory region, a workspace slot and 256 TMEM columns.
constexpr int kMaxGroups = 2;
__device__ __forceinline__ int gtid() { return threadIdx.x & (kThreads - 1); }
__device__ __forceinline__ int group_id() { return threadIdx.x / kThreads; }
__device__ __forceinline__ void gsync() {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + group_id()), "r"(kThreads) : "memory");
}
// Phase clocks, for profiling builds only (compiled with -DPMOM_PHASES): thread 0 of each task
// group adds the cycles since its previous mark (the variable t) to a per-phase device counter.
// In normal builds the marks expand to nothing.
// Slots 16 and up split phases further (their cycles are also counted in the enclosing phase);
// they are lapped into local accumulators and added once per call (PMOM_LAP / PMOM_LAP_FLUSH).
constexpr int kPhaseSlots = 32;
enum Phase : int {
  kPhGather = 0, kPhLu = 1, kPhSolve0 = 2, kPhResid = 3, kPhSolveCorr = 4, kPhOther = 5, kPhPanelLoad = 6,
  kPhPanelFactor = 7, kPhColGemm = 8, kPhPanel = 9, kPhSwap = 10, kPhInnerU = 11, kPhInnerUpd = 12, kPhRowGemm = 13,
  kPhTrsm = 14,
  kPhTasks = 15,
  kPhSolvePerm = 16, kPhSolveStage = 17, kPhSolveOff = 18, kPhSolveDiag = 19, kPhPanelWork = 20, kPhPanelWait = 21,
  kPhGemmCopyWait = 22, kPhGemmStageWait = 23, kPhGemmSync = 24, kPhGemmMma = 25, kPhGemmEpi = 26,
  kPhGemmIssue = 27, kPhGemmConv = 28
};
#ifdef PMOM_PHASES
__device__ unsigned long long g_phase_cycles[kPhaseSlots];
#define PMOM_PHASE_START(t) long long t = clock64()
#define PMOM_PHASE(slot, t)                                                                      \
  do {                                                                                           \
    if (gtid() == 0) {                                                                           \
      const long long n_ = clock64();                                                            \
      atomicAdd(&g_phase_cycles[slot], static_cast<unsigned long long>(n_ - (t)));               \
      (t) = n_;                                                                                  \
    }                                                                                            \
  } while (0)
#define PMOM_LAP(acc, t)                                                                         \
  do {                                                                                           \
    if (gtid() == 0) {                                                                           \
      const long long n_ = clock64();                                                            \
      (acc) += n_ - (t);                                                                         \
      (t) = n_;                                                                                  \
    }                                                                                            \
  } while (0)
#define PMOM_LAP_FLUSH(slot, acc)                                                                \
  do {                                                                                           \
    if (gtid() == 0) atomicAdd(&g_phase_cycles[slot], static_cast<unsigned long long>(acc));     \
  } while (0)
#else
#define PMOM_PHASE_START(t) do { } while (0)
#define PMOM_PHASE(slot, t) do { } while (0)
#define PMOM_LAP(acc, t) do { } while (0)
#define PMOM_LAP_FLUSH(slot, acc) do { } while (0)
#endif

constexpr int kTile = 64;        // trailing-update tile (rows and columns)
constexpr int kOuter = 64;       // outer panel width of the two-level (tensor-core) LU
constexpr int kMaxRefine = 10;
// Refinement target on the normwise backward error: reachable by the float-float residual
// (about 2^-44 per partial sum) and, with cond(Z_sub) ~ 1e4-1e5, far below |dS| = 1e-6.
constexpr double kEtaTarget = 1e-12;
// Stop without another residual once the predicted forward error of the corrected x -- this
// correction times the contraction rate seen over the last two corrections -- is below this
// fraction of ||x||_inf (the classic correction-norm test of iterative refinement).
constexpr double kDxTarget = 1e-10;

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c - a*b
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
  c.x = fmaf(-a.x, b.x, c.x); c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(-a.x, b.y, c.y); c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
  c.x = fma(-a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
// c + a*b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float2 cinv(float2 a) {
  const float d = cabs2(a);
  return make_float2(a.x / d, -a.y / d);
}
__device__ __forceinline__ double2 cinv(double2 a) {
  const double d = cabs2(a);
  return make_double2(a.x / d, -a.y / d);
}
__device__ __forceinline__ float2 czero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 czero(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 make_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 make_neg(double2 a) { return make_double2(-a.x, -a.y); }

template <typename T> __device__ __forceinline__ T from_f2(float2 z);
template <> __device__ __forceinline__ float2 from_f2<float2>(float2 z) { return z; }
template <> __device__ __forceinline__ double2 from_f2<double2>(float2 z) { return make_double2(z.x, z.y); }
template <typename T> __device__ __forceinline__ T from_d2(double2 z);
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 z) {
  return make_float2(static_cast<float>(z.x), static_cast<float>(z.y));
}
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 z) { return z; }
__device__ __forceinline__ double2 to_d2(float2 z) { return make_double2(z.x, z.y); }
__device__ __forceinline__ double2 to_d2(double2 z) { return z; }

template <typename ZT, typename T> __device__ __forceinline__ T zload(const ZT* p);
template <> __device__ __forceinline__ float2 zload<float2, float2>(const float2* p) { return __ldg(p); }
template <> __device__ __forceinline__ double2 zload<float2, double2>(const float2* p) { return to_d2(__ldg(p)); }
template <> __device__ __forceinline__ double2 zload<double2, double2>(const double2* p) { return __ldg(p); }
template <> __device__ __forceinline__ float2 zload<double2, float2>(const double2* p) {
  return from_d2<float2>(__ldg(p));
}

// the same conversions for a value already loaded (from shared memory)
template <typename ZT, typename T> __device__ __forceinline__ T zconv(ZT v);
template <> __device__ __forceinline__ float2 zconv<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 zconv<float2, double2>(float2 v) { return to_d2(v); }
template <> __device__ __forceinline__ double2 zconv<double2, double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 zconv<double2, float2>(double2 v) { return from_d2<float2>(v); }

__device__ __forceinline__ float shfl_f(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_f(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <typename T> __device__ __forceinline__ T shfl_c(T v, int src) {
  v.x = shfl_f(v.x, src);
  v.y = shfl_f(v.y, src);
  return v;
}
template <typename T> __device__ __forceinline__ T shfl_c_down(T v, int d) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, d);
  v.y = __shfl_down_sync(0xffffffffu, v.y, d);
  return v;
}

template <typename T> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

template <typename CT> struct Cfg;
// NB: inner panel width.  NBL: the narrower panel of the large-support-set variant, whose whole
// panel column block must still fit in shared memory for N up to several thousand.
template <> struct Cfg<float2> { static constexpr int NB = 16; static constexpr int NBL = 4; };
template <> struct Cfg<double2> { static constexpr int NB = 8; static constexpr int NBL = 2; };

// ------------------------------------------------------------------ activation (Eq. 3)
__global__ void __launch_bounds__(kThreads) activate_kernel(const int4* __restrict__ rules, int M,
                                                           const uint8_t* __restrict__ maps, int npix, int n_states, int via_top,
                                                           int32_t* __restrict__ idx, int32_t* __restrict__ n_act,
                                                           uint32_t* __restrict__ flags, int* __restrict__ n_max) {
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint8_t* map = maps + static_cast<size_t>(b) * npix;
  __shared__ int s_bad;
  __shared__ int s_warp[kWarps];
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int i = tid; i < npix; i += kThreads)
    if (map[i] >= n_states || (map[i] == 2 && i >= via_top)) s_bad = 1;
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      n_act[b] = -1;
      atomicOr(&flags[b], kFlagBadState);
    }
    return;
  }
  int32_t* out = idx + static_cast<size_t>(b) * M;
  int base = 0;
  for (int m0 = 0; m0 < M; m0 += kThreads) {
    const int m = m0 + tid;
    bool on = false;
    if (m < M) {
      const int4 r = __ldg(&rules[m]);
      switch (r.x) {
        case kAlways: on = true; break;
        case kInner: on = map[r.y] >= 1; break;
        case kInter: on = map[r.y] >= 1 && map[r.z] >= 1; break;
        case kPixPort: on = map[r.y] >= 1; break;
        case kViaStrip:
        case kViaJoin: on = map[r.y] == 2; break;
        case kViaLand: on = map[r.y] == 2 && map[r.z] >= 1; break;
        default: on = false;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int woff = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const int c = s_warp[w];
      woff += (w < warp) ? c : 0;
      total += c;
    }
    if (on) out[base + woff + before] = m;
    base += total;
    __syncthreads();
  }
  if (tid == 0) {
    n_act[b] = base;
    if (n_max) atomicMax(n_max, base);
  }
}

// ------------------------------------------------------------------ block argmax of |a|^2
template <typename R>
__device__ __forceinline__ int block_argmax(R v, int row, R* s_val, int* s_row) {
  const int lane = gtid() & 31, warp = gtid() >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const R ov = __shfl_down_sync(0xffffffffu, v, d);
    const int orow = __shfl_down_sync(0xffffffffu, row, d);
    if (ov > v || (ov == v && orow >= 0 && (row < 0 || orow < row))) { v = ov; row = orow; }
  }
  if (lane == 0) { s_val[warp] = v; s_row[warp] = row; }
  gsync();
  // every warp reduces the per-warp results itself (butterfly over groups of kWarps lanes): one
  // barrier per argmax; the callers' next barrier precedes any reuse of s_val / s_row
  R bv = s_val[lane & (kWarps - 1)];
  int br = s_row[lane & (kWarps - 1)];
#pragma unroll
  for (int d = kWarps / 2; d > 0; d >>= 1) {
    const R ov = __shfl_xor_sync(0xffffffffu, bv, d);
    const int orow = __shfl_xor_sync(0xffffffffu, br, d);
    if (ov > bv || (ov == bv && orow >= 0 && (br < 0 || orow < br))) { bv = ov; br = orow; }
  }
  return br;
}

// ------------------------------------------------------------------ tensor-core block updates
// The single-precision LU runs as a Crout (left-and-right-looking) blocked factorization over
// kOuter-column outer panels: before outer panel J is factored, its columns receive all earlier
// panels' contributions at once (column update, K = J kOuter), and after it is factored, its rows
// receive them to the right of the panel (row update, K = J kOuter) before its triangular solve.
// Each update is one long-K contraction per 128-row output tile, so the tile is read and written
// once per panel instead of once per earlier panel, and the tensor cores run long MMA streams.
//
// Operand pipeline of a task group, per K chunk (kChunk complex values = 16 real K):
//   raw stage   : the chunk's X and Y tiles copied from the task's workspace by two tensor copies
//                 (TMA boxes of the launch's tensor maps, issued by one thread, completion counted
//                 in bytes on the stage's mbarrier; kRaw chunks in flight, no registers held), rows
//                 padded against bank conflicts;
//   MMA stage   : the A operand (128 rows x 16, hi and lo TF32 parts) in tensor memory, written
//                 by the threads (one row each), and the B operand (128 x 16, hi and lo, canonical
//                 K-major layout) in shared memory; kStages of them, one MMA-completion mbarrier
//                 each.
// Shared memory of a group's staging area: [kRaw raw stages | kStages B stages].  TMEM columns:
// [0, 128) accumulator, [128 + 32 s, 160 + 32 s) A of MMA stage s (hi: +0..15, lo: +16..31).
constexpr int kRaw = 3;
constexpr int kStages = 3;
constexpr int kGatherBufs = 8;   // parent rows in flight in the bulk gather
constexpr int kChunk = 8;
// K chunks per accumulation segment: the tensor cores' fp32 accumulation over a long K loses more
// than round-to-nearest fp32 additions would, so each segment is added to C on its own in the
// epilogue.  Default layout: segments of 256 complex terms (1536 products per output with the
// three TF32 terms; one accumulation over K up to 640 needed 12 % more corrections, while 64-, 128-
// and 256-term segments measured the same).  Large-support-set layout: 1024 complex terms (K runs
// to about 4100 there; 1024-term segments took 7 % less time than 256-term ones at N = 4100 with
// the same corrections per task and no repaired task).
constexpr int kSegChunks = 32;
constexpr int kSegChunksLarge = 128;
constexpr uint32_t kRawXBytes = 10240;    // 128 rows x 80 B (column update) / 8 x 1024 B (row update)
constexpr uint32_t kRawBytes = 16384;     // + Y: 8 x 576 B (column update) / 64 x 96 B (row update)
constexpr uint32_t kStageBytes = 16384;   // B hi | B lo of one MMA stage
constexpr uint32_t kAccCols = 128;
// Tensor maps of the updates' operand tiles over a launch's workspace slots: 8-byte elements (one
// complex64 entry), dimensions {lda, ncap rows, slots}, strides {lda * 8, slot bytes}.  Boxes (columns
// x rows) reproduce the raw-stage layouts: column update X 10 x 128 (rows 80 bytes apart), Y 72 x 8
// (576 bytes), row update X 128 x 8 (1024 bytes), Y 12 x 64 (96 bytes); the extra columns land in
// the padding and are never read.
struct TmaMaps {
  CUtensorMap m[4];
};
enum : int { kMapColX = 0, kMapColY = 1, kMapRowX = 2, kMapRowY = 3 };
constexpr uint32_t kBoxW[4] = {10, 72, 128, 12};   // box columns (complex entries) per map
constexpr uint32_t kBoxH[4] = {128, 8, 8, 64};     // box rows per map
constexpr uint32_t box_bytes(int m) { return kBoxW[m] * kBoxH[m] * 8u; }
constexpr uint32_t kColBoxBytes = box_bytes(kMapColX) + box_bytes(kMapColY);   // X + Y of a column-update chunk
constexpr uint32_t kRowBoxBytes = box_bytes(kMapRowX) + box_bytes(kMapRowY);   // X + Y of a row-update chunk
static_assert(box_bytes(kMapColX) <= kRawXBytes && box_bytes(kMapRowX) <= kRawXBytes &&
                  box_bytes(kMapColY) <= kRawBytes - kRawXBytes && box_bytes(kMapRowY) <= kRawBytes - kRawXBytes,
              "a tensor-copy box overruns its raw-stage region");
static_assert(kRawXBytes % 128 == 0 && kRawBytes % 128 == 0, "tensor-copy destinations must stay 128-byte aligned");
static_assert(kBoxW[kMapColX] * 8 == 80 && kBoxW[kMapColY] * 8 == 576 && kBoxW[kMapRowX] * 8 == 1024 &&
                  kBoxW[kMapRowY] * 8 == 96,
              "box row pitches must match the raw-stage layouts the conversion reads");
struct TcState {
  unsigned char* stage;
  uint32_t tmem;
  uint64_t* mbar;     // [kStages]
  uint32_t sph;       // bit s: parity of the next completion awaited on stage s
  bool failed;
  int seg_chunks;     // K chunks per accumulation segment
  const TmaMaps* maps;   // operand tile maps of this launch
  int tz;                // the task's workspace slot (third map coordinate)
  uint64_t* rbar;        // [kRaw] completion of a raw stage's tensor copies
  uint32_t rph;          // bit r: parity of the next completion awaited on raw stage r
};
// bounded wait: 2^18 polls of mbarrier.try_wait (about 1 s at the measured 3.8 us per unanswered
// poll); a stall flags the task instead of hanging, a healthy completion answers in microseconds.
// Once a wait of the task has failed the later ones are skipped (the task is flagged already).
constexpr long long kTcWaitPolls = 1ll << 18;
constexpr int kTcCols = 128;                     // complex output columns per TMEM allocation half
constexpr uint32_t kTmemCols = 2 * kTcCols;      // TMEM columns per task group

__device__ __forceinline__ void stage_wait(TcState& st, int s) {
  if (!st.failed && !tc::mbar_wait(&st.mbar[s], (st.sph >> s) & 1u, kTcWaitPolls)) st.failed = true;
  st.sph ^= 1u << s;
  tc::fence_after_sync();
}

// hi + lo TF32 split of v stored at byte offset `off` of the hi and lo tiles
__device__ __forceinline__ void put_split16(unsigned char* hi, unsigned char* lo, uint32_t off, float v) {
  const float h = tc::to_tf32(v);
  *reinterpret_cast<float*>(hi + off) = h;
  *reinterpret_cast<float*>(lo + off) = tc::to_tf32(v - h);
}

// Complex update on the tensor cores, C -= X Y with K = K complex terms (K a multiple of kChunk).
// Column update (ROWG = false): C = A[r_out + i][c_out + j], i < m (128-row tiles), j < nc <= 64;
//   X = A[r_out + i][0:K] (L rows), Y = A[0:K][c_out + j] (U columns).
// Row update (ROWG = true), computed transposed so that the long dimension fills the MMA's rows:
//   C^T[i][j] = A[r_out + j][c_out + i], i < m (128-column tiles), j < nc <= 64;
//   X = A[0:K][c_out + i]^T (U columns), Y = A[r_out + j][0:K]^T (L rows).
// The complex product is realified as [Xr | Xi] (128 x 2K) times [[Yr, Yi], [-Yi, Yr]] (2K x 128),
// one M = 128, N = 128 MMA shape whose first 64 output columns are the real parts and last 64 the
// imaginary parts; X is negated while staged so TMEM accumulates -X Y.  Each fp32 operand is split
// into TF32 hi + lo and the three significant products (lo*hi, hi*lo, hi*hi) accumulate in fp32
// (3xTF32).  Iteration c of the chunk loop: the tensor copies of chunk c have landed; one
// barrier; one thread issues chunk c - 1's six MMAs (converted in the previous iteration) and
// commits them to its stage's mbarrier; the copies of chunk c + kRaw - 1 are issued into the raw
// stage chunk c - 1 used; chunk c is converted into MMA stage c % kStages once chunk
// c - kStages's MMAs have completed.  K runs in segments of st.seg_chunks chunks; after each the
// epilogue reads the accumulator row by row from TMEM and adds it to C in global memory.  The boxes
// are always full (128 rows or columns of X): entries outside the tile, stale workspace values or
// the zeros of the copy beyond the matrix, reach only accumulator rows and columns that are not
// stored.
template <bool ROWG>
__device__ void gemm_update_tc(float2* __restrict__ A, int lda, int r_out, int c_out, int m, int nc, int K,
                               TcState& st) {
  const int tid = gtid(), warp = tid >> 5, lane = tid & 31;
  const uint32_t idesc = tc::idesc_tf32(128, 128);
  const int nk = K / kChunk;
  // conversion slots: X -- this thread's TMEM lane (row xi of the tile) and K half (4 complex values
  // at 4 xh); Y -- two (k, j) elements, each warp covering 8 rows of the B tile x 4 K values
  // (conflict-free canonical-layout stores)
  const int q = warp & 3, xh = warp >> 2, xi = 32 * q + lane;
  const uint32_t lane_base = st.tmem + (static_cast<uint32_t>(32 * q) << 16);
  int yj[2], yk[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = tid + u * kThreads, ln = e & 31, wt = e >> 5;
    yj[u] = (wt & 7) * 8 + (ROWG ? (ln >> 2) : (ln & 7));
    yk[u] = (wt >> 3) * 4 + (ROWG ? (ln & 3) : (ln >> 3));
  }
  unsigned char* raw0 = st.stage;
  unsigned char* bst0 = st.stage + kRaw * kRawBytes;
  // the operands were written by this group's ordinary stores; the tensor copies read them through
  // the async proxy, so every writer orders its stores before them (proxy fence, then the barrier)
  asm volatile("fence.proxy.async.global;" ::: "memory");
  gsync();
  PMOM_PHASE_START(tg);
#ifdef PMOM_PHASES
  long long l_cp = 0, l_stw = 0, l_sync = 0, l_mma = 0, l_epi = 0, l_iss = 0, l_conv = 0;
#endif
  for (int t0 = 0; t0 < m; t0 += 128) {
    const int mt = min(128, m - t0);
    const bool xv = xi < mt;
    // chunk c's X and Y tiles: two tensor copies into raw stage c % kRaw, issued by thread 0 and
    // counted in bytes on that stage's barrier
    auto issue = [&](int c) {
      if (tid != 0) return;
      const int r = c % kRaw, kb = c * kChunk;
      unsigned char* rx = raw0 + r * kRawBytes;
      unsigned char* ry = rx + kRawXBytes;
      const int mx = ROWG ? kMapRowX : kMapColX, my = ROWG ? kMapRowY : kMapColY;
      tc::mbar_arrive_expect_tx(&st.rbar[r], ROWG ? kRowBoxBytes : kColBoxBytes);
      if (ROWG) {   // X[k][i] = A[kb + k][c_out + t0 + i], Y[j][k] = A[r_out + j][kb + k]
        tc::tma_load_3d(rx, &st.maps->m[mx], c_out + t0, kb, st.tz, &st.rbar[r]);
        tc::tma_load_3d(ry, &st.maps->m[my], kb, r_out, st.tz, &st.rbar[r]);
      } else {      // X[i][k] = A[r_out + t0 + i][kb + k], Y[k][j] = A[kb + k][c_out + j]
        tc::tma_load_3d(rx, &st.maps->m[mx], kb, r_out + t0, st.tz, &st.rbar[r]);
        tc::tma_load_3d(ry, &st.maps->m[my], c_out, kb, st.tz, &st.rbar[r]);
      }
    };
    // chunk c's tiles have landed (every thread waits, in chunk order)
    auto raw_wait = [&](int c) {
      const int r = c % kRaw;
      if (!st.failed && !tc::mbar_wait(&st.rbar[r], (st.rph >> r) & 1u, kTcWaitPolls)) st.failed = true;
      st.rph ^= 1u << r;
    };
    // MMA completions are consumed in chunk order: 0 .. waited
    int waited = -1;
    auto wait_chunk = [&](int x) {
      while (waited < x) {
        ++waited;
        stage_wait(st, waited % kStages);
      }
    };
    // segment epilogue: this thread's accumulator row (TMEM lane xi), complex columns 32 xh ..
    // 32 xh + 31, in two halves of 16, added to C with independent loads in flight
    auto epilogue = [&]() {
#pragma unroll 1
      for (int hh = 0; hh < 2; ++hh) {
        const int j0 = 32 * xh + 16 * hh;
        float re[16], im[16];
        tc::tmem_ld16(lane_base + j0, re);
        tc::tmem_ld16(lane_base + 64 + j0, im);
        if constexpr (!ROWG) {
          // column update: a thread's 16 outputs lie in one row of C, so lane-per-row accesses
          // would touch 32 rows per warp access.  Each warp passes its 32 x 16 block through a
          // padded shared-memory block instead (in the B stages, idle once the segment's MMAs are
          // complete) and moves C in 128-byte row pieces: lane l takes row 4 rr + l / 8 of the
          // warp's 32 and complex columns 2 (l % 8), 2 (l % 8) + 1 (16-byte aligned: lda, c_out
          // and j0 are even).  C is loaded before the accumulator is staged.
          float2* scr = reinterpret_cast<float2*>(bst0) + warp * (32 * 17);
          const int rl = lane >> 3, cp = 2 * (lane & 7), jc = j0 + cp;
          float4 v4[8];
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) {
            const int xr = 32 * q + 4 * rr + rl;
            const float2* crow = A + static_cast<size_t>(r_out + t0 + xr) * lda + c_out + jc;
            if (xr < mt && jc + 1 < nc) v4[rr] = *reinterpret_cast<const float4*>(crow);
            else if (xr < mt && jc < nc) v4[rr] = make_float4(crow[0].x, crow[0].y, 0.f, 0.f);
            else v4[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) scr[lane * 17 + u] = make_float2(re[u], im[u]);
          __syncwarp();
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) {
            const int row = 4 * rr + rl, xr = 32 * q + row;
            const float2 a0 = scr[row * 17 + cp], a1 = scr[row * 17 + cp + 1];
            float2* crow = A + static_cast<size_t>(r_out + t0 + xr) * lda + c_out + jc;
            if (xr < mt && jc + 1 < nc)
              *reinterpret_cast<float4*>(crow) = make_float4(v4[rr].x + a0.x, v4[rr].y + a0.y, v4[rr].z + a1.x, v4[rr].w + a1.y);
            else if (xr < mt && jc < nc)
              crow[0] = make_float2(v4[rr].x + a0.x, v4[rr].y + a0.y);
          }
          __syncwarp();   // the block is rewritten by the second half
        } else {
          // row update: C^T[xi][j] = A[r_out + j][c_out + t0 + xi], so for each j the warp's lanes
          // touch consecutive columns of one row of A
          float2 v[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int j = j0 + u;
            const size_t o = static_cast<size_t>(r_out + j) * lda + c_out + t0 + xi;
            v[u] = (xv && j < nc) ? A[o] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int j = j0 + u;
            if (xv && j < nc) A[static_cast<size_t>(r_out + j) * lda + c_out + t0 + xi] = make_float2(v[u].x + re[u], v[u].y + im[u]);
          }
        }
      }
    };
#pragma unroll
    for (int p = 0; p < kRaw - 1; ++p)
      if (p < nk) issue(p);
    PMOM_LAP(l_iss, tg);
    for (int c = 0; c <= nk; ++c) {
      if (c < nk) {
        raw_wait(c);
        PMOM_LAP(l_cp, tg);
        if (c >= kStages) wait_chunk(c - kStages);   // chunk c - kStages's MMAs have read stage c % kStages
        PMOM_LAP(l_stw, tg);
      }
      tc::tmem_wait_st();
      tc::fence_async_smem();
      tc::fence_before_sync();
      gsync();
      tc::fence_after_sync();
      PMOM_LAP(l_sync, tg);
      if (c > 0) {
        if (tid == 0) {
          const int s1 = (c - 1) % kStages;
          const uint32_t xa = st.tmem + kAccCols + 32 * s1;
          const uint32_t bh = tc::smem_u32(bst0 + s1 * kStageBytes), bl = bh + 8192;
          uint32_t acc = (c - 1) % st.seg_chunks != 0 ? 1u : 0u;   // a new segment starts from zero
#pragma unroll
          for (int term = 0; term < 3; ++term) {
            const uint32_t ao = xa + (term == 0 ? 16u : 0u);   // small terms first: lo*hi, hi*lo, hi*hi
            const uint32_t bo = term == 1 ? bl : bh;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              tc::mma_tf32_ts(st.tmem, ao + 8 * ks, tc::smem_desc16(bo + ks * 256), idesc, acc);
              acc = 1;
            }
          }
          tc::commit(&st.mbar[s1]);
        }
        PMOM_LAP(l_mma, tg);
        // end of a segment: its accumulator added to C (the next segment's copies stay in flight;
        // its first MMA waits for the barrier of the next iteration, after these TMEM reads)
        if ((c - 1) % st.seg_chunks == st.seg_chunks - 1 || c == nk) {
          wait_chunk(c - 1);
          epilogue();
          tc::fence_before_sync();
          if constexpr (!ROWG) gsync();   // the transpose blocks are free before stage c % kStages is written
        }
        PMOM_LAP(l_epi, tg);
      }
      if (c == nk) break;
      if (c + kRaw - 1 < nk) issue(c + kRaw - 1);   // into the raw stage chunk c - 1 used
      PMOM_LAP(l_iss, tg);
      if (c >= kStages) wait_chunk(c - kStages);   // (consumed above unless a segment ended)
      PMOM_LAP(l_stw, tg);
      // convert chunk c: X -> TMEM (negated, split; real parts at K columns 4 xh + u, imaginary at
      // 8 + 4 xh + u), Y -> canonical B tile
      const int s = c % kStages;
      const unsigned char* rx = raw0 + (c % kRaw) * kRawBytes;
      const unsigned char* ry = rx + kRawXBytes;
      {
        float2 x[4];
        if (ROWG) {
#pragma unroll
          for (int u = 0; u < 4; ++u) x[u] = *reinterpret_cast<const float2*>(rx + (4 * xh + u) * 1024 + xi * 8);
        } else {
          const float4 a = *reinterpret_cast<const float4*>(rx + xi * 80 + xh * 32);
          const float4 b = *reinterpret_cast<const float4*>(rx + xi * 80 + xh * 32 + 16);
          x[0] = make_float2(a.x, a.y); x[1] = make_float2(a.z, a.w);
          x[2] = make_float2(b.x, b.y); x[3] = make_float2(b.z, b.w);
        }
        float hr[4], lr[4], hi[4], li[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float re = -x[u].x, im = -x[u].y;
          hr[u] = tc::to_tf32(re); lr[u] = tc::to_tf32(re - hr[u]);
          hi[u] = tc::to_tf32(im); li[u] = tc::to_tf32(im - hi[u]);
        }
        const uint32_t col = lane_base + kAccCols + 32 * s + 4 * xh;
        tc::tmem_st4(col, hr[0], hr[1], hr[2], hr[3]);
        tc::tmem_st4(col + 8, hi[0], hi[1], hi[2], hi[3]);
        tc::tmem_st4(col + 16, lr[0], lr[1], lr[2], lr[3]);
        tc::tmem_st4(col + 24, li[0], li[1], li[2], li[3]);
      }
      unsigned char* yh = bst0 + s * kStageBytes;
      unsigned char* yl = yh + 8192;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 y = *reinterpret_cast<const float2*>(ROWG ? ry + yj[u] * 96 + yk[u] * 8 : ry + yk[u] * 576 + yj[u] * 8);
        put_split16(yh, yl, tc::kmajor16_off(yj[u], yk[u]), y.x);
        put_split16(yh, yl, tc::kmajor16_off(yj[u], kChunk + yk[u]), -y.y);
        put_split16(yh, yl, tc::kmajor16_off(64 + yj[u], yk[u]), y.y);
        put_split16(yh, yl, tc::kmajor16_off(64 + yj[u], kChunk + yk[u]), y.x);
      }
      PMOM_LAP(l_conv, tg);
    }
    // the accumulator is read and the staging area is free before the next tile starts (every
    // issued copy has been waited for)
    gsync();
    PMOM_LAP(l_sync, tg);
  }
#ifdef PMOM_PHASES
  PMOM_LAP_FLUSH(kPhGemmCopyWait, l_cp);
  PMOM_LAP_FLUSH(kPhGemmStageWait, l_stw);
  PMOM_LAP_FLUSH(kPhGemmSync, l_sync);
  PMOM_LAP_FLUSH(kPhGemmMma, l_mma);
  PMOM_LAP_FLUSH(kPhGemmEpi, l_epi);
  PMOM_LAP_FLUSH(kPhGemmIssue, l_iss);
  PMOM_LAP_FLUSH(kPhGemmConv, l_conv);
#endif
}

// U12 = L11^-1 A12 for an outer panel: L11 = unit lower A[j0..j0+jb, j0..j0+jb) (jb <= 64, staged in
// shared memory), A12 = A[j0..j0+jb, cb..N); one column per thread, 16 rows at a time.
__device__ void outer_trsm(float2* __restrict__ A, int lda, int N, int j0, int jb, float2* __restrict__ Ls) {
  constexpr int LDL = 65;
  const int tid = gtid(), cb = j0 + jb;
  for (int e = tid; e < jb * 64; e += kThreads) {
    const int r = e >> 6, c = e & 63;
    Ls[r * LDL + c] = c < jb ? A[static_cast<size_t>(j0 + r) * lda + j0 + c] : make_float2(0.f, 0.f);
  }
  gsync();
  for (int c = cb + tid; c < N; c += kThreads) {
    for (int ch = 0; ch * 16 < jb; ++ch) {
      const int rw = min(16, jb - 16 * ch);
      float2 u[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) u[i] = i < rw ? A[static_cast<size_t>(j0 + 16 * ch + i) * lda + c] : make_float2(0.f, 0.f);
      for (int t = 0; t < 16 * ch; t += 4) {   // contributions of the rows already solved, four at a time
        float2 y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) y[k] = A[static_cast<size_t>(j0 + t + k) * lda + c];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int i = 0; i < 16; ++i) u[i] = cfms(Ls[(16 * ch + i) * LDL + t + k], y[k], u[i]);
      }
#pragma unroll
      for (int i = 1; i < 16; ++i)
#pragma unroll
        for (int t = 0; t < i; ++t) u[i] = cfms(Ls[(16 * ch + i) * LDL + 16 * ch + t], u[t], u[i]);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (i < rw) A[static_cast<size_t>(j0 + 16 * ch + i) * lda + c] = u[i];
    }
  }
  gsync();
}

// Trailing update of an NB-column panel on the CUDA cores: A[r_begin:N, r_begin:cend] -= L21 U12,
// L21 = the panel's rows below it (shared memory, leading dimension NB + 1), U12 = A[k0:k0+kb,
// r_begin:cend], in tiles of (1024 / TW) rows x TW columns, 4 x 4 complex outputs per thread.  TW
// follows the columns left to update (within an outer panel of 64 they shrink to 48, 32 and 16),
// so no thread computes columns that are not stored.
template <typename CT, int NB, int TW>
__device__ void inner_trailing(CT* __restrict__ A, int lda, const CT* __restrict__ Pn, CT* __restrict__ Ut, int k0,
                               int kb, int r_begin, int n2, int cend) {
  constexpr int LDP = NB + 1;
  constexpr int LDU = kTile + 1;
  constexpr int TX = TW / 4;                // threads across a tile's columns
  constexpr int TR = 4 * (kThreads / TX);   // tile rows
  static_assert(TW <= kTile && kThreads % TX == 0, "tile wider than the U12 staging block");
  const int tid = gtid(), ty = tid / TX, tx = tid % TX;
  const int ntile = (n2 + TR - 1) / TR;
  const int ntile_c = (cend - r_begin + TW - 1) / TW;
  for (int tc = 0; tc < ntile_c; ++tc) {
    const int c0 = r_begin + tc * TW;
#pragma unroll
    for (int e0 = 0; e0 < NB * TW; e0 += kThreads) {   // compile-time trip count: loads in flight together
      const int e = e0 + tid, t = e / TW, cc = e % TW;
      if (e < NB * TW)
        Ut[t * LDU + cc] = (t < kb && c0 + cc < cend) ? A[static_cast<size_t>(k0 + t) * lda + c0 + cc] : czero(Ut[0]);
    }
    gsync();
    for (int tr = 0; tr < ntile; ++tr) {
      const int r0 = tr * TR;   // relative to r_begin
      CT acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int r = r0 + ty + (TR / 4) * i, c = c0 + tx + TX * jj;
          acc[i][jj] = (r < n2 && c < cend) ? A[static_cast<size_t>(r_begin + r) * lda + c] : czero(acc[0][0]);
        }
#pragma unroll 4
      for (int t = 0; t < NB; ++t) {
        if (t >= kb) break;
        CT a[4], u[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = r0 + ty + (TR / 4) * i;
          a[i] = r < n2 ? Pn[(kb + r) * LDP + t] : czero(a[0]);
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) u[jj] = Ut[t * LDU + tx + TX * jj];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) acc[i][jj] = cfms(a[i], u[jj], acc[i][jj]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int r = r0 + ty + (TR / 4) * i, c = c0 + tx + TX * jj;
          if (r < n2 && c < cend) A[static_cast<size_t>(r_begin + r) * lda + c] = acc[i][jj];
        }
    }
    gsync();
  }
}

// ------------------------------------------------------------------ blocked LU in global memory
// A: row-major N x N (leading dimension lda).  Panel of NB columns factored in shared memory;
// row interchanges applied to whole rows (LAPACK convention: P A = L U, unit-diagonal L).
// Returns true if an exactly zero pivot occurred.
template <typename CT, int NB>
__device__ bool lu_factor(CT* __restrict__ A, int lda, int N, int* __restrict__ piv, CT* __restrict__ Pn,
                          CT* __restrict__ Ut, typename Real<CT>::type* s_val, int* s_row, TcState* tcs) {
  using R = typename Real<CT>::type;
  constexpr int LDP = NB + 1;
  constexpr int LDU = kTile + 1;
  const int tid = gtid();
  bool singular = false;
  // Updates made by each NB-column panel stop at column `cend`: N for the one-level CUDA-core
  // path; the end of the current kOuter-column outer panel for the two-level tensor-core path
  int cend = N;
  PMOM_PHASE_START(tph);
  for (int k0 = 0; k0 < N; k0 += NB) {
    const int kb = min(NB, N - k0);
    const int nr = N - k0;
    if (tcs != nullptr && k0 % kOuter == 0) {
      cend = min(N, k0 + kOuter);
      if constexpr (std::is_same<CT, float2>::value) {
        // Crout column update of the new outer panel: A[k0:N, k0:cend] -= L[k0:N, 0:k0] U[0:k0, k0:cend]
        if (k0 > 0) gemm_update_tc<false>(A, lda, k0, k0, N - k0, cend - k0, k0, *tcs);
      }
      PMOM_PHASE(kPhColGemm, tph);
    }
    // 1. panel -> shared memory (eight independent loads in flight per thread)
    for (int e0 = tid; e0 < nr * NB; e0 += 8 * kThreads) {
      CT v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * kThreads, r = e / NB, c = e % NB;
        v[u] = (e < nr * NB && c < kb) ? A[static_cast<size_t>(k0 + r) * lda + k0 + c] : czero(v[0]);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * kThreads, r = e / NB, c = e % NB;
        if (e < nr * NB && c < kb) Pn[r * LDP + c] = v[u];
      }
    }
    gsync();
    PMOM_PHASE(kPhPanelLoad, tph);
    // 2. factor the panel (partial pivoting on |a|^2, ties to the lowest row), one barrier per
    //    column: each warp publishes its best candidate row for the next column (value, index and
    //    the whole row) in a double-buffered slot; after the barrier every thread picks the pivot
    //    from the slots and updates the rows it owns (row r belongs to thread r mod kThreads), the
    //    owner of row j swapping: it writes the pivot row (from the slot) into row j and its own
    //    old row, updated, into row p, which nobody else touches in that column.
    {
      CT* cdat = Ut;                                            // [2][kWarps][NB]
      R* cval = reinterpret_cast<R*>(Ut + 2 * kWarps * NB);     // [2][kWarps]
      int* crow = reinterpret_cast<int*>(cval + 2 * kWarps);    // [2][kWarps]
      const int lane = tid & 31, warp = tid >> 5;
      // publish this warp's best candidate (v, r) into slot parity `par`
      auto publish = [&](R v, int r, int par) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          const R ov = __shfl_xor_sync(0xffffffffu, v, d);
          const int orow = __shfl_xor_sync(0xffffffffu, r, d);
          if (ov > v || (ov == v && orow >= 0 && (r < 0 || orow < r))) { v = ov; r = orow; }
        }
        if (lane == 0) {
          cval[par * kWarps + warp] = v;
          crow[par * kWarps + warp] = r;
        }
        __syncwarp();   // the winning row was written by a lane of this warp
        if (r >= 0 && lane < NB) cdat[(par * kWarps + warp) * NB + lane] = Pn[r * LDP + lane];
      };
      R best = -1;
      int brow = -1;
      for (int r = tid; r < nr; r += kThreads) {
        const R v = cabs2(Pn[r * LDP]);
        if (v > best) { best = v; brow = r; }
      }
      publish(best, brow, 0);
      PMOM_PHASE_START(tpc);
#ifdef PMOM_PHASES
      long long l_work = 0, l_wait = 0;
#endif
      for (int j = 0; j < kb; ++j) {
        const int par = j & 1;
        PMOM_LAP(l_work, tpc);
        gsync();
        PMOM_LAP(l_wait, tpc);
        R pv = -1;
        int p = -1, pw = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const R v = cval[par * kWarps + w];
          const int r = crow[par * kWarps + w];
          if (r >= 0 && (v > pv || (v == pv && (p < 0 || r < p)))) { pv = v; p = r; pw = w; }
        }
        const CT* prow = cdat + (par * kWarps + pw) * NB;
        if (p < 0) {   // no comparable candidate (non-finite column): no interchange, flagged singular
          p = j;
          prow = Pn + j * LDP;
          singular = true;
        }
        if (tid == 0) piv[k0 + j] = k0 + p;
        const CT d = prow[j];
        const bool zero = cabs2(d) == R(0);
        if (zero) singular = true;
        const CT inv = zero ? czero(d) : cinv(d);
        best = -1;
        brow = -1;
        // rows below the pivot that this thread owns (row p moves to the owner of row j); only the
        // panel's columns right of j are touched (the pivot row's entries read from the slot)
        for (int r = j + 1 + ((tid - j - 1) & (kThreads - 1)); r < nr; r += kThreads) {
          if (r == p) continue;
          CT* row = Pn + r * LDP;
          const CT l = cmul(row[j], inv);
          row[j] = l;
          for (int c = j + 1; c < kb; ++c) row[c] = cfms(l, prow[c], row[c]);
          if (j + 1 < kb) {
            const R v = cabs2(row[j + 1]);
            if (v > best || (v == best && r < brow)) { best = v; brow = r; }
          }
        }
        if (p != j && tid == (j & (kThreads - 1))) {
          // the swap: the pivot row into row j, this thread's old row j (updated) into row p
          CT o[NB];
#pragma unroll
          for (int c = 0; c < NB; ++c) o[c] = c < kb ? Pn[j * LDP + c] : czero(d);
#pragma unroll
          for (int c = 0; c < NB; ++c)
            if (c < kb) Pn[j * LDP + c] = prow[c];
#pragma unroll
          for (int c = 0; c < NB; ++c)
            if (c == j) o[c] = cmul(o[c], inv);
          CT lj = czero(d);
#pragma unroll
          for (int c = 0; c < NB; ++c)
            if (c == j) lj = o[c];
#pragma unroll
          for (int c = 0; c < NB; ++c)
            if (c > j && c < kb) o[c] = cfms(lj, prow[c], o[c]);
#pragma unroll
          for (int c = 0; c < NB; ++c)
            if (c < kb) Pn[p * LDP + c] = o[c];
          if (j + 1 < kb) {
            R v = R(0);
#pragma unroll
            for (int c = 0; c < NB; ++c)
              if (c == j + 1) v = cabs2(o[c]);
            if (v > best || (v == best && p < brow)) { best = v; brow = p; }
          }
        }
        if (j + 1 < kb) publish(best, brow, par ^ 1);
      }
      gsync();
#ifdef PMOM_PHASES
      PMOM_LAP_FLUSH(kPhPanelWork, l_work);
      PMOM_LAP_FLUSH(kPhPanelWait, l_wait);
#endif
    }
    PMOM_PHASE(kPhPanelFactor, tph);
    // 3. panel back to global memory
    for (int e = tid; e < nr * NB; e += kThreads) {
      const int r = e / NB, c = e % NB;
      if (c < kb) A[static_cast<size_t>(k0 + r) * lda + k0 + c] = Pn[r * LDP + c];
    }
    PMOM_PHASE(kPhPanel, tph);
    // 4. the panel's row interchanges on the columns outside it (a barrier only after an actual
    //    interchange: the pivot is usually the diagonal row); four columns per thread in flight
    for (int j = 0; j < kb; ++j) {
      const int p = piv[k0 + j];
      if (p != k0 + j) {
        CT* ra = A + static_cast<size_t>(k0 + j) * lda;
        CT* rb = A + static_cast<size_t>(p) * lda;
        for (int c0 = tid; c0 < N; c0 += 4 * kThreads) {
          CT va[4], vb[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * kThreads;
            const bool mv = c < N && (c < k0 || c >= k0 + kb);
            va[u] = mv ? ra[c] : czero(va[0]);
            vb[u] = mv ? rb[c] : czero(vb[0]);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * kThreads;
            if (c < N && (c < k0 || c >= k0 + kb)) {
              ra[c] = vb[u];
              rb[c] = va[u];
            }
          }
        }
        gsync();
      }
    }
    gsync();
    PMOM_PHASE(kPhSwap, tph);
    // 5. U12 = L11^-1 A12 (one column per thread, unit lower L11 from shared memory), columns up
    //    to the end of the current outer panel
    for (int c = k0 + kb + tid; c < cend; c += kThreads) {
      CT u[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) u[i] = i < kb ? A[static_cast<size_t>(k0 + i) * lda + c] : czero(u[0]);
#pragma unroll
      for (int i = 1; i < NB; ++i)
#pragma unroll
        for (int t = 0; t < i; ++t) u[i] = cfms(Pn[i * LDP + t], u[t], u[i]);
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < kb) A[static_cast<size_t>(k0 + i) * lda + c] = u[i];
    }
    gsync();
    PMOM_PHASE(kPhInnerU, tph);
    // 6. trailing update A22 -= L21 U12 on the CUDA cores, for the columns up to the end of the
    //    current outer panel (the tile as wide as the columns left to update, up to 64)
    const int r_begin = k0 + kb, n2 = N - r_begin;
    if (n2 > 0 && cend > r_begin) {
      const int w = cend - r_begin;
      if (w <= 16) inner_trailing<CT, NB, 16>(A, lda, Pn, Ut, k0, kb, r_begin, n2, cend);
      else if (w <= 32) inner_trailing<CT, NB, 32>(A, lda, Pn, Ut, k0, kb, r_begin, n2, cend);
      else inner_trailing<CT, NB, 64>(A, lda, Pn, Ut, k0, kb, r_begin, n2, cend);
    }
    gsync();
    PMOM_PHASE(kPhInnerUpd, tph);
    // 7-8. end of an outer panel (tensor-core path): the Crout row update of its rows to the right
    //      of the panel, A[j0:cend, cend:N] -= L[j0:cend, 0:j0] U[0:j0, cend:N], then U12 of those
    //      rows (the rows below receive these panels' contributions in their own column updates)
    if constexpr (std::is_same<CT, float2>::value) {
      if (tcs != nullptr && k0 + kb == cend && cend < N) {
        const int j0 = cend - ((cend - 1) % kOuter + 1);
        if (j0 > 0) gemm_update_tc<true>(A, lda, j0, cend, N - cend, cend - j0, j0, *tcs);
        PMOM_PHASE(kPhRowGemm, tph);
        outer_trsm(A, lda, N, j0, cend - j0, reinterpret_cast<float2*>(tcs->stage));
        PMOM_PHASE(kPhTrsm, tph);
      }
    }
  }
  return singular;
}

// ------------------------------------------------------------------ diagonal-block inverses
// After lu_factor: each 32 x 32 diagonal block of the packed factors (unit lower L_bb below the
// diagonal, U_bb on and above it) is replaced by the packed inverses (L_bb^-1 strictly below the
// diagonal, its unit diagonal implicit; U_bb^-1 on and above it), so every later triangular solve
// turns each diagonal step into an independent triangular matrix-vector product instead of a
// 32-step dependent chain.  The factors serve every refinement solve of a task, so the inversion
// is paid once.  D: the group's 32 x 33 staging block.  Each block is inverted by halves: with
// L = [[L11, 0], [L21, L22]] and U = [[U11, U12], [0, U22]] (16 x 16 sub-blocks),
//   L^-1 = [[L11^-1, 0], [-L22^-1 L21 L11^-1, L22^-1]],  U^-1 = [[U11^-1, -U11^-1 U12 U22^-1], [0, U22^-1]].
// Warps 0-3 invert L11, L22, U11, U22 in place (lane c forms column c by substitution, rows in
// lockstep, each row read before any lane overwrites it; the four touch disjoint entries of D),
// then the whole group forms the two off-diagonal blocks as 16 x 16 products, one output of each
// per thread.  A zero pivot gets a zero inverse (the task is flagged singular by lu_factor).
template <typename CT>
__device__ void lu_invert_diag(CT* __restrict__ A, int lda, int N, CT* __restrict__ D) {
  constexpr int LD = 33;
  const int tid = gtid(), lane = tid & 31, warp = tid >> 5;
  for (int i0 = 0; i0 < N; i0 += 32) {
    const int bs = min(32, N - i0);
    const int h1 = min(16, bs), h2 = bs - h1;   // sizes of the two diagonal sub-blocks
    for (int e = tid; e < 32 * 32; e += kThreads) {
      const int r = e >> 5, c = e & 31;
      if (r < bs && c < bs) D[r * LD + c] = A[static_cast<size_t>(i0 + r) * lda + i0 + c];
    }
    gsync();
    if (warp < 4) {
      const int off = (warp & 1) ? 16 : 0, n = (warp & 1) ? h2 : h1, c = lane;
      CT* Db = D + off * LD + off;
      if (warp < 2) {
        // column c of the unit lower inverse: x_c = 1, x_r = -sum_{t=c}^{r-1} L[r][t] x_t for r > c
        for (int r = 1; r < n; ++r) {
          CT acc = czero(D[0]);
          if (c < r) {
            acc = Db[r * LD + c];
#pragma unroll
            for (int t = 1; t < 16; ++t)
              if (t > c && t < r) acc = cfma(Db[r * LD + t], Db[t * LD + c], acc);
            acc.x = -acc.x;
            acc.y = -acc.y;
          }
          __syncwarp();
          if (c < r) Db[r * LD + c] = acc;
          __syncwarp();
        }
      } else {
        // column c of the upper inverse: x_c = 1/u_cc, x_r = -(sum_{t=r+1}^{c} U[r][t] x_t) / u_rr for r < c
        CT dinv = czero(D[0]);
        if (c < n) {
          const CT d = Db[c * LD + c];
          if (cabs2(d) > 0) dinv = cinv(d);
        }
        __syncwarp();
        if (c < n) Db[c * LD + c] = dinv;
        __syncwarp();
        for (int r = n - 2; r >= 0; --r) {
          CT ir;
          ir.x = __shfl_sync(0xffffffffu, dinv.x, r);
          ir.y = __shfl_sync(0xffffffffu, dinv.y, r);
          CT acc = czero(D[0]);
          if (c > r && c < n) {
#pragma unroll
            for (int t = 1; t < 16; ++t)
              if (t > r && t <= c) acc = cfma(Db[r * LD + t], Db[t * LD + c], acc);
            acc = cmul(acc, ir);
            acc.x = -acc.x;
            acc.y = -acc.y;
          }
          __syncwarp();
          if (c > r && c < n) Db[r * LD + c] = acc;
          __syncwarp();
        }
      }
    }
    gsync();
    if (h2 > 0) {
      // T_L = L21 L11^-1 and T_U = U12 U22^-1 (row i, column j), then L21 <- -L22^-1 T_L and
      // U12 <- -U11^-1 T_U
      const int i = tid >> 4, j = tid & 15;
      CT tl = czero(D[0]), tu = czero(D[0]);
      if (i < h2) {
        tl = D[(16 + i) * LD + j];
#pragma unroll
        for (int t = 1; t < 16; ++t)
          if (t > j) tl = cfma(D[(16 + i) * LD + t], D[t * LD + j], tl);
      }
      if (j < h2) {
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (t <= j) tu = cfma(D[i * LD + 16 + t], D[(16 + t) * LD + 16 + j], tu);
      }
      gsync();
      if (i < h2) D[(16 + i) * LD + j] = tl;
      if (j < h2) D[i * LD + 16 + j] = tu;
      gsync();
      if (i < h2) {
        CT a = D[(16 + i) * LD + j];
#pragma unroll
        for (int t = 0; t < 15; ++t)
          if (t < i) a = cfma(D[(16 + i) * LD + 16 + t], D[(16 + t) * LD + j], a);
        tl = make_neg(a);
      }
      if (j < h2) {
        CT a = czero(D[0]);
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (t >= i) a = cfma(D[i * LD + t], D[t * LD + 16 + j], a);
        tu = make_neg(a);
      }
      gsync();
      if (i < h2) D[(16 + i) * LD + j] = tl;
      if (j < h2) D[i * LD + 16 + j] = tu;
    }
    gsync();
    for (int e = tid; e < 32 * 32; e += kThreads) {
      const int r = e >> 5, cc = e & 31;
      if (r < bs && cc < bs) A[static_cast<size_t>(i0 + r) * lda + i0 + cc] = D[r * LD + cc];
    }
    gsync();
  }
}

// The row permutation of the pivots (interchanges k <-> piv[k] applied in order): row k of P b is
// row perm[k] of b.  One thread walks the interchanges in shared memory (scratch: 2 N ints), the
// group copies the result out.
__device__ void pivots_to_perm(const int* __restrict__ piv, int N, int* __restrict__ scratch, int* __restrict__ perm) {
  const int tid = gtid();
  for (int k = tid; k < N; k += kThreads) {
    scratch[k] = k;
    scratch[N + k] = piv[k];
  }
  gsync();
  if (tid == 0) {
    for (int k = 0; k < N; ++k) {
      const int p = scratch[N + k];
      if (p != k) {
        const int t = scratch[k];
        scratch[k] = scratch[p];
        scratch[p] = t;
      }
    }
  }
  gsync();
  for (int k = tid; k < N; k += kThreads) perm[k] = scratch[k];
  gsync();
}

// ------------------------------------------------------------------ triangular solves
// W (shared, N x P) holds the right-hand sides on entry and the solution on exit.
// D: shared 32 x 33 staging of the current diagonal block (read once, coalesced).
// W[i] -= sum over t in [tb, te) of A[i][t] W[t] for the rows i0 .. i0 + bs - 1 of a solve
// block (all P right-hand sides).  Each warp takes RW rows at once, lanes over t, two column
// steps per iteration: 2 RW independent loads in flight, and each W load serves RW rows.
template <typename CT>
__device__ __forceinline__ void offdiag_update(const CT* __restrict__ A, int lda, int i0, int bs, int tb, int te,
                                               CT* __restrict__ W, int P, int ldw) {
  constexpr int RW = sizeof(CT) == sizeof(float2) ? 4 : 2;
  const int tid = gtid(), lane = tid & 31, warp = tid >> 5;
  for (int ii0 = warp; ii0 < bs; ii0 += kWarps * RW) {
    CT acc[RW][kMaxPorts];
    const CT* row[RW];
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const int ii = ii0 + q * kWarps;
      row[q] = A + static_cast<size_t>(i0 + (ii < bs ? ii : ii0)) * lda;   // rows past the block reread ii0
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p) acc[q][p] = czero(acc[0][0]);
    }
    int t = tb + lane;
    for (; t + 32 < te; t += 64) {
      CT l0[RW], l1[RW];
#pragma unroll
      for (int q = 0; q < RW; ++q) {
        l0[q] = row[q][t];
        l1[q] = row[q][t + 32];
      }
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p) {
        if (p < P) {
          const CT w0 = W[t * ldw + p], w1 = W[(t + 32) * ldw + p];
#pragma unroll
          for (int q = 0; q < RW; ++q) {
            acc[q][p] = cfms(l0[q], w0, acc[q][p]);
            acc[q][p] = cfms(l1[q], w1, acc[q][p]);
          }
        }
      }
    }
    if (t < te) {
      CT l0[RW];
#pragma unroll
      for (int q = 0; q < RW; ++q) l0[q] = row[q][t];
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p) {
        if (p < P) {
          const CT w0 = W[t * ldw + p];
#pragma unroll
          for (int q = 0; q < RW; ++q) acc[q][p] = cfms(l0[q], w0, acc[q][p]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const int ii = ii0 + q * kWarps;
      if (ii >= bs) break;
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p) {
        if (p >= P) break;
        CT v = acc[q][p];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          const CT o = shfl_c_down(v, d);
          v.x += o.x;
          v.y += o.y;
        }
        if (lane == 0) {
          CT w = W[(i0 + ii) * ldw + p];
          w.x += v.x;   // acc holds -sum, so adding applies the subtraction
          w.y += v.y;
          W[(i0 + ii) * ldw + p] = w;
        }
      }
    }
  }
}

template <typename CT>
__device__ void lu_solve(const CT* __restrict__ A, int lda, int N, const int* __restrict__ piv, CT* __restrict__ W,
                         int P, CT* __restrict__ D, int ldw = 0, bool permuted = false, int fwd_from = 0) {
  // A: packed factors with inverted diagonal blocks (lu_invert_diag).  ldw: row stride of W (>= P;
  // an odd stride keeps the right-hand sides of consecutive rows in distinct shared-memory banks
  // when P is even).  permuted: W already holds P b (the caller applied the interchanges).
  // fwd_from: rows of P b above it are zero (so are those of y = L^-1 P b, L being unit lower
  // triangular): the forward pass starts at its 32-row block and takes no products with the
  // zero part of y.
  if (ldw < P) ldw = P;
  const int tid = gtid(), lane = tid & 31, warp = tid >> 5;
  PMOM_PHASE_START(tso);
#ifdef PMOM_PHASES
  long long l_perm = 0, l_stage = 0, l_off = 0, l_diag = 0;
#endif
  if (warp == 0 && !permuted) {
    for (int k = 0; k < N; ++k) {
      const int p = piv[k];
      if (p != k && lane < P) {
        const CT t = W[k * ldw + lane];
        W[k * ldw + lane] = W[p * ldw + lane];
        W[p * ldw + lane] = t;
      }
      __syncwarp();
    }
  }
  gsync();
  PMOM_LAP(l_perm, tso);
  // forward: L y = P b, unit diagonal, blocks of 32 rows.  The whole group stages each 32 x 32
  // diagonal block (independent loads, in flight with the off-diagonal products); warp 0 applies
  // the block's inverse, lane r forming row r of L_bb^-1 w_b.
  const int f0 = (max(0, fwd_from) / 32) * 32;
  for (int i0 = f0; i0 < N; i0 += 32) {
    const int bs = min(32, N - i0);
    for (int e = tid; e < 32 * 32; e += kThreads) {
      const int r = e >> 5, c = e & 31;
      D[r * 33 + c] = (r < bs && c < bs) ? A[static_cast<size_t>(i0 + r) * lda + i0 + c] : czero(D[0]);
    }
    PMOM_LAP(l_stage, tso);
    if (i0 == f0) gsync();
    if (i0 > f0) {
      offdiag_update<CT>(A, lda, i0, bs, f0, i0, W, P, ldw);
      gsync();
    }
    PMOM_LAP(l_off, tso);
    if (warp == 0) {
      const int i = i0 + lane;
      CT w[kMaxPorts];
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p) w[p] = (lane < bs && p < P) ? W[i * ldw + p] : czero(w[0]);
      for (int t = 0; t < bs - 1; ++t) {
        const CT l = (lane < bs && lane > t) ? D[lane * 33 + t] : czero(w[0]);
#pragma unroll
        for (int p = 0; p < kMaxPorts; ++p)
          if (p < P) w[p] = cfma(l, W[(i0 + t) * ldw + p], w[p]);
      }
      __syncwarp();
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p)
        if (lane < bs && p < P) W[i * ldw + p] = w[p];
    }
    gsync();
    PMOM_LAP(l_diag, tso);
  }
  // backward: U x = y, the same 32-row blocks (those of the inverted diagonal) from the last up
  for (int i0 = ((N - 1) / 32) * 32; i0 >= 0; i0 -= 32) {
    const int bs = min(32, N - i0), i1 = i0 + bs;
    for (int e = tid; e < 32 * 32; e += kThreads) {
      const int r = e >> 5, c = e & 31;
      D[r * 33 + c] = (r < bs && c < bs) ? A[static_cast<size_t>(i0 + r) * lda + i0 + c] : czero(D[0]);
    }
    PMOM_LAP(l_stage, tso);
    if (i1 == N) gsync();
    if (i1 < N) {
      offdiag_update<CT>(A, lda, i0, bs, i1, N, W, P, ldw);
      gsync();
    }
    PMOM_LAP(l_off, tso);
    if (warp == 0) {   // lane r forms row r of U_bb^-1 w_b
      const int i = i0 + lane;
      CT w[kMaxPorts];
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p) w[p] = czero(w[0]);
      for (int t = 0; t < bs; ++t) {
        const CT u = (lane <= t) ? D[lane * 33 + t] : czero(w[0]);
#pragma unroll
        for (int p = 0; p < kMaxPorts; ++p)
          if (p < P) w[p] = cfma(u, W[(i0 + t) * ldw + p], w[p]);
      }
      __syncwarp();
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p)
        if (lane < bs && p < P) W[i * ldw + p] = w[p];
    }
    gsync();
    PMOM_LAP(l_diag, tso);
  }
#ifdef PMOM_PHASES
  PMOM_LAP_FLUSH(kPhSolvePerm, l_perm);
  PMOM_LAP_FLUSH(kPhSolveStage, l_stage);
  PMOM_LAP_FLUSH(kPhSolveOff, l_off);
  PMOM_LAP_FLUSH(kPhSolveDiag, l_diag);
#endif
}


// ------------------------------------------------------------------ refinement residual
// Error-free transformations on the FP32 pipe (Knuth's TwoSum, FMA-based TwoProduct); the
// explicit _rn intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += z * (xh + xl): z is an exact float, xh + xl the two-float split of a double
__device__ __forceinline__ void df_mac(float z, float xh, float xl, float& hi, float& lo) {
  const float p = __fmul_rn(z, xh);
  const float e = __fmaf_rn(z, xh, -p);
  float sum, err;
  two_sum(hi, p, sum, err);
  hi = sum;
  lo = __fadd_rn(lo, __fadd_rn(err, __fmaf_rn(z, xl, e)));
}

// float-float addition (a_hi, a_lo) += (b_hi, b_lo): TwoSum of the high parts, the low parts and
// the rounding error folded in, then renormalised (Fast2Sum)
__device__ __forceinline__ void dd_add(float& ah, float& al, float bh, float bl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  ah = __fadd_rn(s, e);
  al = __fsub_rn(e, __fsub_rn(ah, s));
}

// r = V - Z_sub x for complex64 storage in float-float arithmetic (about 2^-44 relative of the
// partial sums), lane partials combined across the warp in float-float too, so the FP64 pipe
// (1/64 of the FP32 rate) only sees one conversion per output.  xs: x split as
// (re_hi, re_lo, im_hi, im_lo).  NP: compile-time bound on the port count P.
// V: the port excitation V[k][p] = l_p on port p's gap BFs k = p * gap_stride + gap_off + j,
// j < gap_n (one BF, 3p+1, with two-triangle pixels) when e0 < 0, else the identity columns
// V[e0+p][p] = 1.
// F32OUT (identity columns only): the residual is formed in float-float and written rounded to
// float into rw (the precision of the correction solve that consumes it), with no FP64 work.
// cols (optional): Z_sub is read in place from the parent Z(f) (row-major, leading dimension lda =
// M) through the support set, Z_sub[i][t] = Zs[cols[i] * lda + cols[t]] -- the frequency-major
// task order keeps Z(f) resident in L2 while its candidates are processed -- instead of from a
// gathered copy.
template <int NP, bool F32OUT = false>
__device__ void residual_df(const float2* __restrict__ Zs, int lda, int N, const float4* xs, int P,
                            const double* lport, double2* __restrict__ r, double* s_red, double* s_out,
                            int e0 = -1, float2* __restrict__ rw = nullptr, int gap_stride = 3, int gap_off = 1,
                            int gap_n = 1, const int* __restrict__ cols = nullptr, int ldx = 0) {
  if (ldx < P) ldx = P;   // row stride of xs (and of rw)
  // two rows per warp at a time: independent float-float chains interleave and each x load
  // serves two rows (measured on the 16x16x2 batch: 1, 2, 3, 4 and 6 rows 706, 699, 716, 715 and 762 ms
  // per launch, bit-identical results; more rows cost registers the kernel does not have)
  constexpr int R = 2;
  const int tid = gtid(), lane = tid & 31, warp = tid >> 5;
  double rmax = 0.0, zmax = 0.0;
  float rmaxf = 0.f, zmaxf = 0.f;
  for (int i0 = warp; i0 < N; i0 += kWarps * R) {
    float rh[R][NP], rl[R][NP], ih[R][NP], il[R][NP], ra[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      ra[q] = 0.f;
#pragma unroll
      for (int p = 0; p < NP; ++p) rh[q][p] = rl[q][p] = ih[q][p] = il[q][p] = 0.f;
    }
    const float2* zrow[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = i0 + q * kWarps, ic = i < N ? i : 0;
      zrow[q] = Zs + static_cast<size_t>(cols ? cols[ic] : ic) * lda;
    }
    // the next column step's entries are loaded while this one's are used (one step of prefetch)
    float2 zn[R];
    int cn = lane < N ? (cols ? cols[lane] : lane) : 0;
#pragma unroll
    for (int q = 0; q < R; ++q) zn[q] = (i0 + q * kWarps < N && lane < N) ? zrow[q][cn] : make_float2(0.f, 0.f);
    for (int t = lane; t < N; t += 32) {
      float2 z[R];
      cn = t + 32 < N ? (cols ? cols[t + 32] : t + 32) : 0;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        z[q] = zn[q];
        zn[q] = (i0 + q * kWarps < N && t + 32 < N) ? zrow[q][cn] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (p < P) {
          const float4 x = xs[t * ldx + p];
#pragma unroll
          for (int q = 0; q < R; ++q) {
            df_mac(z[q].x, x.x, x.y, rh[q][p], rl[q][p]);
            df_mac(-z[q].y, x.z, x.w, rh[q][p], rl[q][p]);
            df_mac(z[q].x, x.z, x.w, ih[q][p], il[q][p]);
            df_mac(z[q].y, x.x, x.y, ih[q][p], il[q][p]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < R; ++q) ra[q] += fabsf(z[q].x) + fabsf(z[q].y);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int i = i0 + q * kWarps;
      float rs = ra[q];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) rs += __shfl_down_sync(0xffffffffu, rs, d);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (p >= P) break;
        float xh = rh[q][p], xl = rl[q][p], yh = ih[q][p], yl = il[q][p];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          const float oxh = __shfl_down_sync(0xffffffffu, xh, d), oxl = __shfl_down_sync(0xffffffffu, xl, d);
          const float oyh = __shfl_down_sync(0xffffffffu, yh, d), oyl = __shfl_down_sync(0xffffffffu, yl, d);
          dd_add(xh, xl, oxh, oxl);
          dd_add(yh, yl, oyh, oyl);
        }
        if (lane == 0 && i < N) {
          if constexpr (F32OUT) {
            float a = -xh, b = -xl;
            dd_add(a, b, i == e0 + p ? 1.f : 0.f, 0.f);
            const float rx = a + b, ry = -(yh + yl);
            rw[i * ldx + p] = make_float2(rx, ry);
            rmaxf = fmaxf(rmaxf, fabsf(rx) + fabsf(ry));
          } else {
            const double vx = static_cast<double>(xh) + static_cast<double>(xl);
            const double vy = static_cast<double>(yh) + static_cast<double>(yl);
            const double vv = e0 < 0 ? (static_cast<unsigned>(i - (p * gap_stride + gap_off)) < static_cast<unsigned>(gap_n)
                                             ? lport[p] : 0.0)
                                      : ((i == e0 + p) ? 1.0 : 0.0);
            const double2 ri = make_double2(vv - vx, -vy);
            r[i * P + p] = ri;
            rmax = fmax(rmax, fabs(ri.x) + fabs(ri.y));
          }
        }
      }
      if (lane == 0 && i < N) {
        if constexpr (F32OUT) zmaxf = fmaxf(zmaxf, rs);
        else zmax = fmax(zmax, static_cast<double>(rs));
      }
    }
  }
  if constexpr (F32OUT) {
    rmax = static_cast<double>(rmaxf);
    zmax = static_cast<double>(zmaxf);
  }
  if (lane == 0) {
    s_red[warp] = rmax;
    s_red[kWarps + warp] = zmax;
  }
  gsync();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      a = fmax(a, s_red[w]);
      b = fmax(b, s_red[kWarps + w]);
    }
    s_out[0] = a;
    s_out[1] = b;
  }
  gsync();
}

// double-storage residual (complex128 database): plain FP64
// r = V - Z_sub x in double from the stored entries; returns ||r||_inf (|re|+|im| norm) and
// ||Z_sub||_inf in s_out[0..1].  x_s: shared copy of x (N x P double2).
template <typename ZT>
__device__ void residual(const ZT* __restrict__ Zf, int M, const int* __restrict__ s_idx, int N, const double2* x_s,
                         int P, const double* lport, double2* __restrict__ r, double* s_red, double* s_out,
                         int gap_stride, int gap_off, int gap_n) {
  const int tid = gtid(), lane = tid & 31, warp = tid >> 5;
  double rmax = 0.0, zmax = 0.0;
  for (int i = warp; i < N; i += kWarps) {
    const ZT* zrow = Zf + static_cast<size_t>(s_idx[i]) * M;
    double2 acc[kMaxPorts];
#pragma unroll
    for (int p = 0; p < kMaxPorts; ++p) acc[p] = make_double2(0.0, 0.0);
    double rowabs = 0.0;
    for (int t = lane; t < N; t += 32) {
      const double2 z = zload<ZT, double2>(zrow + s_idx[t]);
      rowabs += fabs(z.x) + fabs(z.y);
#pragma unroll
      for (int p = 0; p < kMaxPorts; ++p)
        if (p < P) acc[p] = cfma(z, x_s[t * P + p], acc[p]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) rowabs += __shfl_down_sync(0xffffffffu, rowabs, d);
#pragma unroll
    for (int p = 0; p < kMaxPorts; ++p) {
      if (p >= P) break;
      double2 v = acc[p];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, d);
        v.y += __shfl_down_sync(0xffffffffu, v.y, d);
      }
      if (lane == 0) {
        const double vv =
            static_cast<unsigned>(i - (p * gap_stride + gap_off)) < static_cast<unsigned>(gap_n) ? lport[p] : 0.0;
        const double2 ri = make_double2(vv - v.x, -v.y);
        r[i * P + p] = ri;
        rmax = fmax(rmax, fabs(ri.x) + fabs(ri.y));
      }
    }
    if (lane == 0) zmax = fmax(zmax, rowabs);
  }
  if (lane == 0) {
    s_red[warp] = rmax;
    s_red[kWarps + warp] = zmax;
  }
  gsync();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      a = fmax(a, s_red[w]);
      b = fmax(b, s_red[kWarps + w]);
    }
    s_out[0] = a;
    s_out[1] = b;
  }
  gsync();
}

// ------------------------------------------------------------------ Y -> S (Eq. 6-7)
// One thread per task converts the port admittance matrix Y (written by the evaluation kernel
// into the S slot) to S = (1 + Z0 Y)^-1 (1 - Z0 Y) in place.
__global__ void ys_kernel(double2* __restrict__ S, int ntask, int F, int P, double Z0, uint32_t* __restrict__ flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntask) return;
  double2* s = S + static_cast<size_t>(t) * P * P;
  double2 Am[kMaxPorts][kMaxPorts], Bm[kMaxPorts][kMaxPorts];
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      const double2 y = s[i * P + j];
      const double d = (i == j) ? 1.0 : 0.0;
      Am[i][j] = make_double2(d + Z0 * y.x, Z0 * y.y);
      Bm[i][j] = make_double2(d - Z0 * y.x, -Z0 * y.y);
    }
  // Gauss-Jordan with partial pivoting on (1 + Z0 Y) S = (1 - Z0 Y)
  for (int k = 0; k < P; ++k) {
    int p = k;
    double best = cabs2(Am[k][k]);
    for (int i = k + 1; i < P; ++i)
      if (cabs2(Am[i][k]) > best) { best = cabs2(Am[i][k]); p = i; }
    if (p != k)
      for (int j = 0; j < P; ++j) {
        double2 tt = Am[k][j]; Am[k][j] = Am[p][j]; Am[p][j] = tt;
        tt = Bm[k][j]; Bm[k][j] = Bm[p][j]; Bm[p][j] = tt;
      }
    const double2 inv = cinv(Am[k][k]);
    for (int j = 0; j < P; ++j) {
      Am[k][j] = cmul(Am[k][j], inv);
      Bm[k][j] = cmul(Bm[k][j], inv);
    }
    for (int i = 0; i < P; ++i) {
      if (i == k) continue;
      const double2 f = Am[i][k];
      for (int j = 0; j < P; ++j) {
        Am[i][j] = cfms(f, Am[k][j], Am[i][j]);
        Bm[i][j] = cfms(f, Bm[k][j], Bm[i][j]);
      }
    }
  }
  bool bad = false;
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      s[i * P + j] = Bm[i][j];
      if (!isfinite(Bm[i][j].x) || !isfinite(Bm[i][j].y)) bad = true;
    }
  if (bad) atomicOr(&flags[t / F], kFlagNonfinite);
}

// ------------------------------------------------------------------ the evaluation kernel
// Per-slot workspace: [LU matrix | exact complex64 copy of Z_sub (factor-only launches of the
// mixed path: the bordered update's refined inverse reads it row by row) | pivots | row
// permutation | x | residual].
struct Slot {
  size_t a_off, zs_off, piv_off, perm_off, x_off, r_off, wx_off, end;
};
__host__ __device__ inline Slot slot_layout(int M, int lda, int P, size_t ct_bytes) {
  Slot s;
  s.a_off = 0;
  s.zs_off = s.a_off + static_cast<size_t>(M) * lda * ct_bytes;
  s.zs_off = (s.zs_off + 255) & ~size_t(255);
  s.piv_off = s.zs_off + static_cast<size_t>(M) * lda * sizeof(float2);
  s.piv_off = (s.piv_off + 255) & ~size_t(255);
  s.perm_off = s.piv_off + static_cast<size_t>(M) * sizeof(int);
  s.perm_off = (s.perm_off + 255) & ~size_t(255);
  s.x_off = s.perm_off + static_cast<size_t>(M) * sizeof(int);
  s.x_off = (s.x_off + 255) & ~size_t(255);
  s.r_off = s.x_off + static_cast<size_t>(M) * P * sizeof(double2);
  s.r_off = (s.r_off + 255) & ~size_t(255);
  // right-hand sides / solution split of the large-support-set variant (in shared memory otherwise)
  s.wx_off = s.r_off + static_cast<size_t>(M) * P * sizeof(double2);
  s.wx_off = (s.wx_off + 255) & ~size_t(255);
  s.end = s.wx_off + static_cast<size_t>(M) * P * sizeof(float4);
  return s;
}

// Dynamic shared memory: [union of the panel (M x (NB+1)), the x cache and, for the tensor-core
// path, the operand staging (96 KB + 2 KB alignment slack) | U tile / diagonal block | idx (M ints)].
// The staging is only live during the outer-panel steps, when the panel has been written back, so
// the two share memory and the tensor-core variant still fits two task groups per SM.
// Large-support-set variant (`large`): panel of NBL columns; the right-hand sides and the x cache
// live in the slot's global workspace and the solve's diagonal block in the (then idle) panel.
constexpr size_t kTcStageBytes = 98304 + 2048;   // 96 KB operands (or the 128 x 65 result tile) + alignment

template <typename CT>
__host__ __device__ inline size_t smem_layout(int M, int use_tc, bool large, size_t* u_off, size_t* idx_off,
                                              size_t* tc_off) {
  const int NB = large ? Cfg<CT>::NBL : Cfg<CT>::NB;
  size_t panel = static_cast<size_t>(M) * (NB + 1) * sizeof(CT);
  const size_t xcache = large ? 32 * 33 * sizeof(CT) : static_cast<size_t>(M) * kMaxPorts * sizeof(double2);
  if (xcache > panel) panel = xcache;
  if (use_tc && panel < kTcStageBytes) panel = kTcStageBytes;
  panel = (panel + 15) & ~size_t(15);
  *tc_off = 0;
  *u_off = panel;
  size_t u = static_cast<size_t>(NB) * (kTile + 1) * sizeof(CT);
  if (!large && u < 32 * 33 * sizeof(CT)) u = 32 * 33 * sizeof(CT);
  *idx_off = panel + ((u + 15) & ~size_t(15));
  return *idx_off + static_cast<size_t>(M) * sizeof(int);
}

// One group's share of the dynamic shared memory (1024-byte multiple so every group's region
// starts aligned like the first).
template <typename CT>
__host__ __device__ inline size_t group_smem_bytes(int M, int use_tc, bool large) {
  size_t u_off, idx_off, tc_off;
  const size_t b = smem_layout<CT>(M, use_tc, large, &u_off, &idx_off, &tc_off);
  return (b + 1023) & ~size_t(1023);
}

template <typename ZT> struct XCache;
template <> struct XCache<float2> { using type = float4; };
template <> struct XCache<double2> { using type = double2; };

// TC: the single-precision LU runs its outer-panel updates on the tensor cores.  LARGE: narrow
// panels and the solve vectors in global memory, for support sets beyond the shared-memory
// capacity of the default layout (one task group per CTA).
template <typename CT, typename ZT, bool MIXED, bool TC, bool LARGE>
__global__ void __launch_bounds__(kThreads * kMaxGroups, 1) eval_kernel(EvalArgs a, const __grid_constant__ TmaMaps tmaps) {
  using R = typename Real<CT>::type;
  extern __shared__ __align__(16) unsigned char smem_all[];
  __shared__ R s_val_g[kMaxGroups][kWarps + 1];
  __shared__ int s_row_g[kMaxGroups][kWarps + 1];
  __shared__ double s_red_g[kMaxGroups][2 * kWarps];
  __shared__ double s_norm_g[kMaxGroups][2];
  __shared__ int s_task_g[kMaxGroups];
  __shared__ int s_flag_g[kMaxGroups];
  __shared__ double s_dx_g[kMaxGroups][2];   // refinement: last correction norm, ||x||_inf
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar_g[kMaxGroups][kStages];
  __shared__ __align__(8) uint64_t s_rbar_g[kMaxGroups][kRaw];
  __shared__ __align__(8) uint64_t s_gbar_g[kMaxGroups][kGatherBufs];
  __shared__ int s_gfail_g[kMaxGroups];   // a bulk gather wait gave up: later tasks are flagged
  constexpr bool use_tc = TC && std::is_same<CT, float2>::value;
  const int g = group_id();
  const int ngroups = blockDim.x / kThreads;
  R* s_val = s_val_g[g];
  int* s_row = s_row_g[g];
  double* s_red = s_red_g[g];
  double* s_norm = s_norm_g[g];
  int& s_task = s_task_g[g];
  int& s_flag = s_flag_g[g];
  double* s_dx = s_dx_g[g];
  size_t u_off, idx_off, tc_off;
  constexpr int NB = LARGE ? Cfg<CT>::NBL : Cfg<CT>::NB;
  const size_t group_bytes = group_smem_bytes<CT>(a.ncap, use_tc, LARGE);
  smem_layout<CT>(a.ncap, use_tc, LARGE, &u_off, &idx_off, &tc_off);
  unsigned char* smem = smem_all + g * group_bytes;
  CT* Pn = reinterpret_cast<CT*>(smem);
  CT* Ut = reinterpret_cast<CT*>(smem + u_off);
  int* s_idx = reinterpret_cast<int*>(smem + idx_off);
  const int tid = gtid();
  TcState tcs;
  tcs.stage = nullptr;
  tcs.tmem = 0;
  tcs.seg_chunks = LARGE ? kSegChunksLarge : kSegChunks;
  tcs.mbar = s_mbar_g[g];
  tcs.sph = 0;
  tcs.failed = false;
  tcs.maps = &tmaps;
  tcs.tz = 0;
  tcs.rbar = s_rbar_g[g];
  tcs.rph = 0;
  uint64_t* gbar = s_gbar_g[g];
  volatile int& s_gfail = s_gfail_g[g];
  uint32_t gph = 0;   // bit b: parity of the next completion awaited on gather buffer b
  if (threadIdx.x == 0) {
    for (int i = 0; i < ngroups; ++i) {
      s_gfail_g[i] = 0;
      for (int j = 0; j < kGatherBufs; ++j) tc::mbar_init(&s_gbar_g[i][j], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (use_tc) {
    // 1024-byte aligned operand staging inside this group's tensor-core region
    const uint32_t base = tc::smem_u32(smem + tc_off);
    tcs.stage = smem + tc_off + ((1024u - (base & 1023u)) & 1023u);
    if (threadIdx.x < 32) {   // one warp allocates 256 TMEM columns per group for the whole CTA
      tc::tmem_alloc(&s_tmem, kTmemCols * ngroups);
      tc::tmem_relinquish();
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i < ngroups; ++i) {
        for (int j = 0; j < kStages; ++j) tc::mbar_init(&s_mbar_g[i][j], 1);
        for (int j = 0; j < kRaw; ++j) tc::mbar_init(&s_rbar_g[i][j], 1);
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tcs.tmem = s_tmem + kTmemCols * g;
  }
  const int P = a.P, M = a.M, lda = a.lda;
  const Slot sl = slot_layout(a.ncap, lda, P, sizeof(CT));
  const int slot = blockIdx.x * ngroups + g;
  CT* Dg = LARGE ? Pn : Ut;
  const ZT* Zall = static_cast<const ZT*>(a.Z);
  const int ntasks = a.ntasks_list ? *a.repair_count : a.B * a.F;
  double lport[kMaxPorts];
#pragma unroll
  for (int p = 0; p < kMaxPorts; ++p) lport[p] = a.port_len[p];

  for (;;) {
    if (slot >= a.nslots) break;   // a spare group (odd slot count): no workspace
    if (tid == 0) s_task = atomicAdd(a.task_counter, 1);
    gsync();
    const int tq = s_task;
    gsync();
    if (tq >= ntasks) break;
    PMOM_PHASE_START(tev);
    const int t = a.ntasks_list ? a.repair_list[tq] : tq;
    const int f = t / a.B, b = a.order ? a.order[t % a.B] : t % a.B;
    const int N = a.n_act[b];
    // the task's workspace: the group's slot, or (factor-only launches) slot t, which keeps the
    // factors for a later kernel
    unsigned char* ws = static_cast<unsigned char*>(a.work) + a.slot_bytes * (a.factor_only ? t : slot);
    tcs.tz = a.factor_only ? t : slot;
    CT* A = reinterpret_cast<CT*>(ws + sl.a_off);
    float2* Zs = reinterpret_cast<float2*>(ws + sl.zs_off);
    int* piv = reinterpret_cast<int*>(ws + sl.piv_off);
    int* perm = reinterpret_cast<int*>(ws + sl.perm_off);
    double2* X = reinterpret_cast<double2*>(ws + sl.x_off);
    double2* Rv = reinterpret_cast<double2*>(ws + sl.r_off);
    // right-hand sides / corrections (W), the x cache of the residual
    unsigned char* vec = LARGE ? ws + sl.wx_off : smem;
    CT* W = reinterpret_cast<CT*>(vec);
    // the right-hand sides are written already permuted (row k of W = row perm[k])
    auto solve = [&](int fwd_from) { lu_solve<CT>(A, lda, N, piv, W, P, Dg, 0, true, fwd_from); };
    uint32_t* flag_of = &a.flags[a.factor_only ? t : b];
    if (N <= 0 || N > a.ncap) {
      // bad pixel states, or a support set larger than the shared memory this launch was sized
      // for (a graph captured with a smaller capacity): no solve, NaN S, flagged candidate
      if (!a.factor_only && tid < P * P)
        a.S[(static_cast<size_t>(b) * a.F + f) * P * P + tid] = make_double2(__longlong_as_double(0x7ff8000000000000ll), 0.0);
      if (tid == 0 && N > a.ncap) atomicOr(flag_of, kFlagCapacity);
      continue;
    }
    double2* Sout = a.S + (static_cast<size_t>(b) * a.F + f) * P * P;
    const ZT* Zf = Zall + static_cast<size_t>(f) * M * M;
    const int32_t* gidx = a.idx + static_cast<size_t>(b) * M;
    for (int i = tid; i < N; i += kThreads) s_idx[i] = gidx[i];
    gsync();
    // gather Z_sub (Eq. 5): row i of Z_sub = row I_i of Z(f) at the columns I.  Whole parent rows
    // stream into shared memory by bulk asynchronous copies (up to kGatherBufs rows in flight from
    // the L2-resident Z(f)); the group picks the support set's columns out of each staged row and
    // writes row i of the workspace with coalesced stores.  Parents whose rows do not fit two
    // buffers, or are not a multiple of 16 bytes, take the element-wise gather.
    // The exact complex64 copy is kept only for factor-only launches (the bordered update's refined
    // inverse reads it); the evaluation's own residual reads Z(f) in place through the support set.
    constexpr bool kZsMixed = MIXED && std::is_same<ZT, float2>::value;
    const bool zs_copy = kZsMixed && a.factor_only;
    const uint32_t row_bytes = static_cast<uint32_t>(M) * sizeof(ZT);
    const int nbuf = min(kGatherBufs, static_cast<int>(u_off / row_bytes));
    if (nbuf >= 2 && (row_bytes & 15u) == 0 && !s_gfail) {
      ZT* gbuf = reinterpret_cast<ZT*>(smem);
      if (tid == 0) {
        for (int b = 0; b < nbuf && b < N; ++b) {
          tc::mbar_arrive_expect_tx(&gbar[b], row_bytes);
          tc::bulk_g2s(gbuf + static_cast<size_t>(b) * M, Zf + static_cast<size_t>(s_idx[b]) * M, row_bytes, &gbar[b]);
        }
      }
      for (int i = 0; i < N; ++i) {
        const int b = i % nbuf;
        if (!tc::mbar_wait(&gbar[b], (gph >> b) & 1u, kTcWaitPolls)) s_gfail = 1;
        gph ^= 1u << b;
        const ZT* row = gbuf + static_cast<size_t>(b) * M;
        for (int j = tid; j < N; j += kThreads) {
          const CT v = zconv<ZT, CT>(row[s_idx[j]]);
          A[static_cast<size_t>(i) * lda + j] = v;
          if constexpr (kZsMixed) {
            if (zs_copy) Zs[static_cast<size_t>(i) * lda + j] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
          }
        }
        tc::fence_async_smem();   // these reads come before the next bulk write into the buffer
        gsync();
        if (tid == 0 && i + nbuf < N) {
          tc::mbar_arrive_expect_tx(&gbar[b], row_bytes);
          tc::bulk_g2s(gbuf + static_cast<size_t>(b) * M, Zf + static_cast<size_t>(s_idx[i + nbuf]) * M, row_bytes,
                       &gbar[b]);
        }
      }
    } else {
      // element-wise: eight independent loads in flight per thread, then the stores
      const int NN = N * N;
      for (int e0 = tid; e0 < NN; e0 += 8 * kThreads) {
        CT v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kThreads, i = e / N, j = e - i * N;
          v[u] = e < NN ? zload<ZT, CT>(Zf + static_cast<size_t>(s_idx[i]) * M + s_idx[j]) : czero(v[0]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int e = e0 + u * kThreads, i = e / N, j = e - i * N;
          if (e < NN) {
            A[static_cast<size_t>(i) * lda + j] = v[u];
            if constexpr (kZsMixed) {
              if (zs_copy) Zs[static_cast<size_t>(i) * lda + j] = make_float2(static_cast<float>(v[u].x), static_cast<float>(v[u].y));
            }
          }
        }
      }
    }
    gsync();
    PMOM_PHASE(kPhGather, tev);
    // the autotuner's choice for this support-set size (the large layout always takes the tensor cores)
    const bool task_tc = use_tc && (LARGE || a.tc_bucket[n_bucket(N)] != 0);
    const bool singular = lu_factor<CT, NB>(A, lda, N, piv, Pn, Ut, s_val, s_row, task_tc ? &tcs : nullptr);
    gsync();
    lu_invert_diag<CT>(A, lda, N, Dg);
    PMOM_PHASE(kPhLu, tev);
    if (a.factor_only) {   // factors stay in slot t; a zero pivot or a failed tensor-core wait is flagged
      if (tid == 0 && (singular || tcs.failed || s_gfail)) atomicOr(flag_of, kFlagSingular);
      tcs.failed = false;
      gsync();
      continue;
    }
    if (tid == 0) s_flag = N;   // the first nonzero row of P V (pivot order), found below
    pivots_to_perm(piv, N, reinterpret_cast<int*>(Pn), perm);
    // right-hand sides: V[k][p] = l_p on port p's gap BFs (a delta gap of 1 V; one BF, 3p+1,
    // with two-triangle pixels), rows in pivot order
    for (int e = tid; e < N * P; e += kThreads) {
      const int i = perm[e / P], p = e % P;
      const bool gap = static_cast<unsigned>(i - (p * a.gap_stride + a.gap_off)) < static_cast<unsigned>(a.gap_n);
      W[e] = from_d2<CT>(make_double2(gap ? lport[p] : 0.0, 0.0));
      if (gap) atomicMin(&s_flag, e / P);
    }
    gsync();
    solve(s_flag);
    for (int e = tid; e < N * P; e += kThreads) X[e] = to_d2(W[e]);
    gsync();
    PMOM_PHASE(kPhSolve0, tev);
    int iters = 0;
    bool repaired = false;
    if (MIXED) {
      double rprev = 0.0;
      double2* xs = reinterpret_cast<double2*>(vec);
      const double vnorm = fmax(fmax(lport[0], P > 1 ? lport[1] : 0.0), fmax(P > 2 ? lport[2] : 0.0, P > 3 ? lport[3] : 0.0));
      bool converged = false;
      for (int it = 0; it <= kMaxRefine; ++it) {
        double xmax = 0.0;   // ||x||_inf (|re|+|im|), reduced over the block
        if constexpr (std::is_same<ZT, float2>::value) {
          float4* xf = reinterpret_cast<float4*>(vec);
          for (int e = tid; e < N * P; e += kThreads) {
            const double2 v = X[e];
            const float hx = static_cast<float>(v.x), hy = static_cast<float>(v.y);
            xf[e] = make_float4(hx, static_cast<float>(v.x - hx), hy, static_cast<float>(v.y - hy));
            xmax = fmax(xmax, fabs(v.x) + fabs(v.y));
          }
          gsync();
          const float2* Zf32 = reinterpret_cast<const float2*>(Zf);
          if (P <= 3)
            residual_df<3>(Zf32, M, N, xf, P, lport, Rv, s_red, s_norm, -1, nullptr, a.gap_stride, a.gap_off, a.gap_n,
                           s_idx);
          else
            residual_df<kMaxPorts>(Zf32, M, N, xf, P, lport, Rv, s_red, s_norm, -1, nullptr, a.gap_stride, a.gap_off,
                                   a.gap_n, s_idx);
        } else {
          for (int e = tid; e < N * P; e += kThreads) {
            xs[e] = X[e];
            xmax = fmax(xmax, fabs(X[e].x) + fabs(X[e].y));
          }
          gsync();
          residual<ZT>(Zf, M, s_idx, N, xs, P, lport, Rv, s_red, s_norm, a.gap_stride, a.gap_off, a.gap_n);
        }
        PMOM_PHASE(kPhResid, tev);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) xmax = fmax(xmax, __shfl_down_sync(0xffffffffu, xmax, d));
        if ((tid & 31) == 0) s_red[tid >> 5] = xmax;
        gsync();
        if (tid == 0) {
          double m = 0.0;
          for (int w = 0; w < kWarps; ++w) m = fmax(m, s_red[w]);
          s_dx[1] = m;
          const double rn = s_norm[0], zn = s_norm[1];
          const double eta = rn / (zn * m + vnorm);
          int flag = 0;   // 0 continue, 1 converged, 2 stop (stagnated or out of iterations)
          if (eta <= kEtaTarget) flag = 1;
          else if (it > 0 && rn > 0.5 * rprev) flag = 2;      // stagnated above the target
          else if (it == kMaxRefine) flag = 2;
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
        for (int e = tid; e < N * P; e += kThreads) W[e] = from_d2<CT>(Rv[perm[e / P] * P + e % P]);
        gsync();
        PMOM_PHASE(kPhOther, tev);
        solve(0);
        PMOM_PHASE(kPhSolveCorr, tev);
        double dmax = 0.0;   // ||correction||_inf
        for (int e = tid; e < N * P; e += kThreads) {
          const double2 d = to_d2(W[e]);
          X[e] = make_double2(X[e].x + d.x, X[e].y + d.y);
          dmax = fmax(dmax, fabs(d.x) + fabs(d.y));
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, d));
        if ((tid & 31) == 0) s_red[tid >> 5] = dmax;
        gsync();
        ++iters;
        if (tid == 0) {
          double dn = 0.0;
          for (int w = 0; w < kWarps; ++w) dn = fmax(dn, s_red[w]);
          const double dprev = s_dx[0];
          s_flag = (it > 0 && dn < 0.5 * dprev && (dn / dprev) * dn <= kDxTarget * s_dx[1]) ? 1 : 0;
          s_dx[0] = dn;
        }
        gsync();
        if (s_flag) {
          converged = true;
          break;
        }
      }
      if (!converged) repaired = true;
    }
    if (tid == 0) {
      if (MIXED) {
        atomicAdd(&a.counters[0], static_cast<unsigned long long>(iters));
        atomicMax(&a.counters[1], static_cast<unsigned long long>(iters));
      }
      atomicAdd(&a.counters[3], 1ull);
      if (repaired) {
        const int slot = atomicAdd(a.repair_count, 1);
        a.repair_list[slot] = t;
        atomicAdd(&a.counters[2], 1ull);
        atomicOr(&a.flags[b], kFlagRepaired);
      } else if (singular) {
        atomicOr(&a.flags[b], kFlagSingular);
      }
      if (tcs.failed || s_gfail) {   // a completion wait ran out: the task's numbers are not trusted
        atomicOr(&a.flags[b], kFlagNonfinite);
        atomicAdd(&a.counters[4], 1ull);
      }
    }
    tcs.failed = false;
    // port admittances Y_ij = sum over port i's gap BFs k of l_i x_k^(j) (Eq. 7; one BF, 3i+1, with
    // two-triangle pixels) into the S slot; ys_kernel converts them
    if (!repaired && tid < P * P) {
      const int i = tid / P, j = tid % P;
      double2 y = make_double2(0.0, 0.0);
      for (int k = 0; k < a.gap_n; ++k) {
        const double2 xv = X[(i * a.gap_stride + a.gap_off + k) * P + j];
        y.x += lport[i] * xv.x;
        y.y += lport[i] * xv.y;
      }
      Sout[tid] = y;
    }
    gsync();
    PMOM_PHASE(kPhOther, tev);
#ifdef PMOM_PHASES
    if (tid == 0) atomicAdd(&g_phase_cycles[kPhTasks], 1ull);
#endif
  }
  if (use_tc) {   // both groups are done with the tensor memory
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(s_tmem, kTmemCols * ngroups);
  }
}

// ------------------------------------------------------------------ FoM (Eq. 8-9)
__device__ __forceinline__ double sdb(double2 s) {
  double m = sqrt(s.x * s.x + s.y * s.y);
  if (m < 1e-15) m = 1e-15;
  return 20.0 * log10(m);
}

__global__ void fom_kernel(const double2* __restrict__ S, const uint8_t* __restrict__ bands, int F, int P, int B,
                           const uint32_t* __restrict__ flags, const int32_t* __restrict__ n_act, double* __restrict__ fom,
                           int32_t* __restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double sum = 0.0;
  if (P >= 3 && n_act[b] >= 0) {
    for (int f = 0; f < F; ++f) {
      const double2* s = S + (static_cast<size_t>(b) * F + f) * P * P;
      const double s11 = sdb(s[0]), s21 = sdb(s[1 * P + 0]), s31 = sdb(s[2 * P + 0]), s32 = sdb(s[2 * P + 1]);
      switch (bands[f]) {
        case 0:  // 1/rw_p1 + 1/rw_m1 + 1/rw_s2
          sum += pow(10.0, -(s21 + 1.0) / 10.0) + pow(10.0, (15.0 + s11) / 10.0) + pow(10.0, (s31 + 35.0) / 15.0);
          break;
        case 1:  // 1/rw_p2 + 1/rw_m2 + 1/rw_s1
          sum += pow(10.0, -(s31 + 1.0) / 10.0) + pow(10.0, (15.0 + s11) / 10.0) + pow(10.0, (s21 + 35.0) / 15.0);
          break;
        case 2:  // 1/rw_oi
          sum += pow(10.0, (s32 + 20.0) / 15.0);
          break;
        case 3:  // 1/rw_s3 + 1/rw_s4
          sum += pow(10.0, (s21 + 20.0) / 18.0) + pow(10.0, (s31 + 20.0) / 18.0);
          break;
        default: break;
      }
    }
  }
  const uint32_t fl = flags[b];
  int32_t st = PMOM_CAND_OK;
  if (n_act[b] < 0 || (fl & kFlagBadState)) {
    st = PMOM_CAND_BAD_STATE;
    sum = __longlong_as_double(0x7ff8000000000000ll);
  } else if (fl & kFlagCapacity) {
    st = PMOM_CAND_CAPACITY;
    sum = __longlong_as_double(0x7ff8000000000000ll);
  } else if (fl & kFlagFar) {
    st = PMOM_CAND_FAR;
    sum = __longlong_as_double(0x7ff8000000000000ll);
  } else if ((fl & kFlagNonfinite) || !isfinite(sum)) st = PMOM_CAND_NONFINITE;
  else if (fl & kFlagSingular) st = PMOM_CAND_SINGULAR;
  else if (fl & kFlagRepaired) st = PMOM_CAND_REPAIRED;
  fom[b] = sum;
  status[b] = st;
}

// Counting sort of candidates by support-set size, descending (stable).  One block.
__global__ void order_kernel(const int32_t* __restrict__ n_act, int B, int M, int* __restrict__ order) {
  extern __shared__ int cnt[];   // M + 2 bins: N = -1 (bad) .. M
  const int nb = M + 2;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) atomicAdd(&cnt[M - max(n_act[b], -1)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int i = 0; i < nb; ++i) {
      const int c = cnt[i];
      cnt[i] = run;
      run += c;
    }
    for (int b = 0; b < B; ++b) order[cnt[M - max(n_act[b], -1)]++] = b;
  }
}

template <typename ZT>
__global__ void gather_kernel(const ZT* __restrict__ Z, int M, int f, const int32_t* __restrict__ idx, int N,
                              ZT* __restrict__ out) {
  const ZT* Zf = Z + static_cast<size_t>(f) * M * M;
  for (int i = blockIdx.x; i < N; i += gridDim.x) {
    const ZT* zrow = Zf + static_cast<size_t>(idx[i]) * M;
    for (int j = threadIdx.x; j < N; j += blockDim.x) out[static_cast<size_t>(i) * N + j] = zrow[idx[j]];
  }
}

// Batched gather: CTA (y = candidate b, x = block of R rows) copies its parent rows I_b[i] of
// Z(f) into shared memory by bulk asynchronous copies (all R in flight, one mbarrier each), then
// compacts each to the columns I_b with coalesced stores into out[b][i][0..N_b).  bulk = 0 (rows
// that are not a multiple of 16 bytes): element loads instead.
template <typename ZT>
__global__ void __launch_bounds__(256) gather_batch_kernel(const ZT* __restrict__ Z, int M, int f,
                                                           const int32_t* __restrict__ idx, const int32_t* __restrict__ n,
                                                           int ncap, int R, int bulk, ZT* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char gsm[];
  __shared__ __align__(8) uint64_t bar[8];
  __shared__ int s_fail;
  const int b = blockIdx.y, N = n[b], r0 = blockIdx.x * R;
  if (N <= 0 || N > ncap || r0 >= N) return;
  const int rows = min(R, N - r0);
  const ZT* Zf = Z + static_cast<size_t>(f) * M * M;
  const int32_t* I = idx + static_cast<size_t>(b) * M;
  ZT* buf = reinterpret_cast<ZT*>(gsm);
  int* s_idx = reinterpret_cast<int*>(gsm + static_cast<size_t>(R) * M * sizeof(ZT));
  const uint32_t row_bytes = static_cast<uint32_t>(M) * sizeof(ZT);
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int r = 0; r < rows; ++r) tc::mbar_init(&bar[r], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int j = threadIdx.x; j < N; j += blockDim.x) s_idx[j] = I[j];
  __syncthreads();
  if (bulk && threadIdx.x == 0) {
    for (int r = 0; r < rows; ++r) {
      tc::mbar_arrive_expect_tx(&bar[r], row_bytes);
      tc::bulk_g2s(buf + static_cast<size_t>(r) * M, Zf + static_cast<size_t>(s_idx[r0 + r]) * M, row_bytes, &bar[r]);
    }
  }
  ZT* o = out + static_cast<size_t>(b) * ncap * ncap;
  for (int r = 0; r < rows; ++r) {
    const int i = r0 + r;
    if (bulk) {
      if (!tc::mbar_wait(&bar[r], 0, 1ll << 18)) s_fail = 1;
      const ZT* row = buf + static_cast<size_t>(r) * M;
      for (int j = threadIdx.x; j < N; j += blockDim.x) o[static_cast<size_t>(i) * ncap + j] = row[s_idx[j]];
    } else {
      const ZT* row = Zf + static_cast<size_t>(s_idx[i]) * M;
      for (int j = threadIdx.x; j < N; j += blockDim.x) o[static_cast<size_t>(i) * ncap + j] = row[s_idx[j]];
    }
  }
  __syncthreads();
  // a copy that never completed leaves its row unreliable: poison the block's rows (NaN)
  if (s_fail) {
    ZT nan;
    nan.x = __int_as_float(0x7fc00000);
    nan.y = nan.x;
    for (int e = threadIdx.x; e < rows * N; e += blockDim.x)
      o[static_cast<size_t>(r0 + e / N) * ncap + e % N] = nan;
  }
}

int optin_smem() {
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return optin;
}
constexpr size_t kStaticSmemSlack = 2048;   // static shared memory and the runtime's reservation

// The large-support-set layout is used when the default layout's single task group does not fit
// the opt-in shared memory of one CTA.
template <typename CT>
bool needs_large_layout(int ncap, bool tc) {
  return group_smem_bytes<CT>(ncap, tc, false) + kStaticSmemSlack > static_cast<size_t>(optin_smem());
}

// Task groups per CTA: two when both groups' shared memory fits one CTA, else one.
template <typename CT>
int groups_for(int ncap, bool tc, bool large) {
  const size_t gb = group_smem_bytes<CT>(ncap, tc, large);
  return (2 * gb + kStaticSmemSlack <= static_cast<size_t>(optin_smem())) ? 2 : 1;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (tensor_map_encoder_ptr,
// pmom_eval.cu; the library does not link against the driver library).
inline decltype(&cuTensorMapEncodeTiled) tensor_map_encoder() {
  return reinterpret_cast<decltype(&cuTensorMapEncodeTiled)>(tensor_map_encoder_ptr());
}

// The four operand-tile maps (TmaMaps) over `slots` workspace slots of slot_bytes each, starting
// at base, each holding a rows x lda complex64 matrix.  Returns false if the encoder is missing or
// rejects the layout.
inline bool encode_tile_maps(TmaMaps* t, void* base, int lda, int rows, unsigned long long slots, size_t slot_bytes) {
  const auto fn = tensor_map_encoder();
  if (fn == nullptr || base == nullptr) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(lda), static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(slots)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(lda) * 8u, static_cast<cuuint64_t>(slot_bytes)};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int i = 0; i < 4; ++i) {
    const cuuint32_t box[3] = {kBoxW[i], kBoxH[i], 1};
    if (fn(&t->m[i], CU_TENSOR_MAP_DATA_TYPE_INT64, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

template <typename CT, typename ZT, bool MIXED, bool TC, bool LARGE>
cudaError_t launch_eval_t(const EvalArgs& a, int nslots, cudaStream_t s) {
  if (a.ncap < 1 || a.ncap > a.M || a.lda < a.ncap || nslots < 1) return cudaErrorInvalidValue;
  const int gmax = groups_for<CT>(a.ncap, TC, LARGE);
  const int groups = a.max_groups > 0 && a.max_groups < gmax ? a.max_groups : gmax;
  const size_t smem = groups * group_smem_bytes<CT>(a.ncap, TC, LARGE);
  auto k = eval_kernel<CT, ZT, MIXED, TC, LARGE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  EvalArgs b = a;
  b.nslots = nslots;
  TmaMaps maps{};
  if constexpr (TC && std::is_same<CT, float2>::value) {
    // slot t of task t in factor-only launches, else the group's slot
    const unsigned long long slots = a.factor_only ? static_cast<unsigned long long>(a.B) * a.F : nslots;
    if (!encode_tile_maps(&maps, a.work, a.lda, a.ncap, slots, a.slot_bytes)) return cudaErrorInvalidValue;
  }
  k<<<(nslots + groups - 1) / groups, kThreads * groups, smem, s>>>(b, maps);
  return cudaGetLastError();
}

// Resident task groups per SM (CTAs per SM x groups per CTA).
template <typename CT, typename ZT, bool MIXED, bool TC, bool LARGE>
int blocks_per_sm_t(int M, int max_groups = 0) {
  const int gmax = groups_for<CT>(M, TC, LARGE);
  const int groups = max_groups > 0 && max_groups < gmax ? max_groups : gmax;
  const size_t smem = groups * group_smem_bytes<CT>(M, TC, LARGE);
  auto k = eval_kernel<CT, ZT, MIXED, TC, LARGE>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kThreads * groups, smem) != cudaSuccess) return 0;
  return n * groups;
}

}  // namespace
}  // namespace pmom
