// Learned pre-ranker: a multilayer perceptron trained on (pixel map, S-parameter) pairs that the
// evaluator itself produces, used to rank candidate flips so that only the best-ranked ones get an
// exact solve.  Everything runs in these kernels:
//
//   gemm_bf16_kernel : D = A B^T on the tensor cores (tcgen05.mma kind::f16, BF16 operands staged
//                      in shared memory in the canonical K-major layout, FP32 accumulation in
//                      TMEM), with a fused epilogue (bias, ReLU, ReLU-derivative mask, BF16/FP32
//                      stores); operands are read through strides, so the backward products
//                      (transposed operands) use the same kernel
//   input / loss / bias-gradient / Adam / FoM kernels : elementwise and reductions
//
// Layer l maps h_l (B x d_l, BF16) to z_l = h_l W_l^T + b_l (W_l: d_{l+1} x d_l); hidden layers
// apply ReLU, the last is linear.  Loss: mean squared error over the batch and outputs.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "pmom_internal.h"
#include "pmom_tc.cuh"

struct pmom_mlp {
  int L = 0;                      // layers
  std::vector<int> dims;          // L + 1
  std::vector<size_t> w_off, b_off;   // offsets into the flat parameter vector [W0, b0, W1, b1, ...]
  size_t n_params = 0;
  float* d_p = nullptr;           // FP32 master parameters
  float* d_g = nullptr;           // gradients
  float* d_m = nullptr;           // Adam moments
  float* d_v = nullptr;
  __nv_bfloat16* d_wb = nullptr;  // BF16 copies of the parameters (same offsets as d_p)
  int64_t t = 0;                  // Adam step
  // activations for the batch capacity
  int b_cap = 0;
  std::vector<__nv_bfloat16*> d_h;   // h_0 .. h_{L-1} (B x d_l)
  float* d_out = nullptr;            // B x d_L
  __nv_bfloat16* d_dz = nullptr;     // B x max(d): gradient of the current layer's z
  __nv_bfloat16* d_dz2 = nullptr;
  double* d_loss = nullptr;
  int* d_err = nullptr;              // tensor-core completion waits that ran out
  std::string err;
};

namespace pmom {
namespace {

constexpr int kGT = 256;                          // threads per GEMM CTA
constexpr int kTM = 128, kTN = 128, kTK = 64;     // CTA tile (M x N) and K chunk (BF16 elements)

// byte offset of (row, k) in a 128 x 64 BF16 tile, canonical K-major no-swizzle layout: core
// matrices of 8 rows x 16 bytes, LBO = 128 bytes along K, SBO = 1024 bytes between 8-row groups
__device__ __forceinline__ uint32_t kmaj_bf16(int row, int k) {
  return static_cast<uint32_t>((row >> 3) * tc::kSBO + (k >> 3) * tc::kLBO + (row & 7) * 16 + (k & 7) * 2);
}

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  // D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and 10-12 = 1), both K-major, N >> 3, M >> 4
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

enum Epi : int {
  kEpiStoreF32 = 0,      // D (+ bias) -> out_f32
  kEpiReluBF16 = 1,      // relu(D + bias) -> out_bf16
  kEpiMaskBF16 = 2,      // D * (mask > 0) -> out_bf16   (backward through a ReLU)
};

struct GemmArgs {
  // A(m, k) = A[m * sam + k * sak], B(n, k) = B[n * sbn + k * sbk]; D(m, n) = sum_k A(m, k) B(n, k)
  const __nv_bfloat16* A;
  long long sam, sak;
  const __nv_bfloat16* B;
  long long sbn, sbk;
  int M, N, K;
  int epi;
  const float* bias;                 // [N] or null
  const __nv_bfloat16* mask;         // [M x N] (ld = ldo) for kEpiMaskBF16
  float* out_f32;                    // [M x N] row-major, ld = ldo
  __nv_bfloat16* out_bf16;
  int ldo;
  int* err;
};

__global__ void __launch_bounds__(kGT, 1) gemm_bf16_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 1024-byte aligned operand tiles
  const uint32_t base = tc::smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (base & 1023u)) & 1023u);
  unsigned char* sA = smem;                       // 128 x 64 BF16 = 16 KB
  unsigned char* sB = smem + kTM * kTK * 2;       // 128 x 64 BF16
  float* sT = reinterpret_cast<float*>(smem + 2 * kTM * kTK * 2);   // 32 x 33 epilogue transpose per warp
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 128);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&s_mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  uint32_t phase = 0;
  const uint32_t idesc = idesc_bf16(kTM, kTN);
  for (int k0 = 0; k0 < g.K; k0 += kTK) {
    // stage the A and B chunks (zero outside the matrices)
    for (int e = tid; e < kTM * kTK; e += kGT) {
      const int r = e / kTK, k = e % kTK;
      const int m = m0 + r, n = n0 + r, kk = k0 + k;
      __nv_bfloat16 av = __float2bfloat16(0.f), bv = __float2bfloat16(0.f);
      if (m < g.M && kk < g.K) av = g.A[m * g.sam + kk * g.sak];
      if (n < g.N && kk < g.K) bv = g.B[n * g.sbn + kk * g.sbk];
      *reinterpret_cast<__nv_bfloat16*>(sA + kmaj_bf16(r, k)) = av;
      *reinterpret_cast<__nv_bfloat16*>(sB + kmaj_bf16(r, k)) = bv;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
      for (int kc = 0; kc < kTK / 16; ++kc)   // K = 16 BF16 (32 bytes, two core matrices) per MMA
        mma_bf16(tmem, tc::smem_desc(a0 + kc * 256), tc::smem_desc(b0 + kc * 256), idesc,
                 (k0 > 0 || kc > 0) ? 1u : 0u);
      tc::commit(&s_mbar);
    }
    if (warp == 0) {   // the operands are overwritten by the next chunk: wait for the MMAs
      int ok = 1;
      // at most 2^18 polls (about 1 s at 3.8 us per unanswered try_wait), then the error flag
      if (lane == 0) ok = tc::mbar_wait(&s_mbar, phase, 1ll << 18) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok && lane == 0) s_fail = 1;
    }
    phase ^= 1u;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (s_fail) break;
  }
  if (s_fail) {
    if (tid == 0) atomicAdd(g.err, 1);
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows) and columns 64 (w / 4) .. + 63
    // in two 32-column loads; a per-warp transpose through shared memory makes the stores
    // row-contiguous
    float* T = sT + warp * 32 * 33;
    const int rbase = 32 * (warp & 3);
    for (int half = 0; half < 2; ++half) {
      const int cbase = 64 * (warp >> 2) + 32 * half;
      float v[32];
      tc::tmem_ld32(tmem + (static_cast<uint32_t>(rbase) << 16) + cbase, v);
#pragma unroll
      for (int c = 0; c < 32; ++c) T[lane * 33 + c] = v[c];
      __syncwarp();
      for (int r = 0; r < 32; ++r) {
        const int m = m0 + rbase + r, n = n0 + cbase + lane;
        if (m >= g.M || n >= g.N) continue;
        float d = T[r * 33 + lane];
        if (g.bias) d += g.bias[n];
        const size_t o = static_cast<size_t>(m) * g.ldo + n;
        if (g.epi == kEpiStoreF32) {
          g.out_f32[o] = d;
        } else if (g.epi == kEpiReluBF16) {
          g.out_bf16[o] = __float2bfloat16(d > 0.f ? d : 0.f);
        } else {
          g.out_bf16[o] = __float2bfloat16(__bfloat162float(g.mask[o]) > 0.f ? d : 0.f);
        }
      }
      __syncwarp();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

size_t gemm_smem() { return 2 * kTM * kTK * 2 + 8 * 32 * 33 * sizeof(float) + 1024; }

cudaError_t gemm(const GemmArgs& a, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(gemm_smem()));
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + kTN - 1) / kTN, (a.M + kTM - 1) / kTM);
  gemm_bf16_kernel<<<grid, kGT, gemm_smem(), s>>>(a);
  return cudaGetLastError();
}

__global__ void input_kernel(const uint8_t* __restrict__ x, size_t n, __nv_bfloat16* __restrict__ h) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    h[i] = __float2bfloat16(x[i] ? 1.f : 0.f);
}

// dL/dout = 2 (out - t) / n as BF16 and the loss sum((out - t)^2) / n in FP64
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ t, size_t n, double scale,
                            __nv_bfloat16* __restrict__ dz, double* __restrict__ loss) {
  __shared__ double s_part[256];
  double acc = 0.0;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const double d = static_cast<double>(out[i]) - static_cast<double>(t[i]);
    dz[i] = __float2bfloat16(static_cast<float>(2.0 * d * scale));
    acc += d * d;
  }
  s_part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s_part[threadIdx.x] += s_part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, s_part[0] * scale);
}

// db[n] = sum over the batch of dz[b][n]
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ dz, int B, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int b = 0; b < B; ++b) acc += __bfloat162float(dz[static_cast<size_t>(b) * N + n]);
  db[n] = acc;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ wb, size_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    wb[i] = __float2bfloat16(pi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ p, size_t n, __nv_bfloat16* __restrict__ wb) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    wb[i] = __float2bfloat16(p[i]);
}

// Predicted FoM (Eq. 8-9) from predicted dB values out[b][q * F + f] (q = 0 S11, 1 S21, 2 S31,
// 3 S32), scaled by out_scale.
__global__ void fom_from_db_kernel(const float* __restrict__ out, int B, int F, float out_scale,
                                   const uint8_t* __restrict__ bands, double* __restrict__ fom) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* o = out + static_cast<size_t>(b) * 4 * F;
  double sum = 0.0;
  for (int f = 0; f < F; ++f) {
    const double s11 = o[f] / out_scale, s21 = o[F + f] / out_scale, s31 = o[2 * F + f] / out_scale,
                 s32 = o[3 * F + f] / out_scale;
    switch (bands[f]) {
      case 0: sum += pow(10.0, -(s21 + 1.0) / 10.0) + pow(10.0, (15.0 + s11) / 10.0) + pow(10.0, (s31 + 35.0) / 15.0); break;
      case 1: sum += pow(10.0, -(s31 + 1.0) / 10.0) + pow(10.0, (15.0 + s11) / 10.0) + pow(10.0, (s21 + 35.0) / 15.0); break;
      case 2: sum += pow(10.0, (s32 + 20.0) / 15.0); break;
      case 3: sum += pow(10.0, (s21 + 20.0) / 18.0) + pow(10.0, (s31 + 20.0) / 18.0); break;
      default: break;
    }
  }
  fom[b] = sum;
}

// Training targets from evaluated S (complex128 [B][F][P][P]): out_scale * dB of S11, S21, S31,
// S32 (R6: 20 log10 max(|S|, 1e-15)), laid out t[b][q * F + f].
__global__ void targets_kernel(const double2* __restrict__ S, int B, int F, int P, float out_scale,
                               float* __restrict__ t) {
  const size_t n = static_cast<size_t>(B) * F;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(e / F), f = static_cast<int>(e % F);
    const double2* s = S + e * P * P;
    const int idx[4] = {0, 1 * P + 0, 2 * P + 0, 2 * P + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 v = s[idx[q]];
      double m = sqrt(v.x * v.x + v.y * v.y);
      if (m < 1e-15) m = 1e-15;
      t[static_cast<size_t>(b) * 4 * F + static_cast<size_t>(q) * F + f] = static_cast<float>(out_scale * 20.0 * log10(m));
    }
  }
}

int grid_for(size_t n) {
  const size_t g = (n + 255) / 256;
  return static_cast<int>(g < 4096 ? (g < 1 ? 1 : g) : 4096);
}

pmom_status mfail(pmom_mlp* n, pmom_status st, const std::string& msg) {
  if (n) n->err = msg;
  return st;
}

#define MLP_CUDA(net, call)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return mfail(net, e_ == cudaErrorMemoryAllocation ? PMOM_ERR_OOM : PMOM_ERR_CUDA,       \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

template <typename T>
void mfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// SplitMix64 of a counter: deterministic initial weights
uint64_t smix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

pmom_status ensure_batch_mlp(pmom_mlp* n, int B) {
  if (B <= n->b_cap) return PMOM_OK;
  for (auto& h : n->d_h) mfree(h);
  mfree(n->d_out);
  mfree(n->d_dz);
  mfree(n->d_dz2);
  n->b_cap = 0;
  n->d_h.assign(n->L, nullptr);
  int dmax = 0;
  for (int d : n->dims) dmax = d > dmax ? d : dmax;
  for (int l = 0; l < n->L; ++l)
    MLP_CUDA(n, cudaMalloc(&n->d_h[l], sizeof(__nv_bfloat16) * static_cast<size_t>(B) * n->dims[l]));
  MLP_CUDA(n, cudaMalloc(&n->d_out, sizeof(float) * static_cast<size_t>(B) * n->dims[n->L]));
  MLP_CUDA(n, cudaMalloc(&n->d_dz, sizeof(__nv_bfloat16) * static_cast<size_t>(B) * dmax));
  MLP_CUDA(n, cudaMalloc(&n->d_dz2, sizeof(__nv_bfloat16) * static_cast<size_t>(B) * dmax));
  n->b_cap = B;
  return PMOM_OK;
}

pmom_status forward(pmom_mlp* n, const uint8_t* x, int B, cudaStream_t s) {
  const size_t nin = static_cast<size_t>(B) * n->dims[0];
  input_kernel<<<grid_for(nin), 256, 0, s>>>(x, nin, n->d_h[0]);
  MLP_CUDA(n, cudaGetLastError());
  for (int l = 0; l < n->L; ++l) {
    GemmArgs g{};
    g.A = n->d_h[l]; g.sam = n->dims[l]; g.sak = 1;
    g.B = n->d_wb + n->w_off[l]; g.sbn = n->dims[l]; g.sbk = 1;
    g.M = B; g.N = n->dims[l + 1]; g.K = n->dims[l];
    g.bias = n->d_p + n->b_off[l];
    g.ldo = n->dims[l + 1];
    g.err = n->d_err;
    if (l + 1 < n->L) {
      g.epi = kEpiReluBF16;
      g.out_bf16 = n->d_h[l + 1];
    } else {
      g.epi = kEpiStoreF32;
      g.out_f32 = n->d_out;
    }
    MLP_CUDA(n, gemm(g, s));
  }
  return PMOM_OK;
}

}  // namespace
}  // namespace pmom

using namespace pmom;

pmom_status pmom_mlp_create(int32_t n_layers, const int32_t* dims, uint64_t seed, pmom_mlp** out) {
  if (!out || n_layers < 1 || n_layers > 8 || !dims) return PMOM_ERR_INVALID_ARG;
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] < 1 || dims[l] > 65536) return PMOM_ERR_INVALID_ARG;
  auto* n = new pmom_mlp();
  n->L = n_layers;
  n->dims.assign(dims, dims + n_layers + 1);
  size_t off = 0;
  for (int l = 0; l < n_layers; ++l) {
    n->w_off.push_back(off);
    off += static_cast<size_t>(dims[l + 1]) * dims[l];
    n->b_off.push_back(off);
    off += dims[l + 1];
  }
  n->n_params = off;
  // He-uniform initial weights from a counter-based generator, zero biases
  std::vector<float> p(off, 0.f);
  for (int l = 0; l < n_layers; ++l) {
    const double a = std::sqrt(6.0 / dims[l]);
    for (size_t i = 0; i < static_cast<size_t>(dims[l + 1]) * dims[l]; ++i) {
      const double u = static_cast<double>(smix(seed ^ smix((static_cast<uint64_t>(l) << 48) + i)) >> 11) *
                       (1.0 / 9007199254740992.0);
      p[n->w_off[l] + i] = static_cast<float>((2.0 * u - 1.0) * a);
    }
  }
  bool ok = true;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (ok && cudaMalloc(ptr, bytes) != cudaSuccess) ok = false;
  };
  alloc(reinterpret_cast<void**>(&n->d_p), sizeof(float) * off);
  alloc(reinterpret_cast<void**>(&n->d_g), sizeof(float) * off);
  alloc(reinterpret_cast<void**>(&n->d_m), sizeof(float) * off);
  alloc(reinterpret_cast<void**>(&n->d_v), sizeof(float) * off);
  alloc(reinterpret_cast<void**>(&n->d_wb), sizeof(__nv_bfloat16) * off);
  alloc(reinterpret_cast<void**>(&n->d_loss), sizeof(double));
  alloc(reinterpret_cast<void**>(&n->d_err), sizeof(int));
  pmom_status st = ok ? PMOM_OK : PMOM_ERR_OOM;
  if (!st && (cudaMemcpy(n->d_p, p.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
              cudaMemset(n->d_m, 0, sizeof(float) * off) != cudaSuccess ||
              cudaMemset(n->d_v, 0, sizeof(float) * off) != cudaSuccess ||
              cudaMemset(n->d_g, 0, sizeof(float) * off) != cudaSuccess ||
              cudaMemset(n->d_err, 0, sizeof(int)) != cudaSuccess))
    st = PMOM_ERR_CUDA;
  if (!st) {
    to_bf16_kernel<<<grid_for(off), 256>>>(n->d_p, off, n->d_wb);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) st = PMOM_ERR_CUDA;
  }
  if (st) {
    pmom_mlp_destroy(n);
    return st;
  }
  *out = n;
  return PMOM_OK;
}

pmom_status pmom_mlp_destroy(pmom_mlp* n) {
  if (!n) return PMOM_OK;
  mfree(n->d_p);
  mfree(n->d_g);
  mfree(n->d_m);
  mfree(n->d_v);
  mfree(n->d_wb);
  mfree(n->d_out);
  mfree(n->d_dz);
  mfree(n->d_dz2);
  mfree(n->d_loss);
  mfree(n->d_err);
  for (auto& h : n->d_h) mfree(h);
  delete n;
  return PMOM_OK;
}

const char* pmom_mlp_last_error(const pmom_mlp* n) { return n ? n->err.c_str() : "null network"; }

pmom_status pmom_mlp_num_params(const pmom_mlp* n, int64_t* count) {
  if (!n || !count) return PMOM_ERR_INVALID_ARG;
  *count = static_cast<int64_t>(n->n_params);
  return PMOM_OK;
}

pmom_status pmom_mlp_get_params(pmom_mlp* n, float* params_host, float* grads_host) {
  if (!n) return PMOM_ERR_INVALID_ARG;
  MLP_CUDA(n, cudaDeviceSynchronize());
  if (params_host) MLP_CUDA(n, cudaMemcpy(params_host, n->d_p, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
  if (grads_host) MLP_CUDA(n, cudaMemcpy(grads_host, n->d_g, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost));
  return PMOM_OK;
}

pmom_status pmom_mlp_set_params(pmom_mlp* n, const float* params_host) {
  if (!n || !params_host) return PMOM_ERR_INVALID_ARG;
  MLP_CUDA(n, cudaMemcpy(n->d_p, params_host, sizeof(float) * n->n_params, cudaMemcpyHostToDevice));
  to_bf16_kernel<<<grid_for(n->n_params), 256>>>(n->d_p, n->n_params, n->d_wb);
  MLP_CUDA(n, cudaGetLastError());
  MLP_CUDA(n, cudaMemset(n->d_m, 0, sizeof(float) * n->n_params));
  MLP_CUDA(n, cudaMemset(n->d_v, 0, sizeof(float) * n->n_params));
  n->t = 0;
  MLP_CUDA(n, cudaDeviceSynchronize());
  return PMOM_OK;
}

pmom_status pmom_mlp_forward(pmom_mlp* n, const uint8_t* x, int32_t B, float* y, void* stream) {
  if (!n || !x || !y || B < 1) return PMOM_ERR_INVALID_ARG;
  pmom_status st = ensure_batch_mlp(n, B);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = forward(n, x, B, s);
  if (st) return st;
  MLP_CUDA(n, cudaMemcpyAsync(y, n->d_out, sizeof(float) * static_cast<size_t>(B) * n->dims[n->L],
                              cudaMemcpyDeviceToDevice, s));
  return PMOM_OK;
}

pmom_status pmom_mlp_backward(pmom_mlp* n, const uint8_t* x, const float* target, int32_t B, double* loss_host,
                              void* stream) {
  if (!n || !x || !target || B < 1) return PMOM_ERR_INVALID_ARG;
  pmom_status st = ensure_batch_mlp(n, B);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = forward(n, x, B, s);
  if (st) return st;
  const int L = n->L;
  const size_t nout = static_cast<size_t>(B) * n->dims[L];
  MLP_CUDA(n, cudaMemsetAsync(n->d_loss, 0, sizeof(double), s));
  const int lg = grid_for(nout) < 256 ? grid_for(nout) : 256;
  loss_kernel<<<lg, 256, 0, s>>>(n->d_out, target, nout, 1.0 / static_cast<double>(nout), n->d_dz, n->d_loss);
  MLP_CUDA(n, cudaGetLastError());
  __nv_bfloat16* dz = n->d_dz;     // gradient of z_l, B x d_{l+1}
  __nv_bfloat16* dh = n->d_dz2;
  for (int l = L - 1; l >= 0; --l) {
    const int din = n->dims[l], dout = n->dims[l + 1];
    // dW_l (dout x din) = dz^T h_l: A(m = out unit, k = batch), B(n = in unit, k = batch)
    GemmArgs g{};
    g.A = dz; g.sam = 1; g.sak = dout;
    g.B = n->d_h[l]; g.sbn = 1; g.sbk = din;
    g.M = dout; g.N = din; g.K = B;
    g.epi = kEpiStoreF32; g.out_f32 = n->d_g + n->w_off[l]; g.ldo = din; g.err = n->d_err;
    MLP_CUDA(n, gemm(g, s));
    bias_grad_kernel<<<(dout + 127) / 128, 128, 0, s>>>(dz, B, dout, n->d_g + n->b_off[l]);
    MLP_CUDA(n, cudaGetLastError());
    if (l > 0) {
      // dz_{l-1} (B x din) = (dz W_l) * relu'(h_l): A(m = batch, k = out unit), B(n = in unit, k = out unit)
      GemmArgs h{};
      h.A = dz; h.sam = dout; h.sak = 1;
      h.B = n->d_wb + n->w_off[l]; h.sbn = 1; h.sbk = din;
      h.M = B; h.N = din; h.K = dout;
      h.epi = kEpiMaskBF16; h.mask = n->d_h[l]; h.out_bf16 = dh; h.ldo = din; h.err = n->d_err;
      MLP_CUDA(n, gemm(h, s));
      __nv_bfloat16* t = dz;
      dz = dh;
      dh = t;
    }
  }
  if (loss_host) {
    MLP_CUDA(n, cudaMemcpyAsync(loss_host, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(n, cudaStreamSynchronize(s));
  }
  return PMOM_OK;
}

pmom_status pmom_mlp_adam(pmom_mlp* n, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!n || !(lr > 0.f)) return PMOM_ERR_INVALID_ARG;
  n->t += 1;
  const float c1 = 1.f - std::pow(beta1, static_cast<float>(n->t));
  const float c2 = 1.f - std::pow(beta2, static_cast<float>(n->t));
  adam_kernel<<<grid_for(n->n_params), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n->d_p, n->d_g, n->d_m, n->d_v, n->d_wb, n->n_params, lr, beta1, beta2, eps, c1, c2);
  MLP_CUDA(n, cudaGetLastError());
  return PMOM_OK;
}

pmom_status pmom_mlp_predict_fom(pmom_mlp* n, const uint8_t* x, int32_t B, const uint8_t* bands, int32_t F,
                                 float out_scale, double* fom, void* stream) {
  if (!n || !x || !bands || !fom || B < 1 || F < 1 || n->dims[n->L] != 4 * F || !(out_scale > 0.f))
    return PMOM_ERR_INVALID_ARG;
  pmom_status st = ensure_batch_mlp(n, B);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = forward(n, x, B, s);
  if (st) return st;
  fom_from_db_kernel<<<(B + 127) / 128, 128, 0, s>>>(n->d_out, B, F, out_scale, bands, fom);
  MLP_CUDA(n, cudaGetLastError());
  return PMOM_OK;
}

pmom_status pmom_mlp_errors(pmom_mlp* n, int32_t* timeouts) {
  if (!n || !timeouts) return PMOM_ERR_INVALID_ARG;
  MLP_CUDA(n, cudaMemcpy(timeouts, n->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  return PMOM_OK;
}

pmom_status pmom_mlp_targets(const double* S_dev, int32_t B, int32_t F, int32_t P, float out_scale,
                             float* target_dev, void* stream) {
  if (!S_dev || !target_dev || B < 1 || F < 1 || P < 3 || P > 4) return PMOM_ERR_INVALID_ARG;
  const size_t n = static_cast<size_t>(B) * F;
  targets_kernel<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const double2*>(S_dev), B, F, P, out_scale, target_dev);
  return cudaGetLastError() == cudaSuccess ? PMOM_OK : PMOM_ERR_CUDA;
}
