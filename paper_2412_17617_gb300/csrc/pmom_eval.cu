// Candidate-evaluation launchers for sm_103a: the default-layout evaluation kernels, the
// activation, ordering, Y -> S, FoM and gather kernels.  The large-support-set variants are
// compiled in pmom_eval_large.cu (a separate translation unit so the two build in parallel).
#include <atomic>

#include "pmom_eval_kernels.cuh"

namespace pmom {

cudaError_t launch_activate(const EvalArgs& a, cudaStream_t s) {
  activate_kernel<<<a.B, kThreads, 0, s>>>(a.rules, a.M, a.maps, a.npix, a.n_states, a.via_top, a.idx, a.n_act, a.flags,
                                            a.n_max);
  return cudaGetLastError();
}

bool eval_is_large(int precision, int ncap, int use_tc) {
  return precision == PMOM_FP64 ? needs_large_layout<double2>(ncap, false) : needs_large_layout<float2>(ncap, use_tc != 0);
}

// Failure-detection self-test of the bounded completion wait used by the tensor-core paths: one
// warp initialises an mbarrier that expects one arrival; with `arrive` thread 0 arrives before
// waiting, otherwise nothing ever arrives (a flag that nothing sets).  The wait polls at most
// `polls` times and out[0] reports whether it gave up (1) or saw the phase complete (0).
__global__ void wait_selftest_kernel(long long polls, int arrive, int* out) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) {
      uint64_t state;
      asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(tc::smem_u32(&mbar)) : "memory");
      (void)state;
    }
    out[0] = tc::mbar_wait(&mbar, 0, polls) ? 0 : 1;
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(tc::smem_u32(&mbar)) : "memory");
  }
}

cudaError_t launch_wait_selftest(long long polls, int arrive, int* d_out, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(polls, arrive, d_out);
  return cudaGetLastError();
}

void* tensor_map_encoder_ptr() {
  static std::atomic<void*> cached{nullptr};
  void* p = cached.load(std::memory_order_acquire);
  if (p == nullptr) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;   // not kept: a later call looks again
    cached.store(p, std::memory_order_release);
  }
  return p;
}

cudaError_t launch_eval(const EvalArgs& a, int precision, int nslots, cudaStream_t s) {
  if (eval_is_large(precision, a.ncap, a.use_tc)) return launch_eval_large(a, precision, nslots, s);
  if (precision == PMOM_FP64) {
    return a.z_c128 ? launch_eval_t<double2, double2, false, false, false>(a, nslots, s)
                    : launch_eval_t<double2, float2, false, false, false>(a, nslots, s);
  }
  if (a.use_tc)
    return a.z_c128 ? launch_eval_t<float2, double2, true, true, false>(a, nslots, s)
                    : launch_eval_t<float2, float2, true, true, false>(a, nslots, s);
  return a.z_c128 ? launch_eval_t<float2, double2, true, false, false>(a, nslots, s)
                  : launch_eval_t<float2, float2, true, false, false>(a, nslots, s);
}

int eval_blocks_per_sm(int precision, int ncap, int z_c128, int use_tc, int max_groups) {
  if (eval_is_large(precision, ncap, use_tc)) return eval_blocks_per_sm_large(precision, ncap, z_c128, max_groups);
  if (precision == PMOM_FP64)
    return z_c128 ? blocks_per_sm_t<double2, double2, false, false, false>(ncap, max_groups)
                  : blocks_per_sm_t<double2, float2, false, false, false>(ncap, max_groups);
  if (use_tc)
    return z_c128 ? blocks_per_sm_t<float2, double2, true, true, false>(ncap, max_groups)
                  : blocks_per_sm_t<float2, float2, true, true, false>(ncap, max_groups);
  return z_c128 ? blocks_per_sm_t<float2, double2, true, false, false>(ncap, max_groups)
                : blocks_per_sm_t<float2, float2, true, false, false>(ncap, max_groups);
}

int eval_groups_max(int precision, int ncap, int use_tc) {
  const bool large = eval_is_large(precision, ncap, use_tc);
  if (precision == PMOM_FP64) return groups_for<double2>(ncap, false, large);
  return groups_for<float2>(ncap, large || use_tc != 0, large);
}

int eval_max_ncap(int precision, int M) {
  // largest support set whose large-layout task group fits one CTA (binary search on the layout)
  const size_t optin = static_cast<size_t>(optin_smem());
  auto fits = [&](int n) {
    const size_t b = precision == PMOM_FP64 ? group_smem_bytes<double2>(n, 0, true) : group_smem_bytes<float2>(n, 1, true);
    return b + kStaticSmemSlack <= optin;
  };
  if (fits(M)) return M;
  int lo = 1, hi = M;   // fits(lo), !fits(hi)
  while (hi - lo > 1) {
    const int mid = lo + (hi - lo) / 2;
    if (fits(mid)) lo = mid; else hi = mid;
  }
  return lo;
}

size_t eval_slot_bytes(int precision, int ncap, int P, int* lda) {
  *lda = (ncap + 3) & ~3;
  const size_t ct = precision == PMOM_FP64 ? sizeof(double2) : sizeof(float2);
  const Slot s = slot_layout(ncap, *lda, P, ct);
  return (s.end + 255) & ~size_t(255);
}

size_t eval_smem_bytes(int precision, int ncap, int use_tc) {
  size_t u_off, idx_off, tc_off;
  const bool large = eval_is_large(precision, ncap, use_tc);
  return precision == PMOM_FP64 ? smem_layout<double2>(ncap, 0, large, &u_off, &idx_off, &tc_off)
                                : smem_layout<float2>(ncap, large ? 1 : use_tc, large, &u_off, &idx_off, &tc_off);
}

cudaError_t launch_order(const int32_t* n_act, int B, int M, int* order, cudaStream_t s) {
  order_kernel<<<1, 256, sizeof(int) * (M + 2), s>>>(n_act, B, M, order);
  return cudaGetLastError();
}

cudaError_t launch_ys(double2* S, int B, int F, int P, double Z0, uint32_t* flags, cudaStream_t s) {
  const int n = B * F;
  ys_kernel<<<(n + 127) / 128, 128, 0, s>>>(S, n, F, P, Z0, flags);
  return cudaGetLastError();
}

cudaError_t launch_fom(const double2* S, const uint8_t* bands, int F, int P, int B, const uint32_t* flags,
                       const int32_t* n_act, double* fom, int32_t* status, cudaStream_t s) {
  fom_kernel<<<(B + 127) / 128, 128, 0, s>>>(S, bands, F, P, B, flags, n_act, fom, status);
  return cudaGetLastError();
}

cudaError_t launch_gather(const void* Z, int z_c128, int M, int f, const int32_t* idx, int N, void* out,
                          cudaStream_t s) {
  const int grid = N < 1024 ? (N > 0 ? N : 1) : 1024;
  if (z_c128)
    gather_kernel<double2><<<grid, 256, 0, s>>>(static_cast<const double2*>(Z), M, f, idx, N, static_cast<double2*>(out));
  else
    gather_kernel<float2><<<grid, 256, 0, s>>>(static_cast<const float2*>(Z), M, f, idx, N, static_cast<float2*>(out));
  return cudaGetLastError();
}

cudaError_t launch_gather_batch(const void* Z, int z_c128, int M, int f, const int32_t* idx, const int32_t* n, int B,
                                int ncap, void* out, cudaStream_t s) {
  const size_t zel = z_c128 ? sizeof(double2) : sizeof(float2);
  const size_t row_bytes = zel * M;
  // rows per CTA: as many as fit about 100 KB of staging (two CTAs per SM), at most 8
  int R = static_cast<int>((100u << 10) / row_bytes);
  R = R < 1 ? 1 : (R > 8 ? 8 : R);
  const int bulk = (row_bytes % 16 == 0) && row_bytes <= (100u << 10);
  const size_t smem = (bulk ? R * row_bytes : 0) + sizeof(int) * static_cast<size_t>(ncap);
  const dim3 grid(static_cast<unsigned>((ncap + R - 1) / R), static_cast<unsigned>(B));
  cudaError_t e;
  if (z_c128) {
    e = cudaFuncSetAttribute(gather_batch_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    gather_batch_kernel<double2><<<grid, 256, smem, s>>>(static_cast<const double2*>(Z), M, f, idx, n, ncap, R, bulk,
                                                          static_cast<double2*>(out));
  } else {
    e = cudaFuncSetAttribute(gather_batch_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    gather_batch_kernel<float2><<<grid, 256, smem, s>>>(static_cast<const float2*>(Z), M, f, idx, n, ncap, R, bulk,
                                                         static_cast<float2*>(out));
  }
  return cudaGetLastError();
}

}  // namespace pmom

#ifdef PMOM_PHASES
// Profiling builds only (compiled with -DPMOM_PHASES; paper_2412_17617_gb300/phases.py builds and
// reads them): the phase-clock counters of the default-layout evaluation kernels in this
// translation unit, kPhaseSlots cycle sums (slot kPhTasks counts tasks).  Not part of the public
// C ABI; the product library is built without them.
extern "C" int pmom_phase_slots() { return pmom::kPhaseSlots; }
extern "C" int pmom_phase_read(unsigned long long* out_host) {
  return static_cast<int>(
      cudaMemcpyFromSymbol(out_host, pmom::g_phase_cycles, sizeof(unsigned long long) * pmom::kPhaseSlots));
}
extern "C" int pmom_phase_reset() {
  unsigned long long z[pmom::kPhaseSlots] = {0};
  return static_cast<int>(cudaMemcpyToSymbol(pmom::g_phase_cycles, z, sizeof(z)));
}
#endif
