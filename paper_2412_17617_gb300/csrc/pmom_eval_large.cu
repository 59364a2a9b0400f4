// Large-support-set variants of the evaluation kernel (narrow panels, solve vectors in global
// memory, one task group per CTA) for support sets beyond the default shared-memory layout.  The
// single-precision path always takes the tensor-core LU here: with NBL-column panels a CUDA-core
// trailing update would stream the whole trailing matrix once per NBL columns.
#include "pmom_eval_kernels.cuh"

namespace pmom {

cudaError_t launch_eval_large(const EvalArgs& a, int precision, int nslots, cudaStream_t s) {
  if (precision == PMOM_FP64) {
    return a.z_c128 ? launch_eval_t<double2, double2, false, false, true>(a, nslots, s)
                    : launch_eval_t<double2, float2, false, false, true>(a, nslots, s);
  }
  return a.z_c128 ? launch_eval_t<float2, double2, true, true, true>(a, nslots, s)
                  : launch_eval_t<float2, float2, true, true, true>(a, nslots, s);
}

int eval_blocks_per_sm_large(int precision, int ncap, int z_c128, int max_groups) {
  if (precision == PMOM_FP64)
    return z_c128 ? blocks_per_sm_t<double2, double2, false, false, true>(ncap, max_groups)
                  : blocks_per_sm_t<double2, float2, false, false, true>(ncap, max_groups);
  return z_c128 ? blocks_per_sm_t<float2, double2, true, true, true>(ncap, max_groups)
                : blocks_per_sm_t<float2, float2, true, true, true>(ncap, max_groups);
}

}  // namespace pmom
