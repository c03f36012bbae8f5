// Staged assembly for degree 8: every precision mode of the three mode-product
// kernels, instantiated in a translation unit of its own.
#include "wq_staged_impl.cuh"

namespace wq {

wq_status launch_staged_p8(wq_plan_s* pl, bool mass, const double* kappa, void* vals, int value_dtype,
                            int precision, cudaStream_t s, const SlabHook* hook) {
  return launch_staged_deg<8>(pl, mass, kappa, vals, value_dtype, precision, s, hook);
}

}  // namespace wq
