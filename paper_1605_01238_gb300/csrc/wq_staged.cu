// Entry of the staged WQ assembly (three mode-product kernels, intermediates in
// device memory): dispatch on the degree to the per-degree translation units
// wq_staged_p<P>.cu, which instantiate the kernels of wq_staged_impl.cuh.
#include "wq_internal.h"

namespace wq {

wq_status launch_staged_p2(wq_plan_s*, bool, const double*, void*, int, int, cudaStream_t, const SlabHook*);
wq_status launch_staged_p3(wq_plan_s*, bool, const double*, void*, int, int, cudaStream_t, const SlabHook*);
wq_status launch_staged_p4(wq_plan_s*, bool, const double*, void*, int, int, cudaStream_t, const SlabHook*);
wq_status launch_staged_p5(wq_plan_s*, bool, const double*, void*, int, int, cudaStream_t, const SlabHook*);
wq_status launch_staged_p6(wq_plan_s*, bool, const double*, void*, int, int, cudaStream_t, const SlabHook*);
wq_status launch_staged_p7(wq_plan_s*, bool, const double*, void*, int, int, cudaStream_t, const SlabHook*);
wq_status launch_staged_p8(wq_plan_s*, bool, const double*, void*, int, int, cudaStream_t, const SlabHook*);

wq_status launch_staged(wq_plan_s* pl, bool mass, const double* kappa, void* vals, int value_dtype, int precision,
                        cudaStream_t s, const SlabHook* hook) {
  switch (pl->p) {
    case 2: return launch_staged_p2(pl, mass, kappa, vals, value_dtype, precision, s, hook);
    case 3: return launch_staged_p3(pl, mass, kappa, vals, value_dtype, precision, s, hook);
    case 4: return launch_staged_p4(pl, mass, kappa, vals, value_dtype, precision, s, hook);
    case 5: return launch_staged_p5(pl, mass, kappa, vals, value_dtype, precision, s, hook);
    case 6: return launch_staged_p6(pl, mass, kappa, vals, value_dtype, precision, s, hook);
    case 7: return launch_staged_p7(pl, mass, kappa, vals, value_dtype, precision, s, hook);
    case 8: return launch_staged_p8(pl, mass, kappa, vals, value_dtype, precision, s, hook);
    default: return set_error(WQ_ERR_UNSUPPORTED, "degree out of range");
  }
}

}  // namespace wq
