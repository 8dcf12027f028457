// complex64 (FP32 arithmetic) instantiations of the fused stencil apply.
#include "pc_apply_impl.cuh"
#include "pc_apply_tma_impl.cuh"

namespace pc {
int launch_apply_f32(bool full, bool cubic, int matkind, int shape, const StencilParams<float>& P,
                     const ApplyItem* items, int nitems, int tz, double* dp, int ds, cudaStream_t s) {
    return launch_apply_t<float>(full, cubic, matkind, shape, P, items, nitems, tz, dp, ds, s);
}
int launch_apply_tma_f32(bool full, bool cubic, int matkind, int shape, const StencilParams<float>& P,
                         const ApplyItem* items, int nitems, int tz, double* dp, int ds, int* err, cudaStream_t s) {
    return launch_apply_tma_t<float>(full, cubic, matkind, shape, P, items, nitems, tz, dp, ds, err, s);
}
}  // namespace pc
