// complex64 (FP32 arithmetic) instantiations of the fused stencil apply.
#include "pc_apply_impl.cuh"

namespace pc {
int launch_apply_f32(bool full, bool cubic, int matkind, int shape, const StencilParams<float>& P,
                     const ApplyItem* items, int nitems, int tz, double* dp, int ds, cudaStream_t s) {
    return launch_apply_t<float>(full, cubic, matkind, shape, P, items, nitems, tz, dp, ds, s);
}
}  // namespace pc
