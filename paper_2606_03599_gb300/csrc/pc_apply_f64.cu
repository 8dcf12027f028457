// complex128 (FP64 arithmetic) instantiations of the fused stencil apply.
#include "pc_apply_impl.cuh"

namespace pc {
int launch_apply_f64(bool full, bool cubic, int matkind, int shape, const StencilParams<double>& P,
                     const ApplyItem* items, int nitems, int tz, double* dp, int ds, cudaStream_t s) {
    return launch_apply_t<double>(full, cubic, matkind, shape, P, items, nitems, tz, dp, ds, s);
}
}  // namespace pc
