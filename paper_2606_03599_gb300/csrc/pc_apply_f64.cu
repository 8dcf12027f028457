// complex128 (FP64 arithmetic) instantiations of the fused stencil apply.
#include "pc_apply_impl.cuh"
#include "pc_apply_tma_impl.cuh"

namespace pc {
int launch_apply_f64(bool full, bool cubic, int matkind, int shape, const StencilParams<double>& P,
                     const ApplyItem* items, int nitems, int tz, double* dp, int ds, cudaStream_t s) {
    return launch_apply_t<double>(full, cubic, matkind, shape, P, items, nitems, tz, dp, ds, s);
}
int launch_apply_tma_f64(bool full, bool cubic, int matkind, int shape, const StencilParams<double>& P,
                         const ApplyItem* items, int nitems, int tz, double* dp, int ds, int* err, cudaStream_t s) {
    return launch_apply_tma_t<double>(full, cubic, matkind, shape, P, items, nitems, tz, dp, ds, err, s);
}
}  // namespace pc
