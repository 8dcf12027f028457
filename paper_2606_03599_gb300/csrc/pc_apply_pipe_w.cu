// Plane-pipelined stencil apply: compile-time-width kernels (cubic lattice, phase ids) for the
// quarter-grid widths X = N/2 of N = 32, 48, 64, 96, 128, 160.
#include "pc_apply_pipe_impl.cuh"

namespace pc {

template <int XC>
static int pipe_width_case(int X, const StencilParams<float>& P, const ApplyItem* items, const double* iph,
                           const void* const* mats, int nitems, const PipeGeom& G, int ctas, double* dp, int ds,
                           int* err, cudaStream_t s, bool* handled) {
    if (X != XC || G.T != pipe_rows_for(XC)) return PC_OK;
    *handled = true;
    return launch_pipe_t<true, 0, XC, pipe_rows_for(XC)>(P, items, iph, mats, nitems, G, ctas, dp, ds, err, s);
}

int launch_pipe_widths(int X, const StencilParams<float>& P, const ApplyItem* items, const double* iph,
                       const void* const* mats, int nitems, const PipeGeom& G, int ctas, double* dp, int ds, int* err,
                       cudaStream_t s, bool* handled) {
    *handled = false;
#define PC_PIPE_CASE(W)                                                                            \
    PC_TRY(pipe_width_case<W>(X, P, items, iph, mats, nitems, G, ctas, dp, ds, err, s, handled)); \
    if (*handled) return PC_OK;
    PC_PIPE_CASE(16)
    PC_PIPE_CASE(24)
    PC_PIPE_CASE(32)
    PC_PIPE_CASE(48)
    PC_PIPE_CASE(64)
    PC_PIPE_CASE(80)
#undef PC_PIPE_CASE
    return PC_OK;
}

}  // namespace pc
