// Plane-pipelined stencil apply (complex64 parity blocks): runtime-geometry kernels, the
// dispatch over compile-time widths, and the launch-size rule.
#include <algorithm>

#include "pc_apply_pipe_impl.cuh"

namespace pc {

int launch_apply_pipe_f32(bool cubic, int matkind, const StencilParams<float>& P, const ApplyItem* items,
                          const double* iph, const void* const* mats, int nitems, int ctas, double* dp, int ds,
                          int* err, cudaStream_t s) {
    const PipeGeom G = make_pipe_geom(P.X, P.Y, P.Z, matkind);
    for (int i = 0; i < nitems; ++i)
        if ((reinterpret_cast<uintptr_t>(items[i].x) & 15) != 0 || items[i].block < 0 || mats[i] == nullptr)
            return fail(PC_EINVAL, "apply_pipe: vectors must be 16-byte aligned parity-block vectors");
    if (cubic && matkind == 0 && P.X == P.Y) {
        bool handled = false;
        PC_TRY(launch_pipe_widths(P.X, P, items, iph, mats, nitems, G, ctas, dp, ds, err, s, &handled));
        if (handled) return PC_OK;
    }
    if (cubic) return matkind ? launch_pipe_t<true, 1, 0, 0>(P, items, iph, mats, nitems, G, ctas, dp, ds, err, s)
                              : launch_pipe_t<true, 0, 0, 0>(P, items, iph, mats, nitems, G, ctas, dp, ds, err, s);
    return matkind ? launch_pipe_t<false, 1, 0, 0>(P, items, iph, mats, nitems, G, ctas, dp, ds, err, s)
                   : launch_pipe_t<false, 0, 0, 0>(P, items, iph, mats, nitems, G, ctas, dp, ds, err, s);
}

int pipe_apply_ctas(int X, int Y, int Z, int matkind, int nitems, int minseg) {
    // at least `minseg` planes per CTA (each segment loads four planes beyond its outputs)
    const PipeGeom G = make_pipe_geom(X, Y, Z, matkind);
    const int64_t W = (int64_t)std::min(nitems, kPipeMaxItems) * G.nt * Z;
    if (minseg < 1) minseg = 1;
    int64_t c = (W + minseg - 1) / minseg;
    const int sm = device_sm_count();
    if (c > sm) c = sm;
    if (c < 1) c = 1;
    return (int)c;
}

bool pipe_geom_ok(int X, int Y, int Z, int matkind) {
    if (X & 1) return false;
    const PipeGeom G = make_pipe_geom(X, Y, Z, matkind);
    return pipe_geom_fits(G) && G.NC + 32 <= kPipeMaxThreads;
}

}  // namespace pc
