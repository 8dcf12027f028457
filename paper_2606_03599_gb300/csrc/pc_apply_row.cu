// Row-tile stencil apply (complex64 parity blocks): runtime-width kernels, the dispatch over
// compile-time widths, and the launch-size rule.
#include <algorithm>

#include "pc_apply_row_impl.cuh"

namespace pc {

template <int XC>
static int row_width_case(int X, const StencilParams<float>& P, const ApplyItem* items, const void* const* mats,
                          int nitems, const RowGeom& G, int ctas, double* dp, int ds, int* err, cudaStream_t s,
                          bool* handled) {
    if (X != XC) return PC_OK;
    *handled = true;
    return launch_row_t<true, 0, XC>(P, items, mats, nitems, G, ctas, dp, ds, err, s);
}

int launch_row_narrow(int X, const StencilParams<float>& P, const ApplyItem* items, const void* const* mats,
                      int nitems, const RowGeom& G, int ctas, double* dp, int ds, int* err, cudaStream_t s,
                      bool* handled) {
    *handled = false;
    PC_TRY(row_width_case<16>(X, P, items, mats, nitems, G, ctas, dp, ds, err, s, handled));
    if (*handled) return PC_OK;
    PC_TRY(row_width_case<24>(X, P, items, mats, nitems, G, ctas, dp, ds, err, s, handled));
    if (*handled) return PC_OK;
    return row_width_case<32>(X, P, items, mats, nitems, G, ctas, dp, ds, err, s, handled);
}

int launch_apply_row_f32(bool cubic, int matkind, const StencilParams<float>& P, const ApplyItem* items,
                         const void* const* mats, int nitems, int ctas, double* dp, int ds, int* err, cudaStream_t s) {
    const RowGeom G = make_row_geom(P.X, P.Y, P.Z, matkind);
    for (int i = 0; i < nitems; ++i)
        if ((reinterpret_cast<uintptr_t>(items[i].x) & 15) != 0 || items[i].block < 0 || mats[i] == nullptr)
            return fail(PC_EINVAL, "apply_row: vectors must be 16-byte aligned parity-block vectors");
    if (cubic && matkind == 0 && P.X == P.Y) {
        bool handled = false;
        PC_TRY(launch_row_narrow(P.X, P, items, mats, nitems, G, ctas, dp, ds, err, s, &handled));
        if (handled) return PC_OK;
        PC_TRY(launch_row_wide(P.X, P, items, mats, nitems, G, ctas, dp, ds, err, s, &handled));
        if (handled) return PC_OK;
    }
    if (cubic) return matkind ? launch_row_t<true, 1, 0>(P, items, mats, nitems, G, ctas, dp, ds, err, s)
                              : launch_row_t<true, 0, 0>(P, items, mats, nitems, G, ctas, dp, ds, err, s);
    return matkind ? launch_row_t<false, 1, 0>(P, items, mats, nitems, G, ctas, dp, ds, err, s)
                   : launch_row_t<false, 0, 0>(P, items, mats, nitems, G, ctas, dp, ds, err, s);
}

int row_apply_ctas(int X, int Y, int Z, int matkind, int nitems, int minseg) {
    // at least `minseg` planes per CTA (each segment reloads four halo planes)
    const RowGeom G = make_row_geom(X, Y, Z, matkind);
    const int64_t W = (int64_t)std::min(nitems, kRowMaxItems) * G.nt * Z;
    if (minseg < 1) minseg = 1;
    int64_t c = (W + minseg - 1) / minseg;
    const int sm = device_sm_count();
    if (c > sm) c = sm;
    if (c < 1) c = 1;
    return (int)c;
}

bool row_geom_fits(int X, int Y, int Z, int matkind) {
    const RowGeom G = make_row_geom(X, Y, Z, matkind);
    return G.total + 128 + 1024 <= 227 * 1024 && G.NT <= kRowMaxThreads;
}

}  // namespace pc
