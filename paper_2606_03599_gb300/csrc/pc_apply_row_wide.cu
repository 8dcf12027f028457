// Row-tile stencil apply: compile-time-width kernels for the wider quarter grids (X = 48, 64, 80,
// i.e. N = 96, 128, 160), cubic lattice, phase ids.
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

int launch_row_wide(int X, const StencilParams<float>& P, const ApplyItem* items, const void* const* mats,
                    int nitems, const RowGeom& G, int ctas, double* dp, int ds, int* err, cudaStream_t s,
                    bool* handled) {
    *handled = false;
    PC_TRY(row_width_case<48>(X, P, items, mats, nitems, G, ctas, dp, ds, err, s, handled));
    if (*handled) return PC_OK;
    PC_TRY(row_width_case<64>(X, P, items, mats, nitems, G, ctas, dp, ds, err, s, handled));
    if (*handled) return PC_OK;
    return row_width_case<80>(X, P, items, mats, nitems, G, ctas, dp, ds, err, s, handled);
}

}  // namespace pc
