// Host emulator of the fused stencil kernel: runs the kernel's per-thread phase
// functions sequentially over the simulated threads of every CTA, with index
// checks on every shared-memory and global access.  Support code for the CPU
// tests of the kernel's tiling and Bloch-wrap arithmetic; it is not part of
// the product library.
#define PC_EMU_CHECK 1
#include <cstdio>
#include <cstring>
#include <vector>

#include "../pc_apply_tile.cuh"

using namespace pc;

template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
static void emu_run(const StencilParams<R>& P, int block, const void* x, void* y, const void* mat,
                    double shift, int tz) {
    using T = ApplyTile<R, FULL, CUBIC, MATK, TX, TY>;
    using C = typename CT<R>::T;
    const int ntx = (P.X + TX - 1) / TX, nty = (P.Y + TY - 1) / TY, nch = (P.Z + tz - 1) / tz;
    std::vector<typename T::Regs> regs(T::NT);
    typename T::Shared* sh = new typename T::Shared;
    for (int ch = 0; ch < nch; ++ch)
        for (int tile = 0; tile < ntx * nty; ++tile) {
            std::memset((void*)sh, 0xFF, sizeof(*sh));  // poison: reads of unwritten cells show up as NaN
            typename T::Ctx c;
            c.P = &P;
            c.x = static_cast<const C*>(x);
            c.y = static_cast<C*>(y);
            c.mat = mat;
            c.shift = (R)shift;
            c.a0 = (tile % ntx) * TX;
            c.b0 = (tile / ntx) * TY;
            c.k0 = ch * tz;
            c.tz = tz < P.Z - c.k0 ? tz : P.Z - c.k0;
            c.p12 = FULL ? 0 : (block >> 1);
            c.p13 = FULL ? 0 : (block & 1);
            c.plane = (int64_t)P.X * P.Y;
            c.vstr = c.plane * P.Z;
            for (int t = 0; t < T::NT; ++t) T::load_tables(c, *sh, t);
            for (int t = 0; t < T::NT; ++t) T::init(c, t, regs[t]);
            for (int t = 0; t < T::NT; ++t) T::prologue_load(c, *sh, regs[t], t);
            for (int kf = c.k0 - 1; kf <= c.k0 + c.tz; ++kf) {
                for (int t = 0; t < T::NT; ++t) T::phaseA(c, *sh, regs[t], t, kf);
                for (int t = 0; t < T::NT; ++t) T::phaseB(c, *sh, regs[t], kf);
            }
        }
    delete sh;
}

template <typename R, bool FULL, bool CUBIC, int MATK>
static int emu_shape(int shape, const StencilParams<R>& P, int block, const void* x, void* y, const void* mat,
                     double shift, int tz) {
    switch (shape) {
        case 0: emu_run<R, FULL, CUBIC, MATK, 32, 8>(P, block, x, y, mat, shift, tz); break;
        case 1: emu_run<R, FULL, CUBIC, MATK, 16, 8>(P, block, x, y, mat, shift, tz); break;
        case 2: emu_run<R, FULL, CUBIC, MATK, 8, 8>(P, block, x, y, mat, shift, tz); break;
        default: emu_run<R, FULL, CUBIC, MATK, 4, 4>(P, block, x, y, mat, shift, tz); break;
    }
    return 0;
}

template <typename R>
static int emu_t(int shape, const StencilParams<R>& P, bool full, bool cubic, int matkind, int block,
                 const void* x, void* y, const void* mat, double shift, int tz) {
    if (full) {
        if (cubic) return matkind ? emu_shape<R, true, true, 1>(shape, P, block, x, y, mat, shift, tz)
                                  : emu_shape<R, true, true, 0>(shape, P, block, x, y, mat, shift, tz);
        return matkind ? emu_shape<R, true, false, 1>(shape, P, block, x, y, mat, shift, tz)
                       : emu_shape<R, true, false, 0>(shape, P, block, x, y, mat, shift, tz);
    }
    if (cubic) return matkind ? emu_shape<R, false, true, 1>(shape, P, block, x, y, mat, shift, tz)
                              : emu_shape<R, false, true, 0>(shape, P, block, x, y, mat, shift, tz);
    return matkind ? emu_shape<R, false, false, 1>(shape, P, block, x, y, mat, shift, tz)
                   : emu_shape<R, false, false, 0>(shape, P, block, x, y, mat, shift, tz);
}

extern "C" int pc_emu_apply(int N, int block, int dtype, int shape, int tz, const double* Chat72,
                            const double* rhohat2, const double* ainv9, int cubic, const double* phi3,
                            const void* mat, int matkind, const void* x, void* y, double shift) {
    double Chat[2][36];
    std::memcpy(Chat, Chat72, sizeof(Chat));
    const bool full = block < 0;
    const int X = full ? N : N / 2, Y = X, Z = N;
    if (dtype == PC_C64) {
        StencilParams<float> P;
        make_stencil_params(P, Chat, rhohat2, ainv9, cubic != 0, N, phi3, X, Y, Z);
        return emu_t<float>(shape, P, full, cubic != 0, matkind, block, x, y, mat, shift, tz);
    }
    StencilParams<double> P;
    make_stencil_params(P, Chat, rhohat2, ainv9, cubic != 0, N, phi3, X, Y, Z);
    return emu_t<double>(shape, P, full, cubic != 0, matkind, block, x, y, mat, shift, tz);
}
