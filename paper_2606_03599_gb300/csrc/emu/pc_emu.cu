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
#include "../pc_apply_tma.cuh"

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

// Same step sequence as apply_tma_kernel; a box copy is modelled as an immediate copy with zero fill.
template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
static void emu_run_tma(const StencilParams<R>& P, int block, const void* x, void* y, const void* mat, double shift,
                        int tz) {
    using T = TmaTile<R, FULL, CUBIC, MATK, TX, TY>;
    using C = typename CT<R>::T;
    const int ntx = (P.X + TX - 1) / TX, nty = (P.Y + TY - 1) / TY, nch = (P.Z + tz - 1) / tz;
    std::vector<typename T::Regs> regs(T::NT);
    typename T::Shared* sh = new typename T::Shared;
    for (int ch = 0; ch < nch; ++ch)
        for (int tile = 0; tile < ntx * nty; ++tile) {
            std::memset((void*)sh, 0xFF, sizeof(*sh));
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
            const int kfirst = c.k0 - 2, klast = c.k0 + c.tz + 1;
            for (int t = 0; t < T::NT; ++t) T::load_tables(c, *sh, t);
            for (int t = 0; t < T::NT; ++t) T::init(c, *sh, t, regs[t]);
            for (int kp = kfirst; kp <= klast && kp < kfirst + T::NSLOT; ++kp) T::host_copy_box(c, *sh, kp);
            for (int kp = kfirst; kp < c.k0; ++kp)
                for (int t = 0; t < T::NT; ++t) {
                    T::prefetch_fix(c, regs[t], t, kp);
                    T::apply_fix(c, *sh, regs[t], t, kp);
                }
            for (int t = 0; t < T::NT; ++t) {
                T::prefetch_fix(c, regs[t], t, c.k0);
                int wk;
                const int kw = T::wrapc(c.k0 - 1, P.Z, wk);
                regs[t].fm_cur = regs[t].fvalid ? T::read_mat(c.mat, (int64_t)kw * c.plane + regs[t].foff) : (R)0;
            }
            for (int kf = c.k0 - 1; kf <= c.k0 + c.tz; ++kf) {
                const int p = kf + 1;
                for (int t = 0; t < T::NT; ++t) {
                    T::apply_fix(c, *sh, regs[t], t, p);
                    if (p + 1 <= klast) T::prefetch_fix(c, regs[t], t, p + 1);
                    T::load_mats(c, regs[t], kf);
                }
                if (kf - 2 >= kfirst && kf - 2 + T::NSLOT <= klast) T::host_copy_box(c, *sh, kf - 2 + T::NSLOT);
                for (int t = 0; t < T::NT; ++t) T::flux(c, *sh, regs[t], kf);
                for (int t = 0; t < T::NT; ++t) {
                    T::gather(c, *sh, regs[t], kf);
                    T::rotate_mats(regs[t]);
                }
            }
        }
    delete sh;
}

template <typename R, bool FULL, bool CUBIC, int MATK>
static int emu_shape(int shape, const StencilParams<R>& P, int block, const void* x, void* y, const void* mat,
                     double shift, int tz) {
    constexpr bool F32 = sizeof(R) == 4;
    switch (shape) {
        case 10: emu_run_tma<R, FULL, CUBIC, MATK, 16, (F32 ? 16 : 8)>(P, block, x, y, mat, shift, tz); break;
        case 11: emu_run_tma<R, FULL, CUBIC, MATK, 8, 8>(P, block, x, y, mat, shift, tz); break;
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
