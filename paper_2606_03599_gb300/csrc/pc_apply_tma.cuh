// Fused stencil apply, TMA-staged variant (quarter grids of even width).
//
// Same operator and step structure as pc_apply_tile.cuh (see there for the
// algebra); what changes is the data movement and the thread mapping:
//
// * x planes arrive by one 4D tensor copy per plane (cp.async.bulk.tensor:
//   the box [a0-2, a0+TX+2) x [b0-2, b0+TY+2) x 1 plane x 3 components) into a
//   ring of NSLOT shared-memory slots, each completed through an mbarrier; a
//   plane is requested three steps before it is needed.  The box starts at an
//   even a so that its first element is 16-byte aligned for 8-byte elements.
// * Cells of the box that lie outside the quarter grid (Bloch wrap) come back
//   zero-filled; the thread that owns such a cell loads the wrapped value
//   itself (one step ahead, into a register) and stores it times its Bloch
//   phase after the plane has landed.  Planes outside [0, Z) are fetched from
//   the wrapped k and every cell is multiplied by exp(+-i phi_3).
// * One thread per flux column; the parity-dependent neighbour offsets reduce
//   to a per-step delta i0 + XW j0 added to compile-time constants.
// * The 6x6 stiffness table is stored as duplicated (c, c) pairs so that each
//   real-times-complex FMA is one packed FP32x2 instruction.
//
// Every mbarrier wait is bounded; a CTA whose copy does not arrive in time
// records an error code and leaves after waiting (bounded) for its copies in
// flight, so no wait can hang the GPU.
#pragma once

#include <math.h>
#include <stdint.h>

#include <cuda.h>

#include "pc_apply_tile.cuh"

namespace pc {

constexpr int kTmaMaxItems = 32;

struct TmaBatch {
    CUtensorMap map[kTmaMaxItems];  // one tensor map per item's x vector
    ApplyItem it[kTmaMaxItems];
    int n;
    int* err;             // device error word (nonzero after a timed-out wait)
    uint32_t wait_limit;  // mbarrier polls before a CTA gives up
};

// Stiffness entries as packed-FMA operands: (c, c) pairs for complex64, plain doubles for complex128.
PC_HD float2 stiff_pair(float v) { return make_float2(v, v); }
PC_HD double stiff_pair(double v) { return v; }
PC_HD float2 stiff_fma_pair(float2 c, float2 e, float2 acc) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    return __ffma2_rn(c, e, acc);
#else
    return make_float2(fmaf(c.x, e.x, acc.x), fmaf(c.y, e.y, acc.y));
#endif
}
PC_HD double2 stiff_fma_pair(double c, double2 e, double2 acc) { return cfma(c, e, acc); }

template <typename R> struct PairT;
template <> struct PairT<float> { using T = float2; };
template <> struct PairT<double> { using T = double; };

#if defined(__CUDACC__)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
#endif

template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
struct TmaTile {
    using C = typename CT<R>::T;
    using PR = typename PairT<R>::T;
    static constexpr int XW = TX + 4, XH = TY + 4, XR = XW * XH;  // x box
    static constexpr int FW = TX + 1, FH = TY + 2, FR = FW * FH;  // flux columns
    static constexpr int NY = TX * TY;                            // output columns
    static constexpr int NT = ((FR + 31) / 32) * 32;               // one flux column per thread
    static constexpr int NSLOT = 6;
    static constexpr int SLOT_ELEMS = 3 * XR;
    static constexpr int SLOT_BYTES = ((SLOT_ELEMS * (int)sizeof(C) + 127) / 128) * 128;
    static constexpr int NFIX = (3 * XR + NT - 1) / NT;  // box cells per thread (wrap fix-ups)

    struct Shared {
        alignas(128) unsigned char xs[NSLOT][SLOT_BYTES];
        C fs[5][3][FR];
        alignas(16) PR Cp[2][36];  // stiffness entries (duplicated pairs for complex64)
        R rho[2];
        uint64_t mbar[NSLOT];
        int abort;
    };

    struct Ctx {
        const StencilParams<R>* P;
        const C* x;
        C* y;
        const void* mat;
        R shift;
        int a0, b0, k0, tz;
        int p12, p13;
        int64_t plane, vstr;
    };

    struct Regs {
        // flux column
        bool fvalid;
        int fown;       // x-box index of the column's own node (parity independent)
        int fcol;       // flux-region index
        int foff;       // wrapped in-plane material offset
        R fm_cur, fm_nxt;
        // output column
        bool yvalid;
        int tx, ty, yoff, fbase, xown;
        R ym_cur, ym_nxt;
        C acc_prev[3], acc_cur[3], acc_next[3];
        R dot;
        // wrap fix-up cells of the x box owned by this thread
        int fxoff[NFIX];   // wrapped in-plane offset (a + X b), -1 = not wrapped in a/b
        int fxwa[NFIX], fxwb[NFIX];
        C fxval[NFIX];     // prefetched wrapped value of the next plane
    };

    static PC_HD int wrapc(int v, int n, int& w) {
        w = 0;
        while (v < 0) { v += n; --w; }
        while (v >= n) { v -= n; ++w; }
        return v;
    }

    static PC_HD C* slot_ptr(Shared& sh, int kp, int k0) {
        return reinterpret_cast<C*>(sh.xs[(kp - (k0 - 2)) % NSLOT]);
    }
    static PC_HD const C* slot_ptr(const Shared& sh, int kp, int k0) {
        return reinterpret_cast<const C*>(sh.xs[(kp - (k0 - 2)) % NSLOT]);
    }

    static PC_HD R read_mat(const void* mat, int64_t idx) {
        if (MATK == 0) return (R)(static_cast<const uint8_t*>(mat)[idx]);
        return (R)(static_cast<const float*>(mat)[idx]);
    }

    static PC_HD C wrap_phase(const StencilParams<R>& P, int wa, int wb, int wk) {
        return ApplyTile<R, FULL, CUBIC, MATK, TX, TY>::wrap_phase(P, wa, wb, wk);
    }

    static PC_HD void init(const Ctx& c, Shared& sh, int tid, Regs& r) {
        const StencilParams<R>& P = *c.P;
        r.fvalid = tid < FR;
        const int fcol = r.fvalid ? tid : 0;
        const int fa = fcol % FW, fb = fcol / FW;
        r.fcol = fcol;
        r.fown = (fa + 2) + XW * (fb + 1);
        int wa, wb;
        r.foff = wrapc(c.a0 + fa, P.X, wa) + P.X * wrapc(c.b0 - 1 + fb, P.Y, wb);
        r.fm_cur = r.fm_nxt = (R)0;
        r.tx = tid % TX;
        r.ty = tid / TX;
        const int ya = c.a0 + r.tx, yb = c.b0 + r.ty;
        r.yvalid = tid < NY && ya < P.X && yb < P.Y;
        r.yoff = r.yvalid ? ya + P.X * yb : 0;
        r.fbase = r.tx + FW * (r.ty + 1);
        r.xown = (r.tx + 2) + XW * (r.ty + 2);
        r.ym_cur = r.ym_nxt = (R)0;
        for (int a = 0; a < 3; ++a) r.acc_prev[a] = r.acc_cur[a] = r.acc_next[a] = czero((R)0);
        r.dot = (R)0;
#pragma unroll
        for (int i = 0; i < NFIX; ++i) {
            const int cell = tid + i * NT;
            r.fxoff[i] = -1;
            r.fxwa[i] = r.fxwb[i] = 0;
            r.fxval[i] = czero((R)0);
            if (cell < 3 * XR) {
                const int col = cell % XR;
                const int ra = col % XW, rb = col / XW;
                int a = wrapc(c.a0 - 2 + ra, P.X, wa);
                int b = wrapc(c.b0 - 2 + rb, P.Y, wb);
                if (wa != 0 || wb != 0) {
                    r.fxoff[i] = a + P.X * b;
                    r.fxwa[i] = wa;
                    r.fxwb[i] = wb;
                }
            }
        }
        (void)sh;
    }

    // Wrapped-cell values of plane kp into registers (loads issued one step ahead).
    static PC_HD void prefetch_fix(const Ctx& c, Regs& r, int tid, int kp) {
        const StencilParams<R>& P = *c.P;
        int wk;
        const int k = wrapc(kp, P.Z, wk);
#pragma unroll
        for (int i = 0; i < NFIX; ++i) {
            if (r.fxoff[i] < 0) continue;
            const int comp = (tid + i * NT) / XR;
            const int64_t gi = comp * c.vstr + (int64_t)k * c.plane + r.fxoff[i];
            PC_IDX(gi, 3 * c.vstr);
            r.fxval[i] = cmul(c.x[gi], wrap_phase(P, r.fxwa[i], r.fxwb[i], wk));
        }
    }

    // After plane kp has landed: store wrapped cells; for planes outside [0, Z) multiply the rest by the k phase.
    static PC_HD void apply_fix(const Ctx& c, Shared& sh, const Regs& r, int tid, int kp) {
        const StencilParams<R>& P = *c.P;
        int wk;
        wrapc(kp, P.Z, wk);
        C* s = slot_ptr(sh, kp, c.k0);
        if (wk != 0) {
            const C ph = wrap_phase(P, 0, 0, wk);
#pragma unroll
            for (int i = 0; i < NFIX; ++i) {
                const int cell = tid + i * NT;
                if (cell >= 3 * XR) continue;
                PC_IDX(cell, SLOT_ELEMS);
                s[cell] = (r.fxoff[i] >= 0) ? r.fxval[i] : cmul(s[cell], ph);
            }
        } else {
#pragma unroll
            for (int i = 0; i < NFIX; ++i) {
                if (r.fxoff[i] < 0) continue;
                const int cell = tid + i * NT;
                PC_IDX(cell, SLOT_ELEMS);
                s[cell] = r.fxval[i];
            }
        }
    }

    static PC_HD void load_tables(const Ctx& c, Shared& sh, int tid) {
        for (int i = tid; i < 72; i += NT) {
            const R v = c.P->C[i / 36][i % 36];
            sh.Cp[i / 36][i % 36] = pair_of(v);
        }
        if (tid < 2) sh.rho[tid] = c.P->rho[tid];
    }

    static PC_HD PR pair_of(R v) { return stiff_pair(v); }

    static PC_HD C stiff_fma(PR c, C e, C acc) { return stiff_fma_pair(c, e, acc); }

    // Fluxes of the own column at plane kf -> shared memory.
    static PC_HD void flux(const Ctx& c, Shared& sh, const Regs& r, int kf) {
        if (!r.fvalid) return;
        const StencilParams<R>& P = *c.P;
        int delta, dl[4];
        if (FULL) {
            delta = 0;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int s2 = (l < 2) ? 1 : -1;
                dl[l] = -1 - XW * s2;
            }
        } else {
            const int i0 = (kf + c.p13) & 1, j0 = (kf + c.p12 + c.p13) & 1;
            delta = i0 + XW * j0;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int s2 = (l < 2) ? 1 : -1;
                dl[l] = -1 - XW * ((s2 + 1) >> 1);
            }
        }
        const C* xm = slot_ptr(sh, kf - 1, c.k0);
        const C* x0 = slot_ptr(sh, kf, c.k0);
        const C* xp = slot_ptr(sh, kf + 1, c.k0);
        C g[4][3];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int s3 = (l & 1) ? -1 : 1;
            const int nb = r.fown + delta + dl[l];
            PC_IDX(nb, XR);
            const C* xs = (s3 > 0) ? xm : xp;  // backward step moves k by -s3
#pragma unroll
            for (int a = 0; a < 3; ++a) g[l][a] = csub(xs[a * XR + nb], x0[a * XR + r.fown]);
        }
        C H[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C u = cadd(g[0][a], g[1][a]), v = cadd(g[2][a], g[3][a]);
            C w = csub(g[0][a], g[1][a]), z = csub(g[2][a], g[3][a]);
            H[0][a] = cadd(u, v);
            H[1][a] = csub(u, v);
            H[2][a] = cadd(w, z);
        }
        C G[3][3];
        if (CUBIC) {
#pragma unroll
            for (int mm = 0; mm < 3; ++mm)
#pragma unroll
                for (int a = 0; a < 3; ++a) G[mm][a] = H[mm][a];
        } else {
#pragma unroll
            for (int mm = 0; mm < 3; ++mm)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    C acc = cscale(P.Mmix[0 * 3 + mm], H[0][a]);
                    acc = cfma(P.Mmix[1 * 3 + mm], H[1][a], acc);
                    G[mm][a] = cfma(P.Mmix[2 * 3 + mm], H[2][a], acc);
                }
        }
        C e[6];
        e[0] = G[0][0];
        e[1] = G[1][1];
        e[2] = G[2][2];
        e[3] = cadd(G[2][1], G[1][2]);
        e[4] = cadd(G[2][0], G[0][2]);
        e[5] = cadd(G[1][0], G[0][1]);
        C t[6];
        if (MATK == 0) {
            const PR* Cq = sh.Cp[r.fm_cur != (R)0 ? 1 : 0];
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                C acc = czero((R)0);
#pragma unroll
                for (int q = 0; q < 6; ++q) acc = stiff_fma(Cq[p * 6 + q], e[q], acc);
                t[p] = acc;
            }
        } else {
            const R th = r.fm_cur;
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                C acc = czero((R)0);
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const R c0 = c.P->C[0][p * 6 + q], c1 = c.P->C[1][p * 6 + q];
                    acc = cfma(c0 + th * (c1 - c0), e[q], acc);
                }
                t[p] = acc;
            }
        }
        C S[3][3];
        S[0][0] = t[0]; S[0][1] = t[5]; S[0][2] = t[4];
        S[1][0] = t[5]; S[1][1] = t[1]; S[1][2] = t[3];
        S[2][0] = t[4]; S[2][1] = t[3]; S[2][2] = t[2];
        C Pm[3][3];
        if (CUBIC) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int a = 0; a < 3; ++a) Pm[s][a] = S[a][s];
        } else {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    C acc = cscale(P.Mmix[s * 3 + 0], S[a][0]);
                    acc = cfma(P.Mmix[s * 3 + 1], S[a][1], acc);
                    Pm[s][a] = cfma(P.Mmix[s * 3 + 2], S[a][2], acc);
                }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C u = cadd(Pm[0][a], Pm[1][a]), v = csub(Pm[0][a], Pm[1][a]);
            sh.fs[0][a][r.fcol] = cadd(u, Pm[2][a]);
            sh.fs[1][a][r.fcol] = csub(u, Pm[2][a]);
            sh.fs[2][a][r.fcol] = cadd(v, Pm[2][a]);
            sh.fs[3][a][r.fcol] = csub(v, Pm[2][a]);
            sh.fs[4][a][r.fcol] = cscale((R)4, Pm[0][a]);
        }
    }

    // Finish y(kf-1), local term of y(kf), start y(kf+1).
    static PC_HD void gather(const Ctx& c, Shared& sh, Regs& r, int kf) {
        if (r.yvalid) {
            int delta = 0, dl[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int s2 = (l < 2) ? 1 : -1;
                dl[l] = FULL ? (1 + FW * s2) : (FW * ((s2 - 1) >> 1));
            }
            if (!FULL) {
                const int par = (kf - 1) & 1;
                delta = ((par + c.p13) & 1) + FW * ((par + c.p12 + c.p13) & 1);
            }
            if (kf - 1 >= c.k0) {
                const int nb0 = r.fbase + delta + dl[0], nb2 = r.fbase + delta + dl[2];
                PC_IDX(nb0, FR);
                PC_IDX(nb2, FR);
                const C* xm = slot_ptr(sh, kf - 1, c.k0);
                R rho;
                if (MATK == 0) rho = sh.rho[r.ym_cur != (R)0 ? 1 : 0];
                else rho = sh.rho[0] + r.ym_cur * (sh.rho[1] - sh.rho[0]);
                const R sr = c.shift * rho;
                const int64_t ob = (int64_t)(kf - 1) * c.plane + r.yoff;
                PC_IDX(ob, c.vstr);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    C v = cadd(r.acc_prev[a], cadd(sh.fs[0][a][nb0], sh.fs[2][a][nb2]));
                    const C xv = xm[a * XR + r.xown];
                    v = cfma(-sr, xv, v);
                    c.y[a * c.vstr + ob] = v;
                    r.dot = cdotre(xv, v, r.dot);
                }
            }
            if (kf >= c.k0 && kf < c.k0 + c.tz) {
#pragma unroll
                for (int a = 0; a < 3; ++a) r.acc_cur[a] = csub(r.acc_cur[a], sh.fs[4][a][r.fbase]);
            }
            if (kf + 1 >= c.k0 && kf + 1 < c.k0 + c.tz) {
                const int nb1 = r.fbase + delta + dl[1], nb3 = r.fbase + delta + dl[3];
                PC_IDX(nb1, FR);
                PC_IDX(nb3, FR);
#pragma unroll
                for (int a = 0; a < 3; ++a) r.acc_next[a] = cadd(sh.fs[1][a][nb1], sh.fs[3][a][nb3]);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                r.acc_prev[a] = r.acc_cur[a];
                r.acc_cur[a] = r.acc_next[a];
                r.acc_next[a] = czero((R)0);
            }
        }
    }

    static PC_HD void load_mats(const Ctx& c, Regs& r, int kf) {
        // flux material of plane kf + 1, output material of plane kf (used one step later)
        int wk;
        const int k = wrapc(kf + 1, c.P->Z, wk);
        r.fm_nxt = r.fvalid ? read_mat(c.mat, (int64_t)k * c.plane + r.foff) : (R)0;
        r.ym_nxt = (r.yvalid && kf >= c.k0 && kf < c.k0 + c.tz) ? read_mat(c.mat, (int64_t)kf * c.plane + r.yoff)
                                                                : (R)0;
    }

    static PC_HD void rotate_mats(Regs& r) {
        r.fm_cur = r.fm_nxt;
        r.ym_cur = r.ym_nxt;
    }

    // Host model of one box copy (TMA semantics: cells outside the tensor read as zero).
    static void host_copy_box(const Ctx& c, Shared& sh, int kp) {
        const StencilParams<R>& P = *c.P;
        int wk;
        const int k = wrapc(kp, P.Z, wk);
        C* s = slot_ptr(sh, kp, c.k0);
        for (int comp = 0; comp < 3; ++comp)
            for (int rb = 0; rb < XH; ++rb)
                for (int ra = 0; ra < XW; ++ra) {
                    const int a = c.a0 - 2 + ra, b = c.b0 - 2 + rb;
                    C v = czero((R)0);
                    if (a >= 0 && a < P.X && b >= 0 && b < P.Y)
                        v = c.x[comp * c.vstr + (int64_t)k * c.plane + (int64_t)b * P.X + a];
                    s[comp * XR + rb * XW + ra] = v;
                }
    }
};

}  // namespace pc
