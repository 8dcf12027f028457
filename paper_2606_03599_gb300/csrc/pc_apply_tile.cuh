// Fused stencil apply y = (A - shift M) x on one tile of a parity block (or of
// the full grid), written as per-thread phase functions so that the CUDA kernel
// and a host emulator run the same index arithmetic.
//
// Operator (Sec. 3, Eqs. Sd_def, Dd_def, Dtilde_recon_main, Dhat_def_main,
// Dcal_cartesian_transform_main, B_discrete_main, discrete_GEP_main).  With the
// backward differences g_l = x~(x - d_l) - x(x) along the four body diagonals
// d_l = (1, s2, s3) and the reconstruction signs c_s = (1,1,1,1), (1,1,-1,-1),
// (1,-1,1,-1):
//
//   H_{s a}  = sum_l c_{s l} g_{l a}                     (= 4 h_s Dt_s^H x_a)
//   G'_{m a} = sum_s Mmix_{s m} H_{s a},  Mmix_{s m} = (A^-1)_{s m} / (4 h_s)
//              (Dcal_m^H x_a = i G'_{m a})
//   e'       = Voigt strain from G' (rows of B_h^H), tau' = C_node e'
//   S_{a m}  = stress tensor of tau' (S_11 = t1, S_12 = t6, S_13 = t5, ...)
//   P_{s a}  = sum_m Mmix_{s m} S_{a m},  F_{l a} = sum_s c_{s l} P_{s a}
//   y_a(x)   = sum_l F~_{l a}(x + d_l) - sum_l F_{l a}(x)   (the factors i and
//              -i of Dhat^H and Dhat cancel), then y -= shift rho_node x.
//
// For a cubic lattice Mmix = (N/4) I and the factor (N/4)^2 is folded into C.
//
// Layouts.  A parity block is stored on its quarter grid (a, b, k) = (i', j'', k)
// with extents (X, Y, Z) = (N/2, N/2, N), node i = 2a + i0(k), j = 2b + j0(k),
// i0(k) = (k + p13) mod 2, j0(k) = (k + p12 + p13) mod 2 (Sec. 4, Eq.
// V_sigma_main).  A step (e1, e2, e3) with odd entries moves (a, b, k) by
// (i0(k) + (e1-1)/2, j0(k) + (e2-1)/2, e3).  The full grid uses (a, b, k) =
// (i, j, k) and moves by (e1, e2, e3) directly.  Leaving [0,X) x [0,Y) x [0,Z)
// multiplies by exp(+-i phi_l) of that axis (Eqs. K_def, H_def).
//
// Tiling.  A CTA owns an a-b tile of TX x TY columns and marches through a
// chunk of tz planes in k.  Shared memory holds a ring of four x planes over
// the tile plus a halo (TX+2) x (TY+4), and one plane of fluxes F.  The flux
// columns of plane kf are those of the tile's own nodes (for the local term)
// and those the outputs of planes kf +- 1 read, which sit at a fixed offset
// (i0, j0 - 1 + {0, 1}) of the same parity: (TX + i0) x (TY + 1) columns for a
// parity block, (TX+1) x (TY+2) for the full grid.  Step kf computes F(kf), then finishes y(kf-1)
// (the s3 = +1 neighbours are in plane kf), adds the local term to y(kf) and
// starts y(kf+1) with its s3 = -1 neighbours (also in plane kf).  x planes are
// prefetched one step ahead through registers; Bloch phases of wrapped halo
// cells are applied on the way into shared memory.
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "pc_complex.cuh"
#include "pc_internal.h"

#if !defined(__CUDA_ARCH__) && defined(PC_EMU_CHECK)
#include <cstdio>
#include <cstdlib>
#define PC_IDX(i, n)                                                                   \
    do {                                                                               \
        if ((long long)(i) < 0 || (long long)(i) >= (long long)(n)) {                  \
            std::fprintf(stderr, "index %lld out of [0,%lld) at %s:%d\n", (long long)(i), \
                         (long long)(n), __FILE__, __LINE__);                          \
            std::abort();                                                              \
        }                                                                              \
    } while (0)
#else
#define PC_IDX(i, n) \
    do {             \
    } while (0)
#endif

namespace pc {

template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
struct ApplyTile {
    using C = typename CT<R>::T;
    static constexpr int NT = TX * TY;
    static constexpr int XW = TX + 2, XH = TY + 4, XR = XW * XH;  // x region
    static constexpr int FW = TX + 1, FH = TY + 2, FR = FW * FH;  // flux region (largest; stride FW)
    static constexpr int NXC = (3 * XR + NT - 1) / NT;            // x cells per thread
    static constexpr int NFC = (FR + NT - 1) / NT;                // flux columns per thread
    static constexpr int NSLOT = 4;

    // material value of a node: phase id (MATK 0, kept as an integer so that FP64 kernels spend no
    // FP64 instruction on it) or inclusion fraction (MATK 1)
    using MT = typename std::conditional<MATK == 0, int, R>::type;

    struct Shared {
        C xs[NSLOT][3][XR];
        C fs[5][3][FR];  // F_l for l = 0..3, slot 4 = P_0 (sum_l F_l = 4 P_0)
        R Ct[2][36];
        R rho[2];
        R srho[2];  // shift * rho per phase
    };

    struct Ctx {
        const StencilParams<R>* P;
        const C* x;
        C* y;
        const void* mat;
        R shift;
        bool dot;  // accumulate Re<x, y> for the partial sums
        int a0, b0, k0, tz;
        int p12, p13;
        int64_t plane;  // X * Y
        int64_t vstr;   // X * Y * Z (component stride)
    };

    struct Regs {
        C xpre[NXC];
        int xoff[NXC];   // wrapped in-plane offset, -1 = no cell
        int xcomp[NXC];  // component
        int xwa[NXC], xwb[NXC];
        int foff[2][NFC];  // wrapped in-plane offset of flux column per plane parity, -1 = none
        MT fmat_cur[NFC], fmat_nxt[NFC];
        int ty, tx;
        bool yvalid;
        int yoff;  // in-plane offset of the output column
        MT ymat_cur, ymat_nxt;
        C acc_prev[3], acc_cur[3], acc_next[3];
        R dot;
    };

    // Reduce v into [0, n); w counts the periods crossed (tiles may exceed tiny grids).
    static PC_HD int wrapc(int v, int n, int& w) {
        w = 0;
        while (v < 0) { v += n; --w; }
        while (v >= n) { v -= n; ++w; }
        return v;
    }

    static PC_HD MT read_mat(const void* mat, int64_t idx) {
        PC_IDX(idx, 1LL << 40);
        if (MATK == 0) return (MT)(static_cast<const uint8_t*>(mat)[idx]);
        return (MT)(static_cast<const float*>(mat)[idx]);
    }

    // Flux region of plane kf: columns (a0 + fa, b0 + ob + fb), fa < fw, fb < fh; the outputs of
    // planes kf +- 1 read their neighbours at a-offset oa.
    static PC_HD void flux_region(const Ctx& c, int kf, int& oa, int& ob, int& fw, int& fh) {
        if (FULL) {
            oa = 1;
            ob = -1;
            fw = TX + 1;
            fh = TY + 2;
        } else {
            oa = (kf + 1 + c.p13) & 1;               // i0 of planes kf +- 1
            ob = ((kf + 1 + c.p12 + c.p13) & 1) - 1;  // j0 of planes kf +- 1, minus 1
            fw = TX + oa;
            fh = TY + 1;
        }
    }

    // exp(i (wa phi1 + wb phi2 + wk phi3)) for integer period counts
    static PC_HD C wrap_phase(const StencilParams<R>& P, int wa, int wb, int wk) {
        C ph = cmk((R)1, (R)0);
        const int w[3] = {wa, wb, wk};
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const C e = cmk(P.ph[l][0], w[l] < 0 ? -P.ph[l][1] : P.ph[l][1]);
            for (int q = 0; q < (w[l] < 0 ? -w[l] : w[l]); ++q) ph = cmul(ph, e);
        }
        return ph;
    }

    static PC_HD void init(const Ctx& c, int tid, Regs& r) {
        const StencilParams<R>& P = *c.P;
#pragma unroll
        for (int i = 0; i < NXC; ++i) {
            int cell = tid + i * NT;
            r.xoff[i] = -1;
            r.xcomp[i] = 0;
            r.xwa[i] = r.xwb[i] = 0;
            if (cell < 3 * XR) {
                int comp = cell / XR, col = cell % XR;
                int ra = col % XW, rb = col / XW;
                int wa, wb;
                int a = wrapc(c.a0 - 1 + ra, P.X, wa);
                int b = wrapc(c.b0 - 2 + rb, P.Y, wb);
                r.xoff[i] = a + P.X * b;
                r.xcomp[i] = comp;
                r.xwa[i] = wa;
                r.xwb[i] = wb;
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            int oa, ob, fw, fh;
            flux_region(c, q, oa, ob, fw, fh);  // the region depends on the plane's parity only
#pragma unroll
            for (int i = 0; i < NFC; ++i) {
                int col = tid + i * NT;
                r.foff[q][i] = -1;
                if (col < fw * fh) {
                    int fa = col % fw, fb = col / fw, wa, wb;
                    int a = wrapc(c.a0 + fa, P.X, wa);
                    int b = wrapc(c.b0 + ob + fb, P.Y, wb);
                    r.foff[q][i] = a + P.X * b;
                }
            }
        }
        r.tx = tid % TX;
        r.ty = tid / TX;
        int ya = c.a0 + r.tx, yb = c.b0 + r.ty;
        r.yvalid = (ya < P.X) && (yb < P.Y);
        r.yoff = r.yvalid ? ya + P.X * yb : 0;
        for (int a = 0; a < 3; ++a) r.acc_prev[a] = r.acc_cur[a] = r.acc_next[a] = czero((R)0);
        r.dot = (R)0;
        r.ymat_cur = r.ymat_nxt = (MT)0;
    }

    // Read plane kp (any integer, Bloch-extended) of the x region into registers.
    static PC_HD void load_x(const Ctx& c, Regs& r, int kp) {
        const StencilParams<R>& P = *c.P;
        int wk;
        int k = wrapc(kp, P.Z, wk);
#pragma unroll
        for (int i = 0; i < NXC; ++i) {
            if (r.xoff[i] < 0) continue;
            const int64_t gi = r.xcomp[i] * c.vstr + (int64_t)k * c.plane + r.xoff[i];
            PC_IDX(gi, 3 * c.vstr);
            C v = c.x[gi];
            if (r.xwa[i] | r.xwb[i] | wk) v = cmul(v, wrap_phase(P, r.xwa[i], r.xwb[i], wk));
            r.xpre[i] = v;
        }
    }

    static PC_HD void store_x(Shared& sh, const Regs& r, int tid, int kp) {
        int slot = kp & (NSLOT - 1);
#pragma unroll
        for (int i = 0; i < NXC; ++i) {
            if (r.xoff[i] < 0) continue;
            int cell = tid + i * NT;
            PC_IDX(cell, 3 * XR);
            sh.xs[slot][cell / XR][cell % XR] = r.xpre[i];
        }
    }

    static PC_HD void load_fmat(const Ctx& c, Regs& r, int kp, MT* dst) {
        int wk;
        int k = wrapc(kp, c.P->Z, wk);
        const int q = kp & 1;
#pragma unroll
        for (int i = 0; i < NFC; ++i) {
            const int off = q ? r.foff[1][i] : r.foff[0][i];  // selected, not indexed: stays in registers
            dst[i] = (off >= 0) ? read_mat(c.mat, (int64_t)k * c.plane + off) : (MT)0;
        }
    }

    static PC_HD MT load_ymat(const Ctx& c, const Regs& r, int kp) {
        if (!r.yvalid || kp < c.k0 || kp >= c.k0 + c.tz) return (MT)0;
        return read_mat(c.mat, (int64_t)kp * c.plane + r.yoff);
    }

    // Fluxes at one column of plane kf.
    static PC_HD void flux_column(const Ctx& c, const Shared& sh, int fa, int fb, int ob, int kf, MT m,
                                  C* fout /*15*/) {
        const StencilParams<R>& P = *c.P;
        const int xb = fb + ob + 2;  // x-region row of the flux node
        const int own = (fa + 1) + XW * xb;
        int i0 = 0, j0 = 0;
        if (!FULL) {
            i0 = (kf + c.p13) & 1;
            j0 = (kf + c.p12 + c.p13) & 1;
        }
        const int sc = kf & (NSLOT - 1), sm = (kf - 1) & (NSLOT - 1), sp = (kf + 1) & (NSLOT - 1);
        C g[4][3];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int s2 = (l < 2) ? 1 : -1, s3 = (l & 1) ? -1 : 1;
            int da, db;
            if (FULL) { da = -1; db = -s2; }
            else { da = i0 - 1; db = j0 - ((s2 + 1) >> 1); }
            const int nb = (fa + 1 + da) + XW * (xb + db);
            PC_IDX(fa + 1 + da, XW);
            PC_IDX(xb + db, XH);
            const int slot = (s3 > 0) ? sm : sp;  // backward step moves k by -s3
#pragma unroll
            for (int a = 0; a < 3; ++a) g[l][a] = csub(sh.xs[slot][a][nb], sh.xs[sc][a][own]);
        }
        // Hadamard reconstruction H_s = sum_l c_{s l} g_l
        C H[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C u = cadd(g[0][a], g[1][a]), v = cadd(g[2][a], g[3][a]);
            C w = csub(g[0][a], g[1][a]), z = csub(g[2][a], g[3][a]);
            H[0][a] = cadd(u, v);
            H[1][a] = csub(u, v);
            H[2][a] = cadd(w, z);
        }
        C G[3][3];  // G[m][a]
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
        // Voigt strain [11,22,33,23,13,12] with engineering shear
        C e[6];
        e[0] = G[0][0];
        e[1] = G[1][1];
        e[2] = G[2][2];
        e[3] = cadd(G[2][1], G[1][2]);
        e[4] = cadd(G[2][0], G[0][2]);
        e[5] = cadd(G[1][0], G[0][1]);
        // tau = C_node e
        C t[6];
        if (MATK == 0) {
            const int ph = m != 0 ? 1 : 0;
            const R* Cp = sh.Ct[ph];
            if (warp_all(P.ortho[ph] != 0)) {  // every node of the warp: normal block and shear diagonal only
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    C acc = cscale(Cp[p * 6 + 0], e[0]);
                    acc = cfma(Cp[p * 6 + 1], e[1], acc);
                    t[p] = cfma(Cp[p * 6 + 2], e[2], acc);
                }
#pragma unroll
                for (int p = 3; p < 6; ++p) t[p] = cscale(Cp[p * 6 + p], e[p]);
            } else {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    C acc = cscale(Cp[p * 6 + 0], e[0]);
#pragma unroll
                    for (int q = 1; q < 6; ++q) acc = cfma(Cp[p * 6 + q], e[q], acc);
                    t[p] = acc;
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                R c0 = sh.Ct[0][p * 6 + 0];
                C acc = cscale(c0 + m * (sh.Ct[1][p * 6 + 0] - c0), e[0]);
#pragma unroll
                for (int q = 1; q < 6; ++q) {
                    R cq = sh.Ct[0][p * 6 + q];
                    acc = cfma(cq + m * (sh.Ct[1][p * 6 + q] - cq), e[q], acc);
                }
                t[p] = acc;
            }
        }
        // stress tensor S[a][m]
        C S[3][3];
        S[0][0] = t[0]; S[0][1] = t[5]; S[0][2] = t[4];
        S[1][0] = t[5]; S[1][1] = t[1]; S[1][2] = t[3];
        S[2][0] = t[4]; S[2][1] = t[3]; S[2][2] = t[2];
        C Pm[3][3];  // P[s][a]
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
        // F_l = sum_s c_{s l} P_s, and P_0 (the local sum is 4 P_0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C u = cadd(Pm[0][a], Pm[1][a]), v = csub(Pm[0][a], Pm[1][a]);
            fout[0 * 3 + a] = cadd(u, Pm[2][a]);
            fout[1 * 3 + a] = csub(u, Pm[2][a]);
            fout[2 * 3 + a] = cadd(v, Pm[2][a]);
            fout[3 * 3 + a] = csub(v, Pm[2][a]);
            fout[4 * 3 + a] = Pm[0][a];
        }
    }

    // Phase A of step kf: fluxes of plane kf; stage x plane kf+2; prefetch kf+3 and materials.
    static PC_HD void phaseA(const Ctx& c, Shared& sh, Regs& r, int tid, int kf) {
        int oa, ob, fw, fh;
        flux_region(c, kf, oa, ob, fw, fh);
#pragma unroll
        for (int i = 0; i < NFC; ++i) {
            int col = tid + i * NT;
            if (col >= fw * fh) continue;
            const int fa = col % fw, fb = col / fw, fidx = fa + FW * fb;
            PC_IDX(fidx, FR);
            C f[15];
            flux_column(c, sh, fa, fb, ob, kf, r.fmat_cur[i], f);
#pragma unroll
            for (int l = 0; l < 5; ++l)
#pragma unroll
                for (int a = 0; a < 3; ++a) sh.fs[l][a][fidx] = f[l * 3 + a];
        }
        load_fmat(c, r, kf + 1, r.fmat_nxt);
        r.ymat_nxt = load_ymat(c, r, kf);
        const int klast = c.k0 + c.tz + 1;
        if (kf + 2 <= klast) store_x(sh, r, tid, kf + 2);
        if (kf + 3 <= klast) load_x(c, r, kf + 3);
    }

    // Phase B of step kf: finish y(kf-1), local term of y(kf), start y(kf+1).
    static PC_HD void phaseB(const Ctx& c, Shared& sh, Regs& r, int kf) {
        if (r.yvalid) {
            int da[4], db[4];
            const int par = (kf - 1) & 1;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int s2 = (l < 2) ? 1 : -1;
                if (FULL) { da[l] = 1; db[l] = s2; }
                else {
                    const int i0 = (par + c.p13) & 1, j0 = (par + c.p12 + c.p13) & 1;
                    da[l] = i0;
                    db[l] = j0 + ((s2 - 1) >> 1);
                }
            }
            int oa, ob, fw, fh;
            flux_region(c, kf, oa, ob, fw, fh);
            const int fbase = r.tx + FW * (r.ty - ob);  // own column in the flux region of plane kf
#if !defined(__CUDA_ARCH__) && defined(PC_EMU_CHECK)
            PC_IDX(r.tx, fw);
            PC_IDX(r.ty - ob, fh);
            for (int l = 0; l < 4; ++l) {
                PC_IDX(r.tx + da[l], fw);
                PC_IDX(r.ty - ob + db[l], fh);
            }
#endif
            if (kf - 1 >= c.k0) {
                const int nb0 = fbase + da[0] + FW * db[0];
                const int nb2 = fbase + da[2] + FW * db[2];
                const int xo = (r.tx + 1) + XW * (r.ty + 2);
                const int sl = (kf - 1) & (NSLOT - 1);
                R sr;
                if (MATK == 0) sr = sh.srho[r.ymat_cur != 0 ? 1 : 0];
                else sr = c.shift * (sh.rho[0] + r.ymat_cur * (sh.rho[1] - sh.rho[0]));
                const int64_t obase = (int64_t)(kf - 1) * c.plane + r.yoff;
                PC_IDX(obase, c.vstr);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    C v = cadd(r.acc_prev[a], cadd(sh.fs[0][a][nb0], sh.fs[2][a][nb2]));
                    C xv = sh.xs[sl][a][xo];
                    v = cfma(-sr, xv, v);
                    c.y[a * c.vstr + obase] = v;
                    if (c.dot) r.dot = cdotre(xv, v, r.dot);
                }
            }
            if (kf >= c.k0 && kf < c.k0 + c.tz) {
#pragma unroll
                for (int a = 0; a < 3; ++a) r.acc_cur[a] = cfma((R)(-4), sh.fs[4][a][fbase], r.acc_cur[a]);
            }
            if (kf + 1 >= c.k0 && kf + 1 < c.k0 + c.tz) {
                const int nb1 = fbase + da[1] + FW * db[1];
                const int nb3 = fbase + da[3] + FW * db[3];
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
#pragma unroll
        for (int i = 0; i < NFC; ++i) r.fmat_cur[i] = r.fmat_nxt[i];
        r.ymat_cur = r.ymat_nxt;
    }

    // Prologue: planes k0-2, k0-1, k0 into shared memory, k0+1 into registers.
    static PC_HD void prologue_load(const Ctx& c, Shared& sh, Regs& r, int tid) {
        for (int kp = c.k0 - 2; kp <= c.k0; ++kp) {
            load_x(c, r, kp);
            store_x(sh, r, tid, kp);
        }
        load_x(c, r, c.k0 + 1);
        load_fmat(c, r, c.k0 - 1, r.fmat_cur);
        r.ymat_cur = (MT)0;
    }

    static PC_HD void load_tables(const Ctx& c, Shared& sh, int tid) {
        for (int i = tid; i < 72; i += NT) sh.Ct[i / 36][i % 36] = c.P->C[i / 36][i % 36];
        if (tid < 2) {
            sh.rho[tid] = c.P->rho[tid];
            sh.srho[tid] = c.shift * c.P->rho[tid];
        }
    }
};

}  // namespace pc
