// Two-pass stencil apply for complex128 (FP64), written as per-node functions so that
// the CUDA kernels and a host emulator share the index arithmetic.
//
// Operator and layouts as in pc_apply_tile.cuh (Sec. 3: y = (A - shift M) x with the
// fluxes F_l of the adjoint differences).  On GB300 the FP64 pipe (2 lanes per cycle per
// SM) bounds a complex128 apply, not memory; the fused tile kernels compute the fluxes of
// every halo column again in each neighbouring tile and k-chunk, and leave lanes idle where
// a flux region is not a multiple of the warp width.  Here each node's fluxes are computed
// exactly once, by one lane, and go through memory (L2 at the solver's grid sizes):
//
//   1. fill:   the ghost layer of x (one cell deep on every side the flux pass reads; ghost =
//              wrapped node times exp(i w.phi)) -> x_g, a compact array of ghost cells;
//   2. flux:   per node, g_l = x(node - d_l) - x(node), the neighbour read from x itself when it
//              lies inside the grid and from x_g when not (an address choice, no arithmetic:
//              the FP64 pipe that bounds this pass does no phase work), the strain, the stress
//              and the fluxes F_l and P_0 (sum_l F_l = 4 P_0) -> f_e;
//   3. fill:   ghost cells of f_e (F_0..F_3) from their wrapped nodes, times exp(i w.phi);
//   4. gather: y(node) = sum_l F_l(node + d_l) - 4 P_0(node) - shift rho x(node), with
//              optional partial sums of Re<x, y>.
//
// Extended cell (a, b, k), a in [-1, X], b in [-1, Y], k in [-1, Z], has index
// (a + 1) + Xe ((b + 1) + Ye (k + 1)) with Xe = X + 2, Ye = Y + 2; each of the 15 values of f_e
// (F_l of component c at l * 3 + c, P_0 of c at 12 + c) is a separate array of Xe Ye Ze cells.
// Each of the 3 components of x_g is an array of the extended grid's ghost cells, in the order
// of ghost_cell.
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "pc_apply_tile.cuh"  // PC_IDX (index checks in the host emulator)
#include "pc_complex.cuh"
#include "pc_internal.h"

namespace pc {

struct SplitGeom {
    int X, Y, Z;       // interior extents of the vector layout
    int Xe, Ye, Ze;    // X + 2, Y + 2, Z + 2
    int64_t ne;        // cells per extended array
    int64_t m;         // interior nodes X Y Z
    int64_t ghosts;    // ghost cells per extended array
};

inline SplitGeom make_split_geom(int X, int Y, int Z) {
    SplitGeom G;
    G.X = X;
    G.Y = Y;
    G.Z = Z;
    G.Xe = X + 2;
    G.Ye = Y + 2;
    G.Ze = Z + 2;
    G.ne = (int64_t)G.Xe * G.Ye * G.Ze;
    G.m = (int64_t)X * Y * Z;
    G.ghosts = G.ne - G.m;
    return G;
}

// Complex values of scratch per item: x_g (3 arrays of ghost cells) and f_e (15 extended arrays).
inline int64_t split_item_elems(const SplitGeom& G) { return 3 * G.ghosts + 15 * G.ne; }

// Upper-triangular position (row order, p <= r) of Voigt entry (p, r) among the 21 independent
// entries of a symmetric 6x6 stiffness.
PC_HD constexpr int voigt_upper(int p, int r) {
    return p <= r ? p * 6 - p * (p - 1) / 2 + (r - p) : r * 6 - r * (r - 1) / 2 + (p - r);
}

// MATK: 0 = phase ids (uint8), 1 = inclusion fraction theta (float), 2 = nodewise material (FP64,
// component-major [22][m]: the 21 upper-triangular stiffness entries scaled as the kernel's tables
// (hat units, (N/4)^2 folded in on a cubic lattice), then the density in hat units).
template <typename R, bool FULL, bool CUBIC, int MATK>
struct SplitApply {
    using C = typename CT<R>::T;
    using MT = typename std::conditional<MATK == 0, int, R>::type;

    static PC_HD int64_t eidx(const SplitGeom& G, int a, int b, int k) {
        return (a + 1) + (int64_t)G.Xe * ((b + 1) + (int64_t)G.Ye * (k + 1));
    }

    // exp(i (wa phi_1 + wb phi_2 + wk phi_3)), w in {-1, 0, 1}; kph[l] = (cos phi_l, sin phi_l) of
    // the item's Bloch vector
    static PC_HD C phase(const R (*kph)[2], int wa, int wb, int wk) {
        C ph = cmk((R)1, (R)0);
        const int w[3] = {wa, wb, wk};
#pragma unroll
        for (int l = 0; l < 3; ++l)
            if (w[l] != 0) ph = cmul(ph, cmk(kph[l][0], w[l] < 0 ? -kph[l][1] : kph[l][1]));
        return ph;
    }

    static PC_HD int wrap1(int v, int n, int& w) {
        w = v < 0 ? -1 : (v >= n ? 1 : 0);
        return v - w * n;
    }

    // Ghost cell number gi (0 <= gi < G.ghosts) -> extended coordinates.  Order: the planes
    // k = -1 and k = Z (Xe Ye cells each), then for k in [0, Z) the rows b = -1 and b = Y
    // (Xe cells each), then for k in [0, Z), b in [0, Y) the columns a = -1 and a = X.
    static PC_HD void ghost_cell(const SplitGeom& G, int64_t gi, int& a, int& b, int& k) {
        uint32_t g = (uint32_t)gi;  // 32-bit arithmetic: ghost counts are far below 2^32
        const uint32_t pl = (uint32_t)G.Xe * (uint32_t)G.Ye, xe = (uint32_t)G.Xe;
        if (g < 2 * pl) {
            k = g < pl ? -1 : G.Z;
            const uint32_t r = g < pl ? g : g - pl, rq = r / xe;
            a = (int)(r - rq * xe) - 1;
            b = (int)rq - 1;
            return;
        }
        g -= 2 * pl;
        const uint32_t rows = 2u * xe * (uint32_t)G.Z;
        if (g < rows) {
            const uint32_t row = g / xe;  // 2 rows per plane
            k = (int)(row >> 1);
            b = (row & 1) ? G.Y : -1;
            a = (int)(g - row * xe) - 1;
            return;
        }
        g -= rows;
        const uint32_t col = g >> 1, cq = col / (uint32_t)G.Y;  // (b, k) pairs
        a = (g & 1) ? G.X : -1;
        b = (int)(col - cq * (uint32_t)G.Y);
        k = (int)cq;
    }

    // Inverse of ghost_cell: the number of the ghost cell (a, b, k) (one coordinate outside the
    // interior range at least).
    static PC_HD int64_t ghost_index(const SplitGeom& G, int a, int b, int k) {
        const int64_t pl = (int64_t)G.Xe * G.Ye;
        if (k < 0 || k >= G.Z) return (k < 0 ? 0 : pl) + (a + 1) + (int64_t)G.Xe * (b + 1);
        if (b < 0 || b >= G.Y) return 2 * pl + (int64_t)(2 * k + (b < 0 ? 0 : 1)) * G.Xe + (a + 1);
        return 2 * pl + 2 * (int64_t)G.Xe * G.Z + 2 * (b + (int64_t)G.Y * k) + (a < 0 ? 0 : 1);
    }

    // Pass 1, ghost cell gi (all three components): the wrapped node times its Bloch phase.
    static PC_HD void fill_x_ghost(const R (*kph)[2], const SplitGeom& G, const C* x, C* xg, int64_t gi) {
        int a, b, k, wa, wb, wk;
        ghost_cell(G, gi, a, b, k);
        if (a >= G.X) return;  // the flux pass reads a in [-1, X) only
        const int aw = wrap1(a, G.X, wa), bw = wrap1(b, G.Y, wb), kw = wrap1(k, G.Z, wk);
        const int64_t src = aw + (int64_t)G.X * (bw + (int64_t)G.Y * kw);
        PC_IDX(src, G.m);
        PC_IDX(gi, G.ghosts);
        const C ph = phase(kph, wa, wb, wk);
#pragma unroll
        for (int c = 0; c < 3; ++c) xg[c * G.ghosts + gi] = cmul(x[c * G.m + src], ph);
    }

    // Pass 3, ghost cell gi of the flux arrays F_0..F_3 (12 arrays).
    static PC_HD void fill_f_ghost(const R (*kph)[2], const SplitGeom& G, C* fe, int64_t gi) {
        int a, b, k, wa, wb, wk;
        ghost_cell(G, gi, a, b, k);
        if (a < 0) return;  // the gather reads a in [0, X] only
        const int aw = wrap1(a, G.X, wa), bw = wrap1(b, G.Y, wb), kw = wrap1(k, G.Z, wk);
        const int64_t src = eidx(G, aw, bw, kw), dst = eidx(G, a, b, k);
        PC_IDX(src, G.ne);
        const C ph = phase(kph, wa, wb, wk);
#pragma unroll
        for (int f = 0; f < 12; ++f) fe[f * G.ne + dst] = cmul(fe[f * G.ne + src], ph);
    }

    static PC_HD MT read_mat(const void* mat, int64_t t) {
        if (MATK == 0) return (MT)(static_cast<const uint8_t*>(mat)[t]);
        if (MATK == 2) return (MT)0;
        return (MT)(static_cast<const float*>(mat)[t]);
    }

    // Pass 2, interior node t: fluxes F_l (l = 0..3) and P_0 of the three components.
    // Ct: the two stiffness tables (shared memory on the device).
    static PC_HD void flux_node(const StencilParams<R>& P, const R (*Ct)[36], const SplitGeom& G, int p12, int p13,
                                const C* x, const C* xg, const void* mat, C* fe, int64_t t, bool uniform_ortho_ok) {
        int a, b, k;
        split3(t, G.X, G.Y, a, b, k);
        const int64_t own = eidx(G, a, b, k);
        int da = -1, j0 = 0;
        if (!FULL) {
            da = ((k + p13) & 1) - 1;
            j0 = (k + p12 + p13) & 1;
        }
        // H_s = sum_l c_{s l} g_l with g_l = n_l - x(node): the own value cancels from H_1 and H_2
        // (their sign rows sum to zero) and enters H_0 as -4 x(node), so the four differences are
        // never formed (16 instead of 22 FP64 operations per component).
        // neighbour l: inside the grid from x, else from the ghost cells (array base and stride
        // per neighbour, the same for the three components)
        const C* nbase[4];
        int64_t nstr[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int s2 = (l < 2) ? 1 : -1, s3 = (l & 1) ? -1 : 1;
            const int db = FULL ? -s2 : j0 - ((s2 + 1) >> 1);
            const int na = a + da, nb = b + db, nk = k - s3;
            const bool in = (unsigned)na < (unsigned)G.X && (unsigned)nb < (unsigned)G.Y && (unsigned)nk < (unsigned)G.Z;
            if (in) {
                const int64_t i = na + (int64_t)G.X * (nb + (int64_t)G.Y * nk);
                PC_IDX(i, G.m);
                nbase[l] = x + i;
                nstr[l] = G.m;
            } else {
                const int64_t i = ghost_index(G, na, nb, nk);
                PC_IDX(i, G.ghosts);
                nbase[l] = xg + i;
                nstr[l] = G.ghosts;
            }
        }
        C H[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C n[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) n[l] = nbase[l][c * nstr[l]];
            const C u = cadd(n[0], n[1]), v = cadd(n[2], n[3]);
            const C w = csub(n[0], n[1]), z = csub(n[2], n[3]);
            PC_IDX(c * G.m + t, 3 * G.m);
            H[0][c] = cfma((R)(-4), x[c * G.m + t], cadd(u, v));
            H[1][c] = csub(u, v);
            H[2][c] = cadd(w, z);
        }
        C Gm[3][3];
        if (CUBIC) {
#pragma unroll
            for (int mm = 0; mm < 3; ++mm)
#pragma unroll
                for (int c = 0; c < 3; ++c) Gm[mm][c] = H[mm][c];
        } else {
#pragma unroll
            for (int mm = 0; mm < 3; ++mm)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    C acc = cscale(P.Mmix[0 * 3 + mm], H[0][c]);
                    acc = cfma(P.Mmix[1 * 3 + mm], H[1][c], acc);
                    Gm[mm][c] = cfma(P.Mmix[2 * 3 + mm], H[2][c], acc);
                }
        }
        C e[6];
        e[0] = Gm[0][0];
        e[1] = Gm[1][1];
        e[2] = Gm[2][2];
        e[3] = cadd(Gm[2][1], Gm[1][2]);
        e[4] = cadd(Gm[2][0], Gm[0][2]);
        e[5] = cadd(Gm[1][0], Gm[0][1]);
        const MT mv = read_mat(mat, t);
        C tt[6];
        if (MATK == 2) {
            const R* md = static_cast<const R*>(mat);
            R cn[21];
#pragma unroll
            for (int q = 0; q < 21; ++q) {
                PC_IDX((int64_t)q * G.m + t, 22 * G.m);
                cn[q] = md[(int64_t)q * G.m + t];
            }
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                C acc = cscale(cn[voigt_upper(p, 0)], e[0]);
#pragma unroll
                for (int q = 1; q < 6; ++q) acc = cfma(cn[voigt_upper(p, q)], e[q], acc);
                tt[p] = acc;
            }
        } else if (MATK == 0) {
            const int ph = mv != 0 ? 1 : 0;
            const R* Cp = Ct[ph];
            if (uniform_ortho_ok && warp_all(P.ortho[ph] != 0)) {  // normal block and shear diagonal only
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    C acc = cscale(Cp[p * 6 + 0], e[0]);
                    acc = cfma(Cp[p * 6 + 1], e[1], acc);
                    tt[p] = cfma(Cp[p * 6 + 2], e[2], acc);
                }
#pragma unroll
                for (int p = 3; p < 6; ++p) tt[p] = cscale(Cp[p * 6 + p], e[p]);
            } else {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    C acc = cscale(Cp[p * 6 + 0], e[0]);
#pragma unroll
                    for (int q = 1; q < 6; ++q) acc = cfma(Cp[p * 6 + q], e[q], acc);
                    tt[p] = acc;
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                const R c0 = Ct[0][p * 6 + 0];
                C acc = cscale(c0 + (R)mv * (Ct[1][p * 6 + 0] - c0), e[0]);
#pragma unroll
                for (int q = 1; q < 6; ++q) {
                    const R cq = Ct[0][p * 6 + q];
                    acc = cfma(cq + (R)mv * (Ct[1][p * 6 + q] - cq), e[q], acc);
                }
                tt[p] = acc;
            }
        }
        C S[3][3];
        S[0][0] = tt[0]; S[0][1] = tt[5]; S[0][2] = tt[4];
        S[1][0] = tt[5]; S[1][1] = tt[1]; S[1][2] = tt[3];
        S[2][0] = tt[4]; S[2][1] = tt[3]; S[2][2] = tt[2];
        C Pm[3][3];
        if (CUBIC) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) Pm[s][c] = S[c][s];
        } else {
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    C acc = cscale(P.Mmix[s * 3 + 0], S[c][0]);
                    acc = cfma(P.Mmix[s * 3 + 1], S[c][1], acc);
                    Pm[s][c] = cfma(P.Mmix[s * 3 + 2], S[c][2], acc);
                }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const C u = cadd(Pm[0][c], Pm[1][c]), v = csub(Pm[0][c], Pm[1][c]);
            fe[(0 * 3 + c) * G.ne + own] = cadd(u, Pm[2][c]);
            fe[(1 * 3 + c) * G.ne + own] = csub(u, Pm[2][c]);
            fe[(2 * 3 + c) * G.ne + own] = cadd(v, Pm[2][c]);
            fe[(3 * 3 + c) * G.ne + own] = csub(v, Pm[2][c]);
            fe[(12 + c) * G.ne + own] = Pm[0][c];
        }
    }

    // Pass 4, interior node t: y = sum_l F_l(node + d_l) - 4 P_0 - shift rho x; returns Re<x, y>
    // of the node when want_dot.
    static PC_HD R gather_node(const StencilParams<R>& P, const SplitGeom& G, int p12, int p13, const C* fe,
                               const C* x, C* y, const void* mat, R shift, int64_t t, bool want_dot) {
        int a, b, k;
        split3(t, G.X, G.Y, a, b, k);
        int da = 1, j0 = 0;
        if (!FULL) {
            da = (k + p13) & 1;
            j0 = (k + p12 + p13) & 1;
        }
        const MT mv = read_mat(mat, t);
        R rho;
        if (MATK == 2) rho = static_cast<const R*>(mat)[21 * G.m + t];
        else if (MATK == 0) rho = P.rho[mv != 0 ? 1 : 0];
        else rho = P.rho[0] + (R)mv * (P.rho[1] - P.rho[0]);
        const R sr = shift * rho;
        const int64_t own = eidx(G, a, b, k);
        int64_t nb[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int s2 = (l < 2) ? 1 : -1, s3 = (l & 1) ? -1 : 1;
            const int db = FULL ? s2 : j0 + ((s2 - 1) >> 1);
            nb[l] = eidx(G, a + da, b + db, k + s3);
            PC_IDX(nb[l], G.ne);
        }
        R dot = (R)0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C v = cadd(cadd(fe[(0 * 3 + c) * G.ne + nb[0]], fe[(1 * 3 + c) * G.ne + nb[1]]),
                       cadd(fe[(2 * 3 + c) * G.ne + nb[2]], fe[(3 * 3 + c) * G.ne + nb[3]]));
            v = cfma((R)(-4), fe[(12 + c) * G.ne + own], v);
            const C xv = x[c * G.m + t];
            v = cfma(-sr, xv, v);
            y[c * G.m + t] = v;
            if (want_dot) dot = cdotre(xv, v, dot);
        }
        return dot;
    }
};

}  // namespace pc
