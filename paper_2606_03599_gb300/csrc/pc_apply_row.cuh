// Fused stencil apply, row-tile variant (complex64, parity blocks).
//
// Same operator as pc_apply_tile.cuh (see there for the algebra and the
// quarter-grid layout).  What changes is the tiling and the data movement:
//
// * A tile spans whole rows of the quarter grid: all X columns of the rows
//   [b0, b0 + V).  The a-direction therefore has no halo: a neighbour that
//   leaves [0, X) is the same row's other end times exp(-+i phi_1), selected
//   in registers.
// * The parity structure of the blocks bounds the b-halo to one row per side:
//   fluxes of plane kf are needed on rows [b0 - j0(kf), b0 + V - j0(kf)]
//   (V + 1 rows, the extra row alternating sides with the plane parity), and
//   they read x on rows [b0 - 1, b0 + V].  So one x plane of a tile is V + 2
//   contiguous rows of each component in global memory, fetched by one bulk
//   copy per component (cp.async.bulk, completion on an mbarrier) into a ring
//   of NS plane slots; wrapped halo rows (b0 = 0 or b0 + V = Y) come from the
//   other end of the plane by one-row copies, and planes outside [0, Z) from
//   the wrapped plane.  Their Bloch phases are applied in shared memory after
//   arrival, by the threads, before the plane is used.
// * The material is read the same way from a row-padded copy of the block's
//   phase ids (or theta), so that every row starts 16-byte aligned.
// * Thread (a, tau) owns column a of tile row tau (tau < V) for both the flux
//   and the output, so the local term sum_l F_l and the x and material values
//   needed by the shift term stay in registers; thread row TY computes the
//   extra flux row.  Fluxes go through shared memory once: F_l of node m is
//   read by node m - d_l only.
// * The kernel is persistent: the (item, tile, plane) work is split into equal
//   contiguous ranges, one per CTA, each made of at most a few (item, tile)
//   segments, so every SM gets the same number of planes.
//
// Every mbarrier wait is bounded; a CTA whose copy does not arrive in time
// records an error code and leaves after waiting (bounded) for its copies in
// flight.
#pragma once

#include <math.h>
#include <stdint.h>

#include <cstring>

#include "pc_apply_tma.cuh"

namespace pc {

constexpr int kRowMaxItems = 64;
constexpr int kRowMaxThreads = 512;  // X * (TY + 1) threads per CTA, one CTA per SM
constexpr int kRowMaxSlots = 8;      // x plane ring depth (the most that fits, at least 4)

// Geometry shared by the host launcher, the kernel and the emulator.
struct RowGeom {
    int X, Y, Z;
    int TY;      // maximum tile height (rows)
    int nt;      // tiles per plane
    int NT;      // threads per CTA = X * (TY + 1)
    int SR;      // rows per plane slot = TY + 2
    int Xp;      // material row pitch in elements (16-byte rows)
    int matsz;   // material element size (1 = uint8 phase id, 4 = float theta)
    int ns;      // plane slots in the ring (8 or 4: a power of two, so that ring positions are masks)
    int ns_log2;
    // dynamic shared memory layout (byte offsets from a 128-byte aligned base)
    int slot_bytes, off_mat, off_flux, off_cp, off_rho, off_bar, off_abort, total;
};

PC_HD int row_tile_lo(const RowGeom& G, int t) { return (int)(((int64_t)t * G.Y) / G.nt); }

// Tiles per plane and maximum tile height: as many rows as kRowMaxThreads threads allow
// (one thread per column and tile row, plus the extra flux row), balanced over the tiles.
constexpr int row_tiles_for(int X, int Y) {
    return (Y + ((kRowMaxThreads / X - 1) < 1 ? 1 : ((kRowMaxThreads / X - 1) > Y ? Y : (kRowMaxThreads / X - 1))) -
            1) /
           ((kRowMaxThreads / X - 1) < 1 ? 1 : ((kRowMaxThreads / X - 1) > Y ? Y : (kRowMaxThreads / X - 1)));
}
constexpr int row_ty_for(int X, int Y) { return (Y + row_tiles_for(X, Y) - 1) / row_tiles_for(X, Y); }

inline RowGeom make_row_geom(int X, int Y, int Z, int matkind) {
    RowGeom G;
    G.X = X;
    G.Y = Y;
    G.Z = Z;
    G.nt = row_tiles_for(X, Y);
    G.TY = row_ty_for(X, Y);
    G.NT = X * (G.TY + 1);
    G.SR = G.TY + 2;
    G.matsz = matkind ? 4 : 1;
    const int q = 16 / G.matsz;
    G.Xp = (X + q - 1) / q * q;
    auto al = [](int v) { return (v + 127) / 128 * 128; };
    G.off_mat = 3 * G.SR * X * 8;                            // inside a slot: x [3][SR][X] then material [SR][Xp]
    G.slot_bytes = al(G.off_mat + G.SR * G.Xp * G.matsz);
    const int fixed = al(2 * 12 * G.SR * X * 8) + al(2 * 36 * 8 + 2 * 4) + al(kRowMaxSlots * 8 + 4);
    G.ns = kRowMaxSlots;
    if (G.ns * G.slot_bytes + fixed + 128 + 1024 > 227 * 1024) G.ns = 4;
    G.ns_log2 = G.ns == 8 ? 3 : 2;
    G.off_flux = G.ns * G.slot_bytes;                        // fluxes [2 buffers][4][3][SR][X] float2
    G.off_cp = al(G.off_flux + 2 * 12 * G.SR * X * 8);       // stiffness pairs [2][36] float2
    G.off_rho = G.off_cp + 2 * 36 * 8;
    G.off_bar = al(G.off_rho + 2 * 4);
    G.off_abort = G.off_bar + kRowMaxSlots * 8;
    G.total = al(G.off_abort + 4);
    return G;
}

struct RowBatch {
    ApplyItem it[kRowMaxItems];
    const void* mat_row[kRowMaxItems];  // row-padded material of each item's block
    int n;
    int* err;             // device error word (set to 1 when a bounded wait expires)
    uint32_t wait_limit;  // mbarrier polls before a CTA gives up
};

// One (item, tile) piece of a CTA's plane range.
struct RowSeg {
    int item;
    int b0, V;     // tile rows [b0, b0 + V)
    int ks, ke;    // output planes [ks, ke)
    int p12, p13;
    const float2* x;
    float2* y;
    const void* mat;
    float shift;
};

// Split of the linear work index u = (item * nt + tile) * Z + k.
PC_HD void row_seg_at(const RowGeom& G, int64_t u, int64_t uend, int& item, int& tile, int& ks, int& ke) {
    const int64_t it_tile = u / G.Z;
    item = (int)(it_tile / G.nt);
    tile = (int)(it_tile % G.nt);
    ks = (int)(u % G.Z);
    const int64_t lim = (it_tile + 1) * (int64_t)G.Z;
    ke = (int)((uend < lim ? uend : lim) - it_tile * (int64_t)G.Z);
}

// XC > 0: compile-time row width (then Y = X and the tile height follow at compile time, so all
// shared-memory strides are immediates); XC = 0: runtime width.
template <bool CUBIC, int MATK, int XC = 0>
struct RowTile {
    using C = float2;
    static constexpr int TYC = XC > 0 ? row_ty_for(XC, XC) : 0;

    // Complex arithmetic of this kernel in scalar FP32 instructions: measured on GB300, the
    // packed FP32x2 forms (one issue slot, but the heavy FMA pipe and operand pairing moves)
    // made this latency-bound kernel 3 % slower despite 14 % fewer instructions.  Member
    // functions, so that they take precedence over the packed namespace-level helpers here.
    static PC_HD C cadd(C a, C b) { return make_float2(a.x + b.x, a.y + b.y); }
    static PC_HD C csub(C a, C b) { return make_float2(a.x - b.x, a.y - b.y); }
    static PC_HD C cscale(float r, C a) { return make_float2(r * a.x, r * a.y); }
    static PC_HD C cfma(float r, C a, C acc) { return make_float2(fmaf(r, a.x, acc.x), fmaf(r, a.y, acc.y)); }
    static PC_HD C cmul(C a, C b) { return make_float2(fmaf(-a.y, b.y, a.x * b.x), fmaf(a.y, b.x, a.x * b.y)); }
    static PC_HD C stiff_fma_pair(C c, C e, C acc) { return make_float2(fmaf(c.x, e.x, acc.x), fmaf(c.y, e.y, acc.y)); }
    static PC_HD int Xw(const RowGeom& G) { return XC > 0 ? XC : G.X; }
    static PC_HD int SRw(const RowGeom& G) { return XC > 0 ? TYC + 2 : G.SR; }
    static PC_HD int TYw(const RowGeom& G) { return XC > 0 ? TYC : G.TY; }

    struct Regs {
        int a, tau;
        C acc_prev[3], acc_cur[3];  // outputs of planes kf - 1 and kf
        C xo_prev[3];               // own x of plane kf - 1 (shift term)
        float mo_prev;              // own material of plane kf - 1
        C xo_new[3];
        float mo_new;
        C local[3];                 // sum_l F_l of the own node at plane kf
        float dot;
    };

    struct Sh {  // views into dynamic shared memory
        unsigned char* base;
        const RowGeom* G;
        PC_HD C* xslot(int slot) const { return reinterpret_cast<C*>(base + (size_t)slot * G->slot_bytes); }
        PC_HD unsigned char* mslot(int slot) const { return base + (size_t)slot * G->slot_bytes + G->off_mat; }
        PC_HD C* flux(int buf) const {
            return reinterpret_cast<C*>(base + G->off_flux + (size_t)buf * 12 * G->SR * G->X * sizeof(C));
        }
        PC_HD float2* cp() const { return reinterpret_cast<float2*>(base + G->off_cp); }
        PC_HD float* rho() const { return reinterpret_cast<float*>(base + G->off_rho); }
        PC_HD uint64_t* bar() const { return reinterpret_cast<uint64_t*>(base + G->off_bar); }
        PC_HD int* abort_flag() const { return reinterpret_cast<int*>(base + G->off_abort); }
    };

    static PC_HD C phase_of(const StencilParams<float>& P, int axis, int w) {
        if (w == 0) return cmk(1.f, 0.f);
        return cmk(P.ph[axis][0], w < 0 ? -P.ph[axis][1] : P.ph[axis][1]);
    }

    static PC_HD float mat_at(const Sh& sh, int slot, int s, int a) {
        const unsigned char* m = sh.mslot(slot);
        const int idx = s * sh.G->Xp + a;
        PC_IDX(idx, sh.G->SR * sh.G->Xp);
        if (MATK == 0) return (float)m[idx];
        return reinterpret_cast<const float*>(m)[idx];
    }

    static PC_HD void load_tables(const StencilParams<float>& P, const Sh& sh, int tid, int nthreads) {
        for (int i = tid; i < 72; i += nthreads) sh.cp()[i] = make_float2(P.C[i / 36][i % 36], P.C[i / 36][i % 36]);
        if (tid < 2) sh.rho()[tid] = P.rho[tid];
    }

    static PC_HD void init(const RowGeom& G, int tid, Regs& r) {
        r.a = tid % Xw(G);
        r.tau = tid / Xw(G);
        r.dot = 0.f;
    }

    static PC_HD void seg_begin(Regs& r) {
        for (int c = 0; c < 3; ++c) {
            r.acc_prev[c] = r.acc_cur[c] = r.xo_prev[c] = r.xo_new[c] = r.local[c] = czero(0.f);
        }
        r.mo_prev = r.mo_new = 0.f;
    }

    // Plane kp has landed in `slot`: apply the Bloch phases of wrapped rows / planes.
    static PC_HD void fix_plane(const StencilParams<float>& P, const RowGeom& G, const RowSeg& S, const Sh& sh,
                                int slot, int kp, int tid) {
        const int wk = kp < 0 ? -1 : (kp >= G.Z ? 1 : 0);
        const bool top = S.b0 == 0, bot = S.b0 + S.V == G.Y;
        if (wk == 0 && !top && !bot) return;
        C* xs = sh.xslot(slot);
        const C phk = phase_of(P, 2, wk);
        const C pht = cmul(phk, phase_of(P, 1, -1)), phb = cmul(phk, phase_of(P, 1, 1));
        const int rows = S.V + 2;
        if (wk != 0) {
            const int n = 3 * rows * G.X;
            for (int e = tid; e < n; e += G.NT) {
                const int s = (e / G.X) % rows, c = e / (G.X * rows);
                const int idx = (c * G.SR + s) * G.X + e % G.X;
                PC_IDX(idx, 3 * G.SR * G.X);
                const C ph = (s == 0 && top) ? pht : ((s == rows - 1 && bot) ? phb : phk);
                xs[idx] = cmul(xs[idx], ph);
            }
        } else {
            const int n = 3 * 2 * G.X;
            for (int e = tid; e < n; e += G.NT) {
                const int side = (e / G.X) & 1, c = e / (2 * G.X);
                if (side == 0 && !top) continue;
                if (side == 1 && !bot) continue;
                const int s = side == 0 ? 0 : rows - 1;
                const int idx = (c * G.SR + s) * G.X + e % G.X;
                PC_IDX(idx, 3 * G.SR * G.X);
                xs[idx] = cmul(xs[idx], side == 0 ? pht : phb);
            }
        }
    }

    // Fluxes F_l (l = 0..3) of one node from its backward differences g[l][alpha] and material m;
    // also returns sum_l F_l (= 4 P_0).
    static PC_HD void flux_math(const StencilParams<float>& P, const Sh& sh, float m, const C g[4][3], C F[4][3],
                                C loc[3]) {
        C H[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const C u = cadd(g[0][a], g[1][a]), v = cadd(g[2][a], g[3][a]);
            const C w = csub(g[0][a], g[1][a]), z = csub(g[2][a], g[3][a]);
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
            const int ph = m != 0.f ? 1 : 0;
            const float2* Cq = sh.cp() + 36 * ph;
            if (warp_all(P.ortho[ph] != 0)) {  // every node of the warp: normal block and shear diagonal only
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    C acc = czero(0.f);
#pragma unroll
                    for (int q = 0; q < 3; ++q) acc = stiff_fma_pair(Cq[p * 6 + q], e[q], acc);
                    t[p] = acc;
                }
#pragma unroll
                for (int p = 3; p < 6; ++p) t[p] = stiff_fma_pair(Cq[p * 6 + p], e[p], czero(0.f));
            } else {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    C acc = czero(0.f);
#pragma unroll
                    for (int q = 0; q < 6; ++q) acc = stiff_fma_pair(Cq[p * 6 + q], e[q], acc);
                    t[p] = acc;
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                C acc = czero(0.f);
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const float c0 = P.C[0][p * 6 + q], c1 = P.C[1][p * 6 + q];
                    acc = cfma(c0 + m * (c1 - c0), e[q], acc);
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
            const C u = cadd(Pm[0][a], Pm[1][a]), v = csub(Pm[0][a], Pm[1][a]);
            F[0][a] = cadd(u, Pm[2][a]);
            F[1][a] = csub(u, Pm[2][a]);
            F[2][a] = cadd(v, Pm[2][a]);
            F[3][a] = csub(v, Pm[2][a]);
            loc[a] = cscale(4.f, Pm[0][a]);
        }
    }

    // Fluxes of the thread's node at plane kf (slots of planes kf - 1, kf, kf + 1) into shared memory.
    static PC_HD void flux(const StencilParams<float>& P, const RowGeom& G, const RowSeg& S, const Sh& sh, Regs& r,
                           int kf, int slot_m, int slot_0, int slot_p, int buf) {
        const int i0 = (kf + S.p13) & 1, j0 = (kf + S.p12 + S.p13) & 1;
        int b;
        if (r.tau < S.V) b = S.b0 + r.tau;
        else if (r.tau == TYw(G)) b = j0 ? S.b0 - 1 : S.b0 + S.V;
        else return;
        const int so = b - S.b0 + 1;
        const int X = Xw(G), SR = SRw(G), a = r.a;
        int na = a + i0 - 1;
        const bool wa = na < 0;
        if (wa) na += X;
        const C* xm = sh.xslot(slot_m);
        const C* x0 = sh.xslot(slot_0);
        const C* xp = sh.xslot(slot_p);
        const int rowp = so + j0 - 1, rowm = so + j0;  // neighbour rows of s2 = +1 and s2 = -1
        PC_IDX(rowp, S.V + 2);
        PC_IDX(rowm, S.V + 2);
        const C pha = phase_of(P, 0, -1);
        C g[4][3], xo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int cb = c * SR;
            xo[c] = x0[(cb + so) * X + a];
            C n0 = xm[(cb + rowp) * X + na];  // l = 0: s2 = +1, s3 = +1 (plane kf - 1)
            C n1 = xp[(cb + rowp) * X + na];  // l = 1: s2 = +1, s3 = -1 (plane kf + 1)
            C n2 = xm[(cb + rowm) * X + na];  // l = 2: s2 = -1, s3 = +1
            C n3 = xp[(cb + rowm) * X + na];  // l = 3: s2 = -1, s3 = -1
            if (wa) {
                n0 = cmul(n0, pha);
                n1 = cmul(n1, pha);
                n2 = cmul(n2, pha);
                n3 = cmul(n3, pha);
            }
            g[0][c] = csub(n0, xo[c]);
            g[1][c] = csub(n1, xo[c]);
            g[2][c] = csub(n2, xo[c]);
            g[3][c] = csub(n3, xo[c]);
        }
        const float m = mat_at(sh, slot_0, so, a);
        C F[4][3], loc[3];
        flux_math(P, sh, m, g, F, loc);
        C* fs = sh.flux(buf);
#pragma unroll
        for (int l = 0; l < 4; ++l)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int idx = ((l * 3 + c) * SR + so) * X + a;
                PC_IDX(idx, 12 * G.SR * G.X);
                fs[idx] = F[l][c];
            }
        if (r.tau < S.V) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                r.local[c] = loc[c];
                r.xo_new[c] = xo[c];
            }
            r.mo_new = m;
        }
    }

    // Finish y(kf - 1), add the local term of y(kf), start y(kf + 1).
    static PC_HD void gather(const StencilParams<float>& P, const RowGeom& G, const RowSeg& S, const Sh& sh,
                             Regs& r, int kf, int buf) {
        if (r.tau >= S.V) return;
        const int X = Xw(G), SR = SRw(G), a = r.a, so = r.tau + 1;
        const int p = kf - 1;  // planes kf - 1 and kf + 1 have the same parity
        const int i0 = (p + S.p13) & 1, j0 = (p + S.p12 + S.p13) & 1;
        int na = a + i0;
        const bool wa = na >= X;
        if (wa) na -= X;
        const C pha = phase_of(P, 0, 1);
        const int rp = so + j0, rm = so + j0 - 1;  // flux rows of s2 = +1 and s2 = -1
        PC_IDX(rp, S.V + 2);
        PC_IDX(rm, S.V + 2);
        const C* fs = sh.flux(buf);
        const int64_t plane = (int64_t)X * (XC > 0 ? XC : G.Y), vstr = plane * G.Z;
        C acc_next[3];
        if (p >= S.ks && p < S.ke) {
            const float rho = (MATK == 0) ? sh.rho()[r.mo_prev != 0.f ? 1 : 0]
                                          : sh.rho()[0] + r.mo_prev * (sh.rho()[1] - sh.rho()[0]);
            const float sr = S.shift * rho;
            const int64_t ob = (int64_t)p * plane + (int64_t)(S.b0 + r.tau) * X + a;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                C f = cadd(fs[((0 * 3 + c) * SR + rp) * X + na], fs[((2 * 3 + c) * SR + rm) * X + na]);
                if (wa) f = cmul(f, pha);
                C v = cadd(r.acc_prev[c], f);
                v = cfma(-sr, r.xo_prev[c], v);
                PC_IDX(c * vstr + ob, 3 * vstr);
                S.y[c * vstr + ob] = v;
                r.dot = cdotre(r.xo_prev[c], v, r.dot);
            }
        }
        if (kf >= S.ks && kf < S.ke) {
#pragma unroll
            for (int c = 0; c < 3; ++c) r.acc_cur[c] = csub(r.acc_cur[c], r.local[c]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) acc_next[c] = czero(0.f);
        if (kf + 1 >= S.ks && kf + 1 < S.ke) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                C f = cadd(fs[((1 * 3 + c) * SR + rp) * X + na], fs[((3 * 3 + c) * SR + rm) * X + na]);
                if (wa) f = cmul(f, pha);
                acc_next[c] = f;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            r.acc_prev[c] = r.acc_cur[c];
            r.acc_cur[c] = acc_next[c];
            r.xo_prev[c] = r.xo_new[c];
        }
        r.mo_prev = r.mo_new;
    }

    // Host model of the copies of plane kp (same source rows and wraps as the kernel's bulk copies).
    static void host_copy_plane(const RowGeom& G, const RowSeg& S, const Sh& sh, int slot, int kp) {
        const int kw = ((kp % G.Z) + G.Z) % G.Z;
        C* xs = sh.xslot(slot);
        unsigned char* ms = sh.mslot(slot);
        for (int s = 0; s < S.V + 2; ++s) {
            const int b = ((S.b0 - 1 + s) % G.Y + G.Y) % G.Y;
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < G.X; ++a)
                    xs[(c * G.SR + s) * G.X + a] =
                        S.x[(int64_t)c * G.X * G.Y * G.Z + ((int64_t)kw * G.Y + b) * G.X + a];
            std::memcpy(ms + (size_t)s * G.Xp * G.matsz,
                        static_cast<const unsigned char*>(S.mat) + ((size_t)kw * G.Y + b) * G.Xp * G.matsz,
                        (size_t)G.Xp * G.matsz);
        }
    }
};

}  // namespace pc
