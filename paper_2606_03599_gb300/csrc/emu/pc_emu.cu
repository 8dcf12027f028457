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
#include "../pc_apply_row.cuh"
#include "../pc_apply_pipe.cuh"
#include "../pc_apply_split.cuh"
#include "../pc_small_dft.cuh"

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
            c.dot = true;
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

// Same segment and step sequence as apply_row_kernel (complex64 parity blocks) with `ctas`
// persistent CTAs; the bulk copies are modelled as immediate copies of the same rows.
template <bool CUBIC, int MATK, int XC>
static void emu_run_row(const StencilParams<float>& P, int block, const void* x, void* y, const void* mat,
                        double shift, int ctas) {
    using T = RowTile<CUBIC, MATK, XC>;
    const RowGeom G = make_row_geom(P.X, P.Y, P.Z, MATK);
    if (XC > 0 && (G.X != XC || G.Y != XC)) {
        std::fprintf(stderr, "compile-time width %d does not match the grid\n", XC);
        std::abort();
    }
    const uint32_t NS = (uint32_t)G.ns;
    // row-padded material copy
    std::vector<unsigned char> matp((size_t)G.Xp * G.Y * G.Z * G.matsz, 0);
    for (int64_t row = 0; row < (int64_t)G.Y * G.Z; ++row)
        std::memcpy(&matp[(size_t)row * G.Xp * G.matsz],
                    static_cast<const unsigned char*>(mat) + (size_t)row * G.X * G.matsz, (size_t)G.X * G.matsz);
    std::vector<unsigned char> smem(G.total);
    typename T::Sh sh{smem.data(), &G};
    std::vector<typename T::Regs> regs(G.NT);
    const int64_t W = (int64_t)G.nt * G.Z;  // one item
    for (int cta = 0; cta < ctas; ++cta) {
        std::memset(smem.data(), 0xFF, smem.size());  // poison: reads of unwritten cells show up as NaN
        for (int t = 0; t < G.NT; ++t) T::load_tables(P, sh, t, G.NT);
        for (int t = 0; t < G.NT; ++t) T::init(G, t, regs[t]);
        const int64_t u0 = (int64_t)cta * W / ctas, u1 = (int64_t)(cta + 1) * W / ctas;
        uint32_t gseq = 0;
        for (int64_t u = u0; u < u1;) {
            int item, tile, ks, ke;
            row_seg_at(G, u, u1, item, tile, ks, ke);
            u += ke - ks;
            PC_IDX(item, 1);
            RowSeg S;
            S.item = item;
            S.b0 = row_tile_lo(G, tile);
            S.V = row_tile_lo(G, tile + 1) - S.b0;
            if (S.V < 1 || S.V > G.TY) {
                std::fprintf(stderr, "bad tile height %d\n", S.V);
                std::abort();
            }
            S.ks = ks;
            S.ke = ke;
            S.p12 = block >> 1;
            S.p13 = block & 1;
            S.x = static_cast<const float2*>(x);
            S.y = static_cast<float2*>(y);
            S.mat = matp.data();
            S.shift = (float)shift;
            for (int t = 0; t < G.NT; ++t) T::seg_begin(regs[t]);
            const int kfirst = ks - 2;
            auto slot_of = [&](int kp) { return (int)((gseq + (uint32_t)(kp - kfirst)) & (NS - 1)); };
            for (int kp = kfirst; kp <= ke + 1 && kp < kfirst + (int)NS; ++kp)
                T::host_copy_plane(G, S, sh, slot_of(kp), kp);
            for (int kp = kfirst; kp <= ks; ++kp)
                for (int t = 0; t < G.NT; ++t) T::fix_plane(P, G, S, sh, slot_of(kp), kp, t);
            for (int kf = ks - 1; kf <= ke; ++kf) {
                for (int t = 0; t < G.NT; ++t) {
                    if (kf > ks - 1) T::gather(P, G, S, sh, regs[t], kf - 1, (kf - 1) & 1);
                    T::flux(P, G, S, sh, regs[t], kf, slot_of(kf - 1), slot_of(kf), slot_of(kf + 1), kf & 1);
                }
                if (kf + 2 <= ke + 1)
                    for (int t = 0; t < G.NT; ++t) T::fix_plane(P, G, S, sh, slot_of(kf + 2), kf + 2, t);
                if (kf - 1 >= kfirst && kf - 1 + (int)NS <= ke + 1)
                    T::host_copy_plane(G, S, sh, slot_of(kf - 1 + (int)NS), kf - 1 + (int)NS);
            }
            for (int t = 0; t < G.NT; ++t) T::gather(P, G, S, sh, regs[t], ke, ke & 1);
            gseq += (uint32_t)(ke - ks + 4);
        }
    }
}

template <bool CUBIC, int MATK>
static void emu_row_x(const StencilParams<float>& P, int block, const void* x, void* y, const void* mat,
                      double shift, int ctas, bool ct) {
    if (ct && MATK == 0 && P.X == P.Y) {
        switch (P.X) {
            case 16: return emu_run_row<CUBIC, MATK, 16>(P, block, x, y, mat, shift, ctas);
            case 24: return emu_run_row<CUBIC, MATK, 24>(P, block, x, y, mat, shift, ctas);
            case 32: return emu_run_row<CUBIC, MATK, 32>(P, block, x, y, mat, shift, ctas);
            default: break;
        }
    }
    emu_run_row<CUBIC, MATK, 0>(P, block, x, y, mat, shift, ctas);
}

// Same segment, plane and step sequence as apply_pipe_kernel (complex64 parity blocks) with
// `ctas` persistent CTAs.  The producer is modelled as issuing each plane copy as early as the
// kernel's ring allows (right after the consumers release the slot's previous plane), so a
// premature reuse of a slot shows up as a wrong output; the copies are immediate.
template <bool CUBIC, int MATK, int XC, int TC>
static void emu_run_pipe(const StencilParams<float>& P, int block, const void* x, void* y, const void* mat,
                         double shift, int ctas, int Tr) {
    using T = PipeTile<CUBIC, MATK, XC, TC>;
    const PipeGeom G = make_pipe_geom(P.X, P.Y, P.Z, MATK, XC > 0 ? TC : Tr);
    if ((XC > 0 && (G.X != XC || G.Y != XC)) || !pipe_geom_fits(G) || (G.X & 1)) {
        std::fprintf(stderr, "pipe geometry not supported\n");
        std::abort();
    }
    const size_t NS = (size_t)G.ns;
    std::vector<unsigned char> matp((size_t)G.Xp * G.Y * G.Z * G.matsz, 0);
    for (int64_t row = 0; row < (int64_t)G.Y * G.Z; ++row)
        std::memcpy(&matp[(size_t)row * G.Xp * G.matsz],
                    static_cast<const unsigned char*>(mat) + (size_t)row * G.X * G.matsz, (size_t)G.X * G.matsz);
    std::vector<unsigned char> smem(G.total);
    typename T::Sh sh{smem.data(), &G};
    std::vector<typename T::Regs> regs(G.NC);
    float2 eph[3];  // the item's Bloch phases
    for (int l = 0; l < 3; ++l) eph[l] = make_float2(P.ph[l][0], P.ph[l][1]);
    const int64_t W = (int64_t)G.nt * G.Z;  // one item
    for (int cta = 0; cta < ctas; ++cta) {
        std::memset(smem.data(), 0xFF, smem.size());  // poison: reads of unwritten cells show up as NaN
        for (int t = 0; t < G.NC; ++t) T::load_tables(P, sh, t, G.NC);
        for (int t = 0; t < G.NC; ++t) T::init(G, t, regs[t]);
        const int64_t u0 = (int64_t)cta * W / ctas, u1 = (int64_t)(cta + 1) * W / ctas;
        // the CTA's segments and, in order, every plane the producer copies
        std::vector<PipeSeg> segs;
        std::vector<std::pair<int, int>> seq;  // (segment, plane)
        for (int64_t u = u0; u < u1;) {
            int item, tile, ks, ke;
            pipe_seg_at(G, u, u1, item, tile, ks, ke);
            u += ke - ks;
            PC_IDX(item, 1);
            PipeSeg S;
            S.b0 = pipe_tile_lo(G, tile);
            S.Vt = pipe_tile_lo(G, tile + 1) - S.b0;
            if (S.Vt < 1 || S.Vt > G.V) {
                std::fprintf(stderr, "bad tile height %d\n", S.Vt);
                std::abort();
            }
            S.top = S.b0 == 0;
            S.bot = S.b0 + S.Vt == G.Y;
            S.ks = ks;
            S.ke = ke;
            S.p12 = block >> 1;
            S.p13 = block & 1;
            S.x = static_cast<const float2*>(x);
            S.y = static_cast<float2*>(y);
            S.mat = matp.data();
            S.ph = eph;
            S.shift = (float)shift;
            for (int kp = ks - 2; kp <= ke + 1; ++kp) seq.emplace_back((int)segs.size(), kp);
            segs.push_back(S);
        }
        size_t issued = 0;
        std::vector<char> released(seq.size(), 0);
        auto pump = [&]() {
            while (issued < seq.size() && (issued < NS || released[issued - NS])) {
                T::host_copy_plane(G, segs[seq[issued].first], sh, (int)(issued % NS), seq[issued].second);
                ++issued;
            }
        };
        auto need = [&](size_t qq) {
            pump();
            if (qq >= issued) {
                std::fprintf(stderr, "plane %zu needed before it can be issued (ring deadlock)\n", qq);
                std::abort();
            }
        };
        auto release = [&](size_t qq) {
            PC_IDX(qq, seq.size());
            if (released[qq]) {
                std::fprintf(stderr, "plane %zu released twice\n", qq);
                std::abort();
            }
            released[qq] = 1;
            pump();
        };
        // launches with an odd CTA count model the launch without the inner product (its slots are
        // released before the flux step instead of after the gather)
        const bool want_dot = (ctas & 1) == 0;
        size_t q = 0;
        for (const PipeSeg& S : segs) {
            for (int t = 0; t < G.NC; ++t) T::seg_begin(regs[t]);
            const size_t q0 = q;
            auto slot_of = [&](int kp) { return (int)((q0 + (size_t)(kp - S.ks + 2)) % NS); };
            need(q0);
            need(q0 + 1);
            for (int t = 0; t < G.NC; ++t) T::prologue(P, G, S, sh, regs[t], slot_of(S.ks - 2), slot_of(S.ks - 1));
            const int nsteps = S.ke - S.ks + 2;
            for (int j = 0; j < nsteps; ++j) {
                const int kf = S.ks - 1 + j;
                if (!want_dot) release(q0 + (size_t)j);
                need(q0 + (size_t)j + 2);
                const int buf = j & 1;
                for (int t = 0; t < G.NC; ++t) {
                    if (j & 1) T::template flux_step<1>(P, G, S, sh, regs[t], kf, slot_of(kf), slot_of(kf + 1), buf);
                    else T::template flux_step<0>(P, G, S, sh, regs[t], kf, slot_of(kf), slot_of(kf + 1), buf);
                }
                for (int t = 0; t < G.NC; ++t) {
                    if (j & 1) T::template gather_step<1>(P, G, S, sh, regs[t], kf, slot_of(kf - 1), buf, want_dot);
                    else T::template gather_step<0>(P, G, S, sh, regs[t], kf, slot_of(kf - 1), buf, want_dot);
                }
                if (want_dot) release(q0 + (size_t)j);
            }
            release(q0 + (size_t)nsteps);
            release(q0 + (size_t)nsteps + 1);
            q = q0 + (size_t)nsteps + 2;
        }
        if (q != seq.size()) {
            std::fprintf(stderr, "plane sequence mismatch\n");
            std::abort();
        }
    }
}

template <bool CUBIC, int MATK>
static void emu_pipe_x(const StencilParams<float>& P, int block, const void* x, void* y, const void* mat,
                       double shift, int ctas, bool ct, int Tr) {
    if (ct && MATK == 0 && P.X == P.Y) {
        switch (P.X) {
            case 16: return emu_run_pipe<CUBIC, MATK, 16, pipe_rows_for(16)>(P, block, x, y, mat, shift, ctas, 0);
            case 24: return emu_run_pipe<CUBIC, MATK, 24, pipe_rows_for(24)>(P, block, x, y, mat, shift, ctas, 0);
            case 32: return emu_run_pipe<CUBIC, MATK, 32, pipe_rows_for(32)>(P, block, x, y, mat, shift, ctas, 0);
            default: break;
        }
    }
    emu_run_pipe<CUBIC, MATK, 0, 0>(P, block, x, y, mat, shift, ctas, Tr);
}

// Same four passes as the two-pass complex128 kernels, scratch poisoned with NaN first so that
// a read of a cell no pass wrote shows up in the output.
template <typename R, bool FULL, bool CUBIC, int MATK>
static void emu_run_split(const StencilParams<R>& P, int block, const void* x, void* y, const void* mat,
                          double shift) {
    using T = SplitApply<R, FULL, CUBIC, MATK>;
    using C = typename CT<R>::T;
    const SplitGeom G = make_split_geom(P.X, P.Y, P.Z);
    std::vector<C> xg(3 * G.ghosts), fe(15 * G.ne);
    std::memset((void*)xg.data(), 0xFF, sizeof(C) * xg.size());
    std::memset((void*)fe.data(), 0xFF, sizeof(C) * fe.size());
    const int p12 = FULL ? 0 : (block >> 1), p13 = FULL ? 0 : (block & 1);
    const C* xv = static_cast<const C*>(x);
    for (int64_t gi = 0; gi < G.ghosts; ++gi) T::fill_x_ghost(P.ph, G, xv, xg.data(), gi);
    R Ct[2][36];
    for (int i = 0; i < 72; ++i) Ct[i / 36][i % 36] = P.C[i / 36][i % 36];
    for (int64_t t = 0; t < G.m; ++t) T::flux_node(P, Ct, G, p12, p13, xv, xg.data(), mat, fe.data(), t, true);
    for (int64_t gi = 0; gi < G.ghosts; ++gi) T::fill_f_ghost(P.ph, G, fe.data(), gi);
    for (int64_t t = 0; t < G.m; ++t)
        T::gather_node(P, G, p12, p13, fe.data(), xv, static_cast<C*>(y), mat, (R)shift, t, true);
}

template <typename R, bool FULL, bool CUBIC, int MATK>
static int emu_shape(int shape, const StencilParams<R>& P, int block, const void* x, void* y, const void* mat,
                     double shift, int tz) {
    constexpr bool F32 = sizeof(R) == 4;
    switch (shape) {
        case 30: emu_run_split<R, FULL, CUBIC, MATK>(P, block, x, y, mat, shift); break;
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
        if (shape == 20 || shape == 21) {  // row-tile kernel (21: compile-time width), tz = persistent CTAs
            if (full) return -1;
            const bool ct = shape == 21;
            if (cubic) {
                if (matkind) emu_row_x<true, 1>(P, block, x, y, mat, shift, tz, ct);
                else emu_row_x<true, 0>(P, block, x, y, mat, shift, tz, ct);
            } else {
                if (matkind) emu_row_x<false, 1>(P, block, x, y, mat, shift, tz, ct);
                else emu_row_x<false, 0>(P, block, x, y, mat, shift, tz, ct);
            }
            return 0;
        }
        if (shape == 40 || shape == 41 || (shape > 50 && shape <= 58)) {
            // plane-pipelined kernel (41: compile-time width; 5T: runtime geometry with T thread rows),
            // tz = persistent CTAs
            if (full) return -1;
            const bool ct = shape == 41;
            const int Tr = shape > 50 ? shape - 50 : 0;
            if (cubic) {
                if (matkind) emu_pipe_x<true, 1>(P, block, x, y, mat, shift, tz, ct, Tr);
                else emu_pipe_x<true, 0>(P, block, x, y, mat, shift, tz, ct, Tr);
            } else {
                if (matkind) emu_pipe_x<false, 1>(P, block, x, y, mat, shift, tz, ct, Tr);
                else emu_pipe_x<false, 0>(P, block, x, y, mat, shift, tz, ct, Tr);
            }
            return 0;
        }
        return emu_t<float>(shape, P, full, cubic != 0, matkind, block, x, y, mat, shift, tz);
    }
    StencilParams<double> P;
    make_stencil_params(P, Chat, rhohat2, ainv9, cubic != 0, N, phi3, X, Y, Z);
    if (matkind == 2) {  // nodewise material: the two-pass kernels only ([22][m] FP64 in mat)
        if (shape != 30) return -1;
        if (full) cubic ? emu_run_split<double, true, true, 2>(P, block, x, y, mat, shift)
                        : emu_run_split<double, true, false, 2>(P, block, x, y, mat, shift);
        else cubic ? emu_run_split<double, false, true, 2>(P, block, x, y, mat, shift)
                   : emu_run_split<double, false, false, 2>(P, block, x, y, mat, shift);
        return 0;
    }
    return emu_t<double>(shape, P, full, cubic != 0, matkind, block, x, y, mat, shift, tz);
}

// The L-point DFT of the Bloch transform kernels (compile-time roots) on one complex128 vector.
template <int L>
static void emu_sdft_l(int inv, const double* in, double* out) {
    double2 v[16];
    for (int i = 0; i < L; ++i) v[i] = make_double2(in[2 * i], in[2 * i + 1]);
    if (inv) small_dft_ct<L, true>(v);
    else small_dft_ct<L, false>(v);
    for (int i = 0; i < L; ++i) {
        out[2 * i] = v[i].x;
        out[2 * i + 1] = v[i].y;
    }
}

extern "C" int pc_emu_small_dft(int L, int inv, const double* in, double* out) {
    switch (L) {
#define PC_L(n) case n: emu_sdft_l<n>(inv, in, out); return 0;
        PC_L(1) PC_L(2) PC_L(3) PC_L(4) PC_L(5) PC_L(6) PC_L(7) PC_L(8)
        PC_L(9) PC_L(10) PC_L(11) PC_L(12) PC_L(13) PC_L(14) PC_L(15) PC_L(16)
#undef PC_L
        default: return -1;
    }
}

// The ghost-cell numbering of the two-pass kernels: ghost_cell(gi) lies on the one-cell layer
// around the X x Y x Z interior, every such cell is hit exactly once, and ghost_index inverts it.
// Returns the number of violations (0 = consistent).
extern "C" long long pc_emu_ghost_cells(int X, int Y, int Z) {
    using T = SplitApply<double, false, true, 0>;
    const SplitGeom G = make_split_geom(X, Y, Z);
    std::vector<int> hits((size_t)G.ne, 0);
    long long bad = 0;
    for (int64_t gi = 0; gi < G.ghosts; ++gi) {
        int a, b, k;
        T::ghost_cell(G, gi, a, b, k);
        const bool inside = a >= 0 && a < X && b >= 0 && b < Y && k >= 0 && k < Z;
        const bool layer = a >= -1 && a <= X && b >= -1 && b <= Y && k >= -1 && k <= Z;
        if (inside || !layer) {
            ++bad;
            continue;
        }
        hits[(size_t)T::eidx(G, a, b, k)] += 1;
        if (T::ghost_index(G, a, b, k) != gi) ++bad;
    }
    for (int k = -1; k <= Z; ++k)
        for (int b = -1; b <= Y; ++b)
            for (int a = -1; a <= X; ++a) {
                const bool inside = a >= 0 && a < X && b >= 0 && b < Y && k >= 0 && k < Z;
                if (!inside && hits[(size_t)T::eidx(G, a, b, k)] != 1) ++bad;
            }
    return bad;
}
