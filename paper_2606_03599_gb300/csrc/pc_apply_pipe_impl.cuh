// CUDA kernel of the plane-pipelined stencil apply (complex64 parity blocks) and its launcher.
// Included by the translation units that instantiate it (see pc_apply_pipe.cuh for the design).
#pragma once

#include <cstdlib>
#include <mutex>
#include <string>

#include "pc_apply_pipe.cuh"

namespace pc {

#if defined(__CUDACC__)
__device__ __forceinline__ void pipe_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void pipe_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// named barrier of the consumer warps (id 1; id 0 is __syncthreads)
__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
#endif

template <bool CUBIC, int MATK, int XC, int TC, bool PK>
__global__ void __launch_bounds__(XC > 0 ? (XC * TC + 31) / 32 * 32 + 32 : kPipeMaxThreads, 1)
    apply_pipe_kernel(const __grid_constant__ StencilParams<float> P, const __grid_constant__ PipeBatch B,
                      const __grid_constant__ PipeGeom G, int64_t W, double* __restrict__ dot_partials,
                      int dot_stride) {
    using T = PipeTile<CUBIC, MATK, XC, TC, PK>;
    // The window is used as it comes (16-byte aligned, which is all the bulk copies and the
    // 8-byte mbarriers need): no integer round trip, so every access stays a 32-bit shared one.
    extern __shared__ __align__(16) unsigned char smem_pipe[];
    typename T::Sh sh{smem_pipe, &G};
    const int tid = threadIdx.x;
    const int NC = XC > 0 ? (XC * TC + 31) / 32 * 32 : G.NC;
    const int NS = G.ns;
    uint64_t* full = sh.full();
    uint64_t* empty = sh.empty();
    volatile int* flag = sh.flag();
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC / 32);
        }
        *flag = 0;
        fence_mbar_init();
        if (dot_partials != nullptr)
            for (int i = 0; i < B.n; ++i)
                if (B.it[i].dot_slot >= 0) dot_partials[(int64_t)B.it[i].dot_slot * dot_stride + blockIdx.x] = 0.0;
    }
    if (tid < NC) T::load_tables(P, sh, tid, NC);
    __syncthreads();

    const int64_t u0 = (int64_t)blockIdx.x * W / gridDim.x, u1 = (int64_t)(blockIdx.x + 1) * W / gridDim.x;

    // ------------------------------------------------------------------ producer warp
    if (tid >= NC) {
        if (tid != NC) return;
        uint32_t q = 0;  // planes issued so far; plane q goes to slot q % NS, round q / NS
        bool abort = false;
        for (int64_t u = u0; u < u1 && !abort;) {
            int item, tile, ks, ke;
            pipe_seg_at(G, u, u1, item, tile, ks, ke);
            u += ke - ks;
            const ApplyItem& it = B.it[item];
            if (it.skip != nullptr && *it.skip) continue;
            const int b0 = pipe_tile_lo(G, tile), Vt = pipe_tile_lo(G, tile + 1) - b0;
            const float2* x = static_cast<const float2*>(it.x);
            const char* mat = static_cast<const char*>(B.mat_row[item]);
            const uint32_t xrow = (uint32_t)G.X * 8u, mrow = (uint32_t)G.Xp * (uint32_t)G.matsz;
            const int64_t cstr = (int64_t)G.X * G.Y * G.Z;
            const int lo = b0 - 1 < 0 ? 0 : b0 - 1;
            const int hi = b0 + Vt > G.Y - 1 ? G.Y - 1 : b0 + Vt;
            const int s_lo = lo - (b0 - 1);
            const uint32_t nr = (uint32_t)(hi - lo + 1);
            for (int kp = ks - 2; kp <= ke + 1; ++kp, ++q) {
                const int slot = (int)(q % (uint32_t)NS);
                const uint32_t round = q / (uint32_t)NS;
                if (round > 0) {  // wait until the consumers released the slot's previous plane
                    bool ok = false;
                    for (uint32_t n = 0; n < B.wait_limit && !ok; ++n) {
                        ok = mbar_try_wait(&empty[slot], (round - 1) & 1u);
                        if (!ok && (n & 255u) == 255u && *flag) break;
                    }
                    if (!ok) {
                        abort = true;
                        break;
                    }
                }
                if (*flag) {
                    abort = true;
                    break;
                }
                if (round > 0) fence_proxy_async();  // the consumers' reads of the slot before the new copies
                const int kw = kp < 0 ? kp + G.Z : (kp >= G.Z ? kp - G.Z : kp);
                uint64_t* bar = &full[slot];
                mbar_expect_tx(bar, (uint32_t)(Vt + 2) * (3u * xrow + mrow));
                float2* xs = sh.xslot_w(slot);
                unsigned char* ms = sh.mslot_w(slot);
                for (int c = 0; c < 3; ++c)
                    pipe_bulk_load(xs + ((int64_t)c * G.SR + s_lo) * G.X, x + c * cstr + ((int64_t)kw * G.Y + lo) * G.X,
                                   nr * xrow, bar);
                pipe_bulk_load(ms + (int64_t)s_lo * mrow, mat + ((int64_t)kw * G.Y + lo) * mrow, nr * mrow, bar);
                if (b0 == 0) {  // slot row 0 is row Y - 1
                    for (int c = 0; c < 3; ++c)
                        pipe_bulk_load(xs + (int64_t)c * G.SR * G.X, x + c * cstr + ((int64_t)kw * G.Y + G.Y - 1) * G.X,
                                       xrow, bar);
                    pipe_bulk_load(ms, mat + ((int64_t)kw * G.Y + G.Y - 1) * mrow, mrow, bar);
                }
                if (b0 + Vt == G.Y) {  // slot row Vt + 1 is row 0
                    const int sb = Vt + 1;
                    for (int c = 0; c < 3; ++c)
                        pipe_bulk_load(xs + ((int64_t)c * G.SR + sb) * G.X, x + c * cstr + (int64_t)kw * G.Y * G.X,
                                       xrow, bar);
                    pipe_bulk_load(ms + (int64_t)sb * mrow, mat + (int64_t)kw * G.Y * mrow, mrow, bar);
                }
            }
        }
        if (abort) {
            *flag = 1;
            atomicExch(B.err, 1);
            // let every copy still in flight land: the last plane issued into each slot
            for (int s = 0; s < NS; ++s) {
                if ((uint32_t)s >= q) break;
                const uint32_t last = q - 1 - ((q - 1 - (uint32_t)s) % (uint32_t)NS);
                for (uint32_t n = 0; n < kDrainLimit; ++n)
                    if (mbar_try_wait(&full[s], (last / (uint32_t)NS) & 1u)) break;
            }
        }
        return;
    }

    // ------------------------------------------------------------------ consumer warps
    typename T::Regs r;
    T::init(G, tid, r);
    const bool lane0 = (tid & 31) == 0;
    uint32_t q = 0;  // same plane sequence as the producer
    int cur_item = -1;
    bool ok = true;
    double* red = sh.red();

    auto wait_full = [&](uint32_t qq) {
        const int slot = (int)(qq % (uint32_t)NS);
        const uint32_t par = (qq / (uint32_t)NS) & 1u;
        if (*flag) {
            ok = false;
            return;
        }
        bool got = false;
        for (uint32_t n = 0; n < B.wait_limit && !got; ++n) got = mbar_try_wait(&full[slot], par);
        if (!got) {
            ok = false;
            *flag = 1;
        }
    };
    auto wait_full_at = [&](int slot, uint32_t par) {
        if (*flag) {
            ok = false;
            return;
        }
        bool got = false;
        for (uint32_t n = 0; n < B.wait_limit && !got; ++n) got = mbar_try_wait(&full[slot], par);
        if (!got) {
            ok = false;
            *flag = 1;
        }
    };
    auto release_at = [&](int slot) {
        __syncwarp();
        if (lane0) pipe_arrive(&empty[slot]);
    };
    auto flush_dot = [&]() {
        if (cur_item >= 0 && dot_partials != nullptr && B.it[cur_item].dot_slot >= 0) {
            double v = (double)r.dot;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane0) red[tid >> 5] = v;
            consumer_sync(NC);
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < NC / 32; ++w) s += red[w];
                dot_partials[(int64_t)B.it[cur_item].dot_slot * dot_stride + blockIdx.x] = s;
            }
            consumer_sync(NC);
        }
        r.dot = 0.f;
    };
    auto abort_exit = [&]() {
        if (tid == 0 && dot_partials != nullptr) {
            atomicExch(B.err, 1);
            for (int i = 0; i < B.n; ++i)
                if (B.it[i].dot_slot >= 0)
                    dot_partials[(int64_t)B.it[i].dot_slot * dot_stride + blockIdx.x] =
                        __longlong_as_double(0x7ff8000000000000LL);
        }
        if (tid == 0) atomicExch(B.err, 1);
    };

    for (int64_t u = u0; u < u1;) {
        int item, tile, ks, ke;
        pipe_seg_at(G, u, u1, item, tile, ks, ke);
        u += ke - ks;
        const ApplyItem& it = B.it[item];
        if (it.skip != nullptr && *it.skip) continue;
        if (item != cur_item) {
            flush_dot();
            cur_item = item;
        }
        PipeSeg S;
        S.b0 = pipe_tile_lo(G, tile);
        S.Vt = pipe_tile_lo(G, tile + 1) - S.b0;
        S.ks = ks;
        S.ke = ke;
        S.p12 = it.block >> 1;
        S.p13 = it.block & 1;
        S.x = static_cast<const float2*>(it.x);
        S.y = static_cast<float2*>(it.y);
        S.mat = B.mat_row[item];
        S.ph = B.ph[item];
        S.shift = (float)it.shift;
        S.top = S.b0 == 0;
        S.bot = S.b0 + S.Vt == G.Y;
        const bool want_dot = dot_partials != nullptr && it.dot_slot >= 0;
        T::seg_begin(r);
        // plane ks - 2 is sequence number q0; ring positions advance by one slot per plane (no
        // divisions inside the step loop)
        const uint32_t q0 = q;
        auto nxt = [&](int sl) { return sl + 1 == NS ? 0 : sl + 1; };
        const int s_first = (int)(q0 % (uint32_t)NS);
        wait_full(q0);
        wait_full(q0 + 1);
        int s_m = s_first;       // slot of plane kf - 1 (at step j = 0: plane ks - 2)
        int s_0 = nxt(s_m);      // plane kf
        int s_p = nxt(s_0);      // plane kf + 1
        uint32_t par_p = ((q0 + 2) / (uint32_t)NS) & 1u;  // phase parity of plane kf + 1's copy
        T::prologue(P, G, S, sh, r, s_m, s_0);
        const int nsteps = ke - ks + 2;  // flux planes ks - 1 .. ke
        for (int j = 0; j < nsteps; j += 2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (j + h >= nsteps) break;
                const int kf = ks - 1 + j + h;
                // plane kf - 1 lives on in registers (neighbour set); its slot is read again only by
                // the inner product of the gather
                if (!want_dot) release_at(s_m);
                wait_full_at(s_p, par_p);  // plane kf + 1
                const int buf = h;         // j is even: the step parity is h
                if (h == 0) T::template flux_step<0>(P, G, S, sh, r, kf, s_0, s_p, buf);
                else T::template flux_step<1>(P, G, S, sh, r, kf, s_0, s_p, buf);
                consumer_sync(NC);
                if (*flag) {
                    abort_exit();
                    return;
                }
                if (h == 0) T::template gather_step<0>(P, G, S, sh, r, kf, s_m, buf, want_dot);
                else T::template gather_step<1>(P, G, S, sh, r, kf, s_m, buf, want_dot);
                if (want_dot) release_at(s_m);  // plane kf - 1 is read for the last time
                s_m = s_0;
                s_0 = s_p;
                s_p = nxt(s_p);
                if (s_p == 0) par_p ^= 1u;
            }
        }
        release_at(s_m);  // plane ke
        release_at(s_0);  // plane ke + 1
        q = q0 + (uint32_t)(nsteps + 2);
    }
    if (!ok) {  // a failed wait after the last barrier of the launch
        abort_exit();
        return;
    }
    flush_dot();
}

// PC_PIPE_ARITH=scalar selects the scalar-FP32 form of the complex arithmetic (A/B comparisons).
inline bool pipe_packed() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("PC_PIPE_ARITH");
        v = (e && std::string(e) == "scalar") ? 0 : 1;
    }
    return v != 0;
}

template <bool CUBIC, int MATK, int XC, int TC, bool PK>
static int launch_pipe_pk(const StencilParams<float>& P, const ApplyItem* items, const double* iph,
                          const void* const* mats, int nitems, const PipeGeom& G, int ctas, double* dp, int ds,
                          int* err, cudaStream_t s) {
    auto kern = apply_pipe_kernel<CUBIC, MATK, XC, TC, PK>;
    const int smem = G.total;
    if (!pipe_geom_fits(G)) return fail(PC_EINVAL, "apply_pipe: shared memory layout exceeds 227 KB");
    if (XC > 0 && (G.X != XC || G.Y != XC || G.Z != 2 * XC || G.T != TC))
        return fail(PC_EINVAL, "apply_pipe: geometry mismatch");
    if (G.NC + 32 > kPipeMaxThreads || (G.X & 1)) return fail(PC_EINVAL, "apply_pipe: unsupported geometry");
    {
        // grids of different sizes may launch this kernel from several host threads at once
        static std::mutex mu;
        static int attr_bytes = 0;
        std::lock_guard<std::mutex> lk(mu);
        if (smem > attr_bytes) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(apply_pipe)");
            attr_bytes = smem;
        }
    }
    if (dp != nullptr && ctas > ds) return fail(PC_EINVAL, "apply: launch has more CTAs than partial-sum slots");
    for (int base = 0; base < nitems; base += kPipeMaxItems) {
        PipeBatch B;
        B.n = nitems - base < kPipeMaxItems ? nitems - base : kPipeMaxItems;
        B.err = err;
        B.wait_limit = wait_limit();
        for (int i = 0; i < B.n; ++i) {
            B.it[i] = items[base + i];
            B.mat_row[i] = mats[base + i];
            for (int l = 0; l < 3; ++l)
                B.ph[i][l] = make_float2((float)iph[(size_t)6 * (base + i) + 2 * l],
                                         (float)iph[(size_t)6 * (base + i) + 2 * l + 1]);
        }
        const int64_t W = (int64_t)B.n * G.nt * G.Z;
        kern<<<ctas, G.NC + 32, smem, s>>>(P, B, G, W, dp, ds);
        note_launch();
        note_apply_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "apply_pipe_kernel launch");
    }
    return PC_OK;
}

template <bool CUBIC, int MATK, int XC, int TC>
static int launch_pipe_t(const StencilParams<float>& P, const ApplyItem* items, const double* iph,
                         const void* const* mats, int nitems, const PipeGeom& G, int ctas, double* dp, int ds,
                         int* err, cudaStream_t s) {
    return pipe_packed()
               ? launch_pipe_pk<CUBIC, MATK, XC, TC, true>(P, items, iph, mats, nitems, G, ctas, dp, ds, err, s)
               : launch_pipe_pk<CUBIC, MATK, XC, TC, false>(P, items, iph, mats, nitems, G, ctas, dp, ds, err, s);
}

}  // namespace pc

namespace pc {
// Launchers of the compile-time-width kernels (cubic lattice, phase ids); nonzero return = error,
// *handled = false when the width is not one of them.
int launch_pipe_widths(int X, const StencilParams<float>& P, const ApplyItem* items, const double* iph,
                       const void* const* mats, int nitems, const PipeGeom& G, int ctas, double* dp, int ds, int* err,
                       cudaStream_t s, bool* handled);
}  // namespace pc
