// CUDA kernel of the row-tile stencil apply (complex64, parity blocks) and its
// host launcher.  Included by the complex64 translation unit.
#pragma once

#include <mutex>

#include "pc_apply_row.cuh"

namespace pc {

#if defined(__CUDACC__)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
#endif

template <bool CUBIC, int MATK, int XC>
__global__ void __launch_bounds__(kRowMaxThreads, 1)
    apply_row_kernel(const __grid_constant__ StencilParams<float> P, const __grid_constant__ RowBatch B,
                     const __grid_constant__ RowGeom G, int64_t W, double* __restrict__ dot_partials, int dot_stride) {
    using T = RowTile<CUBIC, MATK, XC>;
    extern __shared__ __align__(128) unsigned char smem_row[];
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_row) + 127) & ~static_cast<uintptr_t>(127));
    typename T::Sh sh{base, &G};
    const int tid = threadIdx.x;
    const uint32_t NS = (uint32_t)G.ns;
    uint64_t* bars = sh.bar();
    if (tid == 0) {
        for (uint32_t s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
        *sh.abort_flag() = 0;
        fence_mbar_init();
        if (dot_partials != nullptr)
            for (int i = 0; i < B.n; ++i)
                if (B.it[i].dot_slot >= 0) dot_partials[(int64_t)B.it[i].dot_slot * dot_stride + blockIdx.x] = 0.0;
    }
    T::load_tables(P, sh, tid, blockDim.x);
    typename T::Regs r;
    T::init(G, tid, r);
    __syncthreads();

    const int64_t u0 = (int64_t)blockIdx.x * W / gridDim.x, u1 = (int64_t)(blockIdx.x + 1) * W / gridDim.x;
    uint32_t gseq = 0;  // ring sequence number of the first plane of the current segment
    int cur_item = -1;
    __shared__ double red[kRowMaxThreads / 32];

    auto flush_dot = [&]() {
        if (cur_item >= 0 && dot_partials != nullptr && B.it[cur_item].dot_slot >= 0) {
            double v = (double)r.dot;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) red[tid >> 5] = v;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += red[w];
                dot_partials[(int64_t)B.it[cur_item].dot_slot * dot_stride + blockIdx.x] = s;
            }
            __syncthreads();
        }
        r.dot = 0.f;
    };

    for (int64_t u = u0; u < u1;) {
        int item, tile, ks, ke;
        row_seg_at(G, u, u1, item, tile, ks, ke);
        u += ke - ks;
        if (item != cur_item) {
            flush_dot();
            cur_item = item;
        }
        const ApplyItem& it = B.it[item];
        if (it.skip != nullptr && *it.skip) continue;
        RowSeg S;
        S.item = item;
        S.b0 = row_tile_lo(G, tile);
        S.V = row_tile_lo(G, tile + 1) - S.b0;
        S.ks = ks;
        S.ke = ke;
        S.p12 = it.block >> 1;
        S.p13 = it.block & 1;
        S.x = static_cast<const float2*>(it.x);
        S.y = static_cast<float2*>(it.y);
        S.mat = B.mat_row[item];
        S.shift = (float)it.shift;
        T::seg_begin(r);
        const int L = ke - ks + 4;  // planes ks - 2 .. ke + 1
        const int kfirst = ks - 2;
        const uint32_t rows = (uint32_t)S.V + 2;
        const uint32_t xrow = (uint32_t)G.X * 8u, mrow = (uint32_t)G.Xp * (uint32_t)G.matsz;
        const int64_t cstr = (int64_t)G.X * G.Y * G.Z;  // component stride (elements)

        auto issue = [&](int kp) {
            const uint32_t q = gseq + (uint32_t)(kp - kfirst);
            const int slot = (int)(q & (NS - 1));
            uint64_t* bar = &bars[slot];
            const int kw = kp < 0 ? kp + G.Z : (kp >= G.Z ? kp - G.Z : kp);
            mbar_expect_tx(bar, rows * (3u * xrow + mrow));
            float2* xs = sh.xslot(slot);
            unsigned char* ms = sh.mslot(slot);
            const char* mat = static_cast<const char*>(S.mat);
            const int lo = S.b0 - 1 < 0 ? 0 : S.b0 - 1;
            const int hi = S.b0 + S.V > G.Y - 1 ? G.Y - 1 : S.b0 + S.V;
            const int s_lo = lo - (S.b0 - 1);
            const uint32_t nr = (uint32_t)(hi - lo + 1);
            for (int c = 0; c < 3; ++c)
                bulk_load(xs + ((int64_t)c * G.SR + s_lo) * G.X, S.x + c * cstr + ((int64_t)kw * G.Y + lo) * G.X,
                          nr * xrow, bar);
            bulk_load(ms + (int64_t)s_lo * mrow, mat + ((int64_t)kw * G.Y + lo) * mrow, nr * mrow, bar);
            if (S.b0 == 0) {  // row -1 is row Y - 1 of the plane
                for (int c = 0; c < 3; ++c)
                    bulk_load(xs + (int64_t)c * G.SR * G.X, S.x + c * cstr + ((int64_t)kw * G.Y + G.Y - 1) * G.X,
                              xrow, bar);
                bulk_load(ms, mat + ((int64_t)kw * G.Y + G.Y - 1) * mrow, mrow, bar);
            }
            if (S.b0 + S.V == G.Y) {  // row Y is row 0 of the plane
                const int sb = S.V + 1;
                for (int c = 0; c < 3; ++c)
                    bulk_load(xs + ((int64_t)c * G.SR + sb) * G.X, S.x + c * cstr + (int64_t)kw * G.Y * G.X, xrow,
                              bar);
                bulk_load(ms + (int64_t)sb * mrow, mat + (int64_t)kw * G.Y * mrow, mrow, bar);
            }
        };
        auto wait_n = [&](int kp, uint32_t limit) -> bool {
            const uint32_t q = gseq + (uint32_t)(kp - kfirst);
            uint64_t* bar = &bars[q & (NS - 1)];
            const uint32_t parity = (q >> G.ns_log2) & 1u;
            for (uint32_t n = 0; n < limit; ++n)
                if (mbar_try_wait(bar, parity)) return true;
            return false;
        };
        auto wait = [&](int kp) -> bool { return wait_n(kp, B.wait_limit); };
        auto slot_of = [&](int kp) { return (int)((gseq + (uint32_t)(kp - kfirst)) & (NS - 1)); };

        if (tid == 0) {
            fence_proxy_async();  // earlier generic accesses of the slots come before the new copies
            for (int kp = kfirst; kp <= ke + 1 && kp < kfirst + (int)NS; ++kp) issue(kp);
        }
        int last_issued = min(ke + 1, kfirst + (int)NS - 1);
        // planes ks - 2, ks - 1, ks feed the first flux plane ks - 1
        bool ok = true;
        for (int kp = kfirst; kp <= ks; ++kp) {
            ok = ok && wait(kp);
            if (ok) T::fix_plane(P, G, S, sh, slot_of(kp), kp, tid);
        }
        // the fixed planes, and the end of the previous segment's last gather, before any flux
        __syncthreads();
        // One barrier per step: flux planes alternate between two shared buffers, so step kf
        // finishes y(kf - 2) from the buffer of plane kf - 1 while it writes the fluxes of plane kf.
        for (int kf = ks - 1; kf <= ke; ++kf) {
            if (kf > ks - 1) T::gather(P, G, S, sh, r, kf - 1, (kf - 1) & 1);
            if (ok) T::flux(P, G, S, sh, r, kf, slot_of(kf - 1), slot_of(kf), slot_of(kf + 1), kf & 1);
            if (kf + 2 <= ke + 1) {
                ok = ok && wait(kf + 2);
                if (ok) T::fix_plane(P, G, S, sh, slot_of(kf + 2), kf + 2, tid);
            }
            if (!ok) *sh.abort_flag() = 1;
            __syncthreads();
            if (*sh.abort_flag()) {
                if (tid == 0) {
                    atomicExch(B.err, 1);
                    // the inner products of this launch are void: NaN in every partial slot of this CTA
                    if (dot_partials != nullptr)
                        for (int i = 0; i < B.n; ++i)
                            if (B.it[i].dot_slot >= 0)
                                dot_partials[(int64_t)B.it[i].dot_slot * dot_stride + blockIdx.x] = __longlong_as_double(
                                    0x7ff8000000000000LL);
                    // let the copies still in flight land before the CTA's shared memory is released
                    for (int kp = max(kfirst, kf - 1); kp <= last_issued; ++kp) wait_n(kp, kDrainLimit);
                }
                return;
            }
            // the slot of plane kf - 1 is free once every thread has finished flux(kf)
            if (kf - 1 >= kfirst && kf - 1 + (int)NS <= ke + 1) {
                if (tid == 0) {
                    fence_proxy_async();
                    issue(kf - 1 + (int)NS);
                }
                last_issued = kf - 1 + (int)NS;
            }
        }
        T::gather(P, G, S, sh, r, ke, ke & 1);
        gseq += (uint32_t)L;
    }
    flush_dot();
}

template <bool CUBIC, int MATK, int XC>
static int launch_row_t(const StencilParams<float>& P, const ApplyItem* items, const void* const* mats, int nitems,
                        const RowGeom& G, int ctas, double* dp, int ds, int* err, cudaStream_t s) {
    auto kern = apply_row_kernel<CUBIC, MATK, XC>;
    const int smem = G.total + 128;  // + alignment slack of the dynamic window
    if (smem + 1024 > 227 * 1024) return fail(PC_EINVAL, "apply_row: shared memory layout exceeds 227 KB");
    {
        // grids of different sizes may launch this kernel from several host threads at once
        static std::mutex mu;
        static int attr_bytes = 0;  // largest dynamic size granted so far
        std::lock_guard<std::mutex> lk(mu);
        if (smem > attr_bytes) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(apply_row)");
            attr_bytes = smem;
        }
    }
    if (G.NT > kRowMaxThreads) return fail(PC_EINVAL, "apply_row: too many threads per CTA");
    if (dp != nullptr && ctas > ds) return fail(PC_EINVAL, "apply: launch has more CTAs than partial-sum slots");
    for (int base = 0; base < nitems; base += kRowMaxItems) {
        RowBatch B;
        B.n = nitems - base < kRowMaxItems ? nitems - base : kRowMaxItems;
        B.err = err;
        B.wait_limit = wait_limit();
        for (int i = 0; i < B.n; ++i) {
            B.it[i] = items[base + i];
            B.mat_row[i] = mats[base + i];
        }
        const int64_t W = (int64_t)B.n * G.nt * G.Z;
        kern<<<ctas, G.NT, smem, s>>>(P, B, G, W, dp, ds);
        note_launch();
        note_apply_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "apply_row_kernel launch");
    }
    return PC_OK;
}

// Launchers of the compile-time-width kernels (cubic lattice, phase ids), one translation unit
// per group of widths; nonzero return = width not handled there.
int launch_row_narrow(int X, const StencilParams<float>& P, const ApplyItem* items, const void* const* mats,
                      int nitems, const RowGeom& G, int ctas, double* dp, int ds, int* err, cudaStream_t s,
                      bool* handled);
int launch_row_wide(int X, const StencilParams<float>& P, const ApplyItem* items, const void* const* mats,
                    int nitems, const RowGeom& G, int ctas, double* dp, int ds, int* err, cudaStream_t s,
                    bool* handled);

}  // namespace pc
