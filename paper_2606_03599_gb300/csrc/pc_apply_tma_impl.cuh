// CUDA kernel of the TMA-staged stencil apply and its host launcher.
// Included by one translation unit per precision.
#pragma once

#include <cudaTypedefs.h>

#include <mutex>
#include <unordered_map>

#include "pc_apply_tma.cuh"

namespace pc {

template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
__global__ void __launch_bounds__(TmaTile<R, FULL, CUBIC, MATK, TX, TY>::NT, 2)
    apply_tma_kernel(const __grid_constant__ StencilParams<R> P, const __grid_constant__ TmaBatch B, int ntx, int tz,
                     double* __restrict__ dot_partials, int dot_stride) {
    using T = TmaTile<R, FULL, CUBIC, MATK, TX, TY>;
    using C = typename CT<R>::T;
    extern __shared__ __align__(128) unsigned char smem_tma[];
    // TMA destinations must be 128-byte aligned: round the dynamic window up (128 spare bytes are allocated)
    unsigned char* smem_base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_tma) + 127) & ~static_cast<uintptr_t>(127));
    typename T::Shared& sh = *reinterpret_cast<typename T::Shared*>(smem_base);
    const ApplyItem& it = B.it[blockIdx.z];
    if (it.skip != nullptr && *it.skip) return;
    const CUtensorMap* map = &B.map[blockIdx.z];

    typename T::Ctx c;
    c.P = &P;
    c.x = static_cast<const C*>(it.x);
    c.y = static_cast<C*>(it.y);
    c.mat = it.mat;
    c.shift = (R)it.shift;
    c.a0 = (blockIdx.x % ntx) * TX;
    c.b0 = (blockIdx.x / ntx) * TY;
    c.k0 = blockIdx.y * tz;
    c.tz = min(tz, P.Z - c.k0);
    c.p12 = FULL ? 0 : (it.block >> 1);
    c.p13 = FULL ? 0 : (it.block & 1);
    c.plane = (int64_t)P.X * P.Y;
    c.vstr = c.plane * P.Z;
    const int tid = threadIdx.x;
    const int kfirst = c.k0 - 2, klast = c.k0 + c.tz + 1;
    constexpr uint32_t kBytes = 3u * T::XR * (uint32_t)sizeof(C);
    constexpr int kUnits = (int)sizeof(C) / 8;  // tensor elements are 8-byte units

    auto issue = [&](int kp) {
        const int j = kp - kfirst;
        uint64_t* bar = &sh.mbar[j % T::NSLOT];
        int wk;
        const int kw = T::wrapc(kp, P.Z, wk);
        mbar_expect_tx(bar, kBytes);
        tma_load_4d(sh.xs[j % T::NSLOT], map, bar, (c.a0 - 2) * kUnits, c.b0 - 2, kw, 0);
    };
    auto wait_n = [&](int kp, uint32_t limit) -> bool {
        const int j = kp - kfirst;
        uint64_t* bar = &sh.mbar[j % T::NSLOT];
        const uint32_t parity = (uint32_t)((j / T::NSLOT) & 1);
        for (uint32_t n = 0; n < limit; ++n)
            if (mbar_try_wait(bar, parity)) return true;
        return false;
    };
    auto wait = [&](int kp) -> bool { return wait_n(kp, B.wait_limit); };

    typename T::Regs r;
    if (tid == 0) {
        for (int s = 0; s < T::NSLOT; ++s) mbar_init(&sh.mbar[s], 1);
        sh.abort = 0;
        fence_mbar_init();
    }
    T::load_tables(c, sh, tid);
    T::init(c, sh, tid, r);
    __syncthreads();
    int last_issued = kfirst - 1;
    if (tid == 0) {
        for (int kp = kfirst; kp <= klast && kp < kfirst + T::NSLOT; ++kp) issue(kp);
    }
    last_issued = min(klast, kfirst + T::NSLOT - 1);

    // prologue: planes k0-2 and k0-1 ready (with wrap fix-ups), flux material of plane k0-1
    bool ok = true;
    for (int kp = kfirst; kp < c.k0; ++kp) {
        T::prefetch_fix(c, r, tid, kp);
        ok = wait(kp) && ok;
        T::apply_fix(c, sh, r, tid, kp);
    }
    T::prefetch_fix(c, r, tid, c.k0);
    {
        int wk;
        const int kw = T::wrapc(c.k0 - 1, P.Z, wk);
        r.fm_cur = r.fvalid ? T::read_mat(c.mat, (int64_t)kw * c.plane + r.foff) : (R)0;
    }
    for (int kf = c.k0 - 1; kf <= c.k0 + c.tz; ++kf) {
        const int p = kf + 1;
        ok = wait(p) && ok;
        T::apply_fix(c, sh, r, tid, p);
        if (p + 1 <= klast) T::prefetch_fix(c, r, tid, p + 1);
        T::load_mats(c, r, kf);
        if (!ok) sh.abort = 1;
        __syncthreads();
        if (sh.abort) {
            if (tid == 0) {
                atomicExch(B.err, 1);
                // this CTA's inner-product partial is void
                if (dot_partials != nullptr && it.dot_slot >= 0)
                    dot_partials[(int64_t)it.dot_slot * dot_stride + blockIdx.x + gridDim.x * blockIdx.y] =
                        __longlong_as_double(0x7ff8000000000000LL);
                // let the copies still in flight land before the CTA's shared memory is released
                for (int kp = p; kp <= last_issued; ++kp) wait_n(kp, kDrainLimit);
            }
            return;
        }
        if (tid == 0 && kf - 2 >= kfirst && kf - 2 + T::NSLOT <= klast) {
            fence_proxy_async();
            issue(kf - 2 + T::NSLOT);
        }
        last_issued = min(klast, max(last_issued, kf - 2 + T::NSLOT));
        T::flux(c, sh, r, kf);
        __syncthreads();
        T::gather(c, sh, r, kf);
        T::rotate_mats(r);
    }
    if (dot_partials != nullptr && it.dot_slot >= 0) {
        __shared__ double red[32];
        double v = (double)r.dot;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < T::NT / 32; ++w) s += red[w];
            dot_partials[(int64_t)it.dot_slot * dot_stride + blockIdx.x + gridDim.x * blockIdx.y] = s;
        }
    }
}

// ----------------------------------------------------------------------------- tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of a component-major vector [3][Z][Y][X] of `esize`-byte complex values,
// box (boxw x boxh x 1 plane x 3 components), cached by base address and shape.
static int tma_map(CUtensorMap* out, const void* base, int X, int Y, int Z, int esize, int boxw, int boxh) {
    struct Key {
        const void* p;
        int X, Y, Z, e, bw, bh;
        bool operator==(const Key& o) const {
            return p == o.p && X == o.X && Y == o.Y && Z == o.Z && e == o.e && bw == o.bw && bh == o.bh;
        }
    };
    struct Hash {
        size_t operator()(const Key& k) const {
            return std::hash<const void*>()(k.p) ^ ((size_t)k.X << 1) ^ ((size_t)k.Z << 21) ^ ((size_t)k.e << 40) ^
                   ((size_t)k.bw << 48);
        }
    };
    static std::mutex mu;
    static std::unordered_map<Key, CUtensorMap, Hash> cache;
    const Key key{base, X, Y, Z, esize, boxw, boxh};
    std::lock_guard<std::mutex> lk(mu);
    auto itc = cache.find(key);
    if (itc != cache.end()) {
        *out = itc->second;
        return PC_OK;
    }
    auto fn = tma_encode_fn();
    if (!fn) return fail(PC_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const int u = esize / 8;
    cuuint64_t dims[4] = {(cuuint64_t)X * u, (cuuint64_t)Y, (cuuint64_t)Z, 3};
    cuuint64_t strides[3] = {(cuuint64_t)X * esize, (cuuint64_t)X * Y * esize, (cuuint64_t)X * Y * Z * esize};
    cuuint32_t box[4] = {(cuuint32_t)(boxw * u), (cuuint32_t)boxh, 1, 3};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUtensorMap m;
    CUresult rc = fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) return fail(PC_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)rc) + ")");
    if (cache.size() > 4096) cache.clear();
    cache.emplace(key, m);
    *out = m;
    return PC_OK;
}

template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
static int launch_tma_tile(const StencilParams<R>& P, const ApplyItem* items, int nitems, int tz, double* dot_partials,
                           int dot_stride, int* err, cudaStream_t s) {
    using T = TmaTile<R, FULL, CUBIC, MATK, TX, TY>;
    auto kern = apply_tma_kernel<R, FULL, CUBIC, MATK, TX, TY>;
    const size_t smem = sizeof(typename T::Shared) + 128;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(apply_tma)");
        attr_set = true;
    }
    const int ntx = (P.X + TX - 1) / TX, nty = (P.Y + TY - 1) / TY;
    const int nch = (P.Z + tz - 1) / tz;
    if (dot_partials != nullptr && ntx * nty * nch > dot_stride)
        return fail(PC_EINVAL, "apply: launch has more CTAs than partial-sum slots");
    for (int base = 0; base < nitems; base += kTmaMaxItems) {
        TmaBatch B;
        B.n = nitems - base < kTmaMaxItems ? nitems - base : kTmaMaxItems;
        B.err = err;
        B.wait_limit = wait_limit();
        for (int i = 0; i < B.n; ++i) {
            B.it[i] = items[base + i];
            PC_TRY(tma_map(&B.map[i], items[base + i].x, P.X, P.Y, P.Z, (int)sizeof(typename CT<R>::T), T::XW,
                           T::XH));
        }
        dim3 grid(ntx * nty, nch, B.n);
        kern<<<grid, T::NT, smem, s>>>(P, B, ntx, tz, dot_partials, dot_stride);
        note_launch();
        note_apply_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "apply_tma_kernel launch");
    }
    return PC_OK;
}

// TMA tile codes: 0 = 16x16, 1 = 8x8 (complex64); 0 = 16x8, 1 = 8x8 (complex128).
template <typename R, bool FULL, bool CUBIC, int MATK>
static int launch_tma_shape(int shape, const StencilParams<R>& P, const ApplyItem* items, int nitems, int tz,
                            double* dp, int ds, int* err, cudaStream_t s) {
    constexpr bool F32 = sizeof(R) == 4;
    if (shape == 0) return launch_tma_tile<R, FULL, CUBIC, MATK, 16, (F32 ? 16 : 8)>(P, items, nitems, tz, dp, ds, err, s);
    return launch_tma_tile<R, FULL, CUBIC, MATK, 8, 8>(P, items, nitems, tz, dp, ds, err, s);
}

template <typename R>
static int launch_apply_tma_t(bool full, bool cubic, int matkind, int shape, const StencilParams<R>& P,
                              const ApplyItem* items, int nitems, int tz, double* dp, int ds, int* err,
                              cudaStream_t s) {
    if (full) {
        if (cubic) return matkind ? launch_tma_shape<R, true, true, 1>(shape, P, items, nitems, tz, dp, ds, err, s)
                                  : launch_tma_shape<R, true, true, 0>(shape, P, items, nitems, tz, dp, ds, err, s);
        return matkind ? launch_tma_shape<R, true, false, 1>(shape, P, items, nitems, tz, dp, ds, err, s)
                       : launch_tma_shape<R, true, false, 0>(shape, P, items, nitems, tz, dp, ds, err, s);
    }
    if (cubic) return matkind ? launch_tma_shape<R, false, true, 1>(shape, P, items, nitems, tz, dp, ds, err, s)
                              : launch_tma_shape<R, false, true, 0>(shape, P, items, nitems, tz, dp, ds, err, s);
    return matkind ? launch_tma_shape<R, false, false, 1>(shape, P, items, nitems, tz, dp, ds, err, s)
                   : launch_tma_shape<R, false, false, 0>(shape, P, items, nitems, tz, dp, ds, err, s);
}

}  // namespace pc
