// CUDA kernel of the fused stencil apply and its dispatch over compile-time
// tile shapes.  Included by one translation unit per precision.
#pragma once

#include "pc_apply_tile.cuh"

namespace pc {

constexpr int kMaxBatchItems = 64;

struct ApplyBatch {
    ApplyItem it[kMaxBatchItems];
    int n;
};

template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
    apply_kernel(const __grid_constant__ StencilParams<R> P, const __grid_constant__ ApplyBatch B,
                 int ntx, int tz, double* __restrict__ dot_partials, int dot_stride) {
    using T = ApplyTile<R, FULL, CUBIC, MATK, TX, TY>;
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::Shared& sh = *reinterpret_cast<typename T::Shared*>(smem_raw);
    const ApplyItem& it = B.it[blockIdx.z];
    if (it.skip != nullptr && *it.skip) return;

    typename T::Ctx c;
    c.P = &P;
    c.x = static_cast<const C*>(it.x);
    c.y = static_cast<C*>(it.y);
    c.mat = it.mat;
    c.shift = (R)it.shift;
    c.dot = dot_partials != nullptr && it.dot_slot >= 0;
    c.a0 = (blockIdx.x % ntx) * TX;
    c.b0 = (blockIdx.x / ntx) * TY;
    c.k0 = blockIdx.y * tz;
    c.tz = min(tz, P.Z - c.k0);
    c.p12 = FULL ? 0 : (it.block >> 1);
    c.p13 = FULL ? 0 : (it.block & 1);
    c.plane = (int64_t)P.X * P.Y;
    c.vstr = c.plane * P.Z;

    typename T::Regs r;
    const int tid = threadIdx.x;
    T::load_tables(c, sh, tid);
    T::init(c, tid, r);
    T::prologue_load(c, sh, r, tid);
    __syncthreads();
    for (int kf = c.k0 - 1; kf <= c.k0 + c.tz; ++kf) {
        T::phaseA(c, sh, r, tid, kf);
        __syncthreads();
        T::phaseB(c, sh, r, kf);
        __syncthreads();
    }
    if (dot_partials != nullptr && it.dot_slot >= 0) {
        __shared__ double red[32];
        double v = (double)r.dot;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < (T::NT + 31) / 32; ++w) s += red[w];
            dot_partials[(int64_t)it.dot_slot * dot_stride + blockIdx.x + gridDim.x * blockIdx.y] = s;
        }
    }
}

template <typename R, bool FULL, bool CUBIC, int MATK, int TX, int TY>
static int launch_tile(const StencilParams<R>& P, const ApplyItem* items, int nitems, int tz,
                       double* dot_partials, int dot_stride, cudaStream_t s) {
    using T = ApplyTile<R, FULL, CUBIC, MATK, TX, TY>;
    auto kern = apply_kernel<R, FULL, CUBIC, MATK, TX, TY>;
    const size_t smem = sizeof(typename T::Shared);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(apply)");
        attr_set = true;
    }
    const int ntx = (P.X + TX - 1) / TX, nty = (P.Y + TY - 1) / TY;
    const int nch = (P.Z + tz - 1) / tz;
    if (dot_partials != nullptr && ntx * nty * nch > dot_stride)
        return fail(PC_EINVAL, "apply: launch has more CTAs than partial-sum slots");
    for (int base = 0; base < nitems; base += kMaxBatchItems) {
        ApplyBatch B;
        B.n = nitems - base < kMaxBatchItems ? nitems - base : kMaxBatchItems;
        for (int i = 0; i < B.n; ++i) B.it[i] = items[base + i];
        dim3 grid(ntx * nty, nch, B.n);
        kern<<<grid, T::NT, smem, s>>>(P, B, ntx, tz, dot_partials, dot_stride);
        note_launch();
        note_apply_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "apply_kernel launch");
    }
    return PC_OK;
}

// Tile shape codes: 0 = 32x8, 1 = 16x8, 2 = 8x8, 3 = 4x4.
template <typename R, bool FULL, bool CUBIC, int MATK>
static int launch_shape(int shape, const StencilParams<R>& P, const ApplyItem* items, int nitems,
                        int tz, double* dp, int ds, cudaStream_t s) {
    switch (shape) {
        case 0: return launch_tile<R, FULL, CUBIC, MATK, 32, 8>(P, items, nitems, tz, dp, ds, s);
        case 1: return launch_tile<R, FULL, CUBIC, MATK, 16, 8>(P, items, nitems, tz, dp, ds, s);
        case 2: return launch_tile<R, FULL, CUBIC, MATK, 8, 8>(P, items, nitems, tz, dp, ds, s);
        default: return launch_tile<R, FULL, CUBIC, MATK, 4, 4>(P, items, nitems, tz, dp, ds, s);
    }
}

template <typename R>
static int launch_apply_t(bool full, bool cubic, int matkind, int shape, const StencilParams<R>& P,
                          const ApplyItem* items, int nitems, int tz, double* dp, int ds,
                          cudaStream_t s) {
    if (full) {
        if (cubic) return matkind ? launch_shape<R, true, true, 1>(shape, P, items, nitems, tz, dp, ds, s)
                                  : launch_shape<R, true, true, 0>(shape, P, items, nitems, tz, dp, ds, s);
        return matkind ? launch_shape<R, true, false, 1>(shape, P, items, nitems, tz, dp, ds, s)
                       : launch_shape<R, true, false, 0>(shape, P, items, nitems, tz, dp, ds, s);
    }
    if (cubic) return matkind ? launch_shape<R, false, true, 1>(shape, P, items, nitems, tz, dp, ds, s)
                              : launch_shape<R, false, true, 0>(shape, P, items, nitems, tz, dp, ds, s);
    return matkind ? launch_shape<R, false, false, 1>(shape, P, items, nitems, tz, dp, ds, s)
                   : launch_shape<R, false, false, 0>(shape, P, items, nitems, tz, dp, ds, s);
}

}  // namespace pc
