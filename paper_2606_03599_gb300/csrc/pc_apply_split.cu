// Two-pass stencil apply (see pc_apply_split.cuh): kernels and launchers.  Complex128 by default
// (bound by the FP64 pipe); complex64 as an autotuner candidate for grids whose fluxes stay in L2.
#include <algorithm>

#include "pc_apply_split.cuh"

namespace pc {

namespace {

constexpr int kSplitMaxItems = 64;
constexpr int kSplitThreads = 128;

template <typename R>
struct SplitBatch {
    using C = typename CT<R>::T;
    ApplyItem it[kSplitMaxItems];
    C* xg[kSplitMaxItems];  // ghost cells of x of each item
    C* fe[kSplitMaxItems];  // extended fluxes of each item
    R ph[kSplitMaxItems][3][2];  // (cos, sin) of each item's Bloch phases
    int n;
};

__device__ __forceinline__ bool item_skipped(const ApplyItem& it) { return it.skip != nullptr && *it.skip; }

// Pass 1: the ghost cells of x (all three components, the only FP64 work of the pass: the Bloch
// phase, computed once per cell); blockIdx.y = item.
template <typename R, bool FULL, bool CUBIC, int MATK>
__global__ void __launch_bounds__(kSplitThreads)
    split_fill_x(const __grid_constant__ StencilParams<R> P, const __grid_constant__ SplitBatch<R> B,
                 const __grid_constant__ SplitGeom G) {
    using T = SplitApply<R, FULL, CUBIC, MATK>;
    using C = typename CT<R>::T;
    const ApplyItem& it = B.it[blockIdx.y];
    if (item_skipped(it)) return;
    const C* x = static_cast<const C*>(it.x);
    for (int64_t gi = blockIdx.x * (int64_t)kSplitThreads + threadIdx.x; gi < G.ghosts;
         gi += (int64_t)gridDim.x * kSplitThreads)
        T::fill_x_ghost(B.ph[blockIdx.y], G, x, B.xg[blockIdx.y], gi);
}

// Pass 2: fluxes of every interior node; blockIdx.y = item.
template <typename R, bool FULL, bool CUBIC, int MATK>
__global__ void __launch_bounds__(kSplitThreads)
    split_flux(const __grid_constant__ StencilParams<R> P, const __grid_constant__ SplitBatch<R> B,
               const __grid_constant__ SplitGeom G) {
    using T = SplitApply<R, FULL, CUBIC, MATK>;
    __shared__ R Ct[2][36];
    for (int i = threadIdx.x; i < 72; i += kSplitThreads) Ct[i / 36][i % 36] = P.C[i / 36][i % 36];
    __syncthreads();
    const ApplyItem& it = B.it[blockIdx.y];
    if (item_skipped(it)) return;
    const int p12 = FULL ? 0 : (it.block >> 1), p13 = FULL ? 0 : (it.block & 1);
    for (int64_t t = blockIdx.x * (int64_t)kSplitThreads + threadIdx.x; t < G.m;
         t += (int64_t)gridDim.x * kSplitThreads)
        T::flux_node(P, Ct, G, p12, p13, static_cast<const typename CT<R>::T*>(it.x), B.xg[blockIdx.y], it.mat,
                     B.fe[blockIdx.y], t, true);
}

// Pass 3: ghost cells of F_0..F_3 (12 arrays per cell); blockIdx.y = item.
template <typename R, bool FULL, bool CUBIC, int MATK>
__global__ void __launch_bounds__(kSplitThreads)
    split_fill_f(const __grid_constant__ StencilParams<R> P, const __grid_constant__ SplitBatch<R> B,
                 const __grid_constant__ SplitGeom G) {
    using T = SplitApply<R, FULL, CUBIC, MATK>;
    const ApplyItem& it = B.it[blockIdx.y];
    if (item_skipped(it)) return;
    for (int64_t gi = blockIdx.x * (int64_t)kSplitThreads + threadIdx.x; gi < G.ghosts;
         gi += (int64_t)gridDim.x * kSplitThreads)
        T::fill_f_ghost(B.ph[blockIdx.y], G, B.fe[blockIdx.y], gi);
}

// Pass 4: outputs and optional Re<x, y> partials (one per CTA, fixed order); blockIdx.y = item.
template <typename R, bool FULL, bool CUBIC, int MATK>
__global__ void __launch_bounds__(kSplitThreads)
    split_gather(const __grid_constant__ StencilParams<R> P, const __grid_constant__ SplitBatch<R> B,
                 const __grid_constant__ SplitGeom G, double* __restrict__ dot_partials, int dot_stride) {
    using T = SplitApply<R, FULL, CUBIC, MATK>;
    using C = typename CT<R>::T;
    const ApplyItem& it = B.it[blockIdx.y];
    if (item_skipped(it)) return;
    const bool want_dot = dot_partials != nullptr && it.dot_slot >= 0;
    const int p12 = FULL ? 0 : (it.block >> 1), p13 = FULL ? 0 : (it.block & 1);
    double dot = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)kSplitThreads + threadIdx.x; t < G.m;
         t += (int64_t)gridDim.x * kSplitThreads)
        dot += (double)T::gather_node(P, G, p12, p13, B.fe[blockIdx.y], static_cast<const C*>(it.x),
                                      static_cast<C*>(it.y), it.mat, (R)it.shift, t, want_dot);
    if (want_dot) {
        __shared__ double red[kSplitThreads / 32];
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dot;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kSplitThreads / 32; ++w) s += red[w];
            dot_partials[(int64_t)it.dot_slot * dot_stride + blockIdx.x] = s;
        }
    }
}

template <typename R, bool FULL, bool CUBIC, int MATK>
int launch_split_t(const StencilParams<R>& P, const SplitBatch<R>& B, const SplitGeom& G, double* dp, int ds,
                   cudaStream_t s) {
    const int sm = device_sm_count();
    const int ngh = (int)std::max<int64_t>(1, std::min<int64_t>((G.ghosts + kSplitThreads - 1) / kSplitThreads, sm));
    split_fill_x<R, FULL, CUBIC, MATK><<<dim3(ngh, B.n), kSplitThreads, 0, s>>>(P, B, G);
    note_launch();
    const int nflux = split_apply_ctas(G.m);
    split_flux<R, FULL, CUBIC, MATK><<<dim3(nflux, B.n), kSplitThreads, 0, s>>>(P, B, G);
    note_launch();
    split_fill_f<R, FULL, CUBIC, MATK><<<dim3(ngh, B.n), kSplitThreads, 0, s>>>(P, B, G);
    note_launch();
    split_gather<R, FULL, CUBIC, MATK><<<dim3(nflux, B.n), kSplitThreads, 0, s>>>(P, B, G, dp, ds);
    note_launch();
    note_apply_launch();
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

}  // namespace

int split_apply_ctas(int64_t m) {
    // one node per thread up to eight CTAs of 128 threads per SM, grid-stride beyond
    return (int)std::max<int64_t>(1, std::min<int64_t>((m + kSplitThreads - 1) / kSplitThreads,
                                                       8LL * device_sm_count()));
}

size_t split_scratch_bytes(int X, int Y, int Z, int nitems, int dtype) {
    const SplitGeom G = make_split_geom(X, Y, Z);
    return (size_t)std::min(nitems, kSplitMaxItems) * split_item_elems(G) * (dtype == PC_C64 ? 8 : 16);
}

template <typename R>
static int launch_apply_split_t(bool full, bool cubic, int matkind, const StencilParams<R>& P, const ApplyItem* items,
                                const double* item_ph, int nitems, void* scratch, size_t scratch_bytes, double* dp, int ds, cudaStream_t s) {
    using C = typename CT<R>::T;
    const SplitGeom G = make_split_geom(P.X, P.Y, P.Z);
    const int64_t per = split_item_elems(G);
    if (dp != nullptr && split_apply_ctas(G.m) > ds)
        return fail(PC_EINVAL, "apply: launch has more CTAs than partial-sum slots");
    for (int base = 0; base < nitems; base += kSplitMaxItems) {
        SplitBatch<R> B;
        B.n = std::min(nitems - base, kSplitMaxItems);
        if ((size_t)B.n * per * sizeof(C) > scratch_bytes) return fail(PC_EINVAL, "apply: split scratch too small");
        for (int i = 0; i < B.n; ++i) {
            B.it[i] = items[base + i];
            for (int e = 0; e < 6; ++e) B.ph[i][e / 2][e % 2] = (R)item_ph[(size_t)6 * (base + i) + e];
            C* w = static_cast<C*>(scratch) + (int64_t)i * per;
            B.xg[i] = w;
            B.fe[i] = w + 3 * G.ghosts;
        }
        int rc;
        if (matkind == 2) {
            if constexpr (sizeof(R) == 8) {
                if (full) rc = cubic ? launch_split_t<R, true, true, 2>(P, B, G, dp, ds, s)
                                     : launch_split_t<R, true, false, 2>(P, B, G, dp, ds, s);
                else rc = cubic ? launch_split_t<R, false, true, 2>(P, B, G, dp, ds, s)
                                : launch_split_t<R, false, false, 2>(P, B, G, dp, ds, s);
            } else {
                rc = fail(PC_EINVAL, "apply: nodewise material needs complex128");
            }
        } else if (full) {
            if (cubic) rc = matkind ? launch_split_t<R, true, true, 1>(P, B, G, dp, ds, s) : launch_split_t<R, true, true, 0>(P, B, G, dp, ds, s);
            else rc = matkind ? launch_split_t<R, true, false, 1>(P, B, G, dp, ds, s) : launch_split_t<R, true, false, 0>(P, B, G, dp, ds, s);
        } else {
            if (cubic) rc = matkind ? launch_split_t<R, false, true, 1>(P, B, G, dp, ds, s) : launch_split_t<R, false, true, 0>(P, B, G, dp, ds, s);
            else rc = matkind ? launch_split_t<R, false, false, 1>(P, B, G, dp, ds, s) : launch_split_t<R, false, false, 0>(P, B, G, dp, ds, s);
        }
        PC_TRY(rc);
    }
    return PC_OK;
}

int launch_apply_split_f64(bool full, bool cubic, int matkind, const StencilParams<double>& P, const ApplyItem* items,
                           const double* item_ph, int nitems, void* scratch, size_t scratch_bytes, double* dp, int ds,
                           cudaStream_t s) {
    return launch_apply_split_t<double>(full, cubic, matkind, P, items, item_ph, nitems, scratch, scratch_bytes, dp, ds,
                                        s);
}

int launch_apply_split_f32(bool full, bool cubic, int matkind, const StencilParams<float>& P, const ApplyItem* items,
                           const double* item_ph, int nitems, void* scratch, size_t scratch_bytes, double* dp, int ds,
                           cudaStream_t s) {
    return launch_apply_split_t<float>(full, cubic, matkind, P, items, item_ph, nitems, scratch, scratch_bytes, dp, ds,
                                       s);
}

}  // namespace pc
