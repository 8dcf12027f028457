// Allocation-free variant of the fused block apply with inner product.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: an application
// whose device memory is already handed out by its own pool (a framework's
// caching allocator sized to nearly all of the GPU), or a latency-sensitive
// loop for which the implicit device-wide synchronisation of cudaMalloc and
// cudaFree is not acceptable.  For them this entry point keeps its scratch -- the
// per-CTA partial sums of <x, y> -- in a fixed file-scope device array instead
// of allocated memory.
//
// The array lives in every GPU that loads the library, for the life of the
// process, and all calls on a device share it.  Each call overwrites exactly the
// partial slots it later reads, so nothing has to start at zero; but two calls
// whose kernels overlap on the GPU (different streams, no ordering) race on the
// same slots and may return wrong inner products.
#include <cuda_runtime.h>

#include <mutex>

#include "pc_internal.h"
#include "pc_solver.h"

namespace pc {

// Capacity: one double per CTA of the stencil launch.  Calls are limited to
// kNoAllocMaxNodes nodes, which keeps the launch far below this many CTAs.
constexpr int kNoAllocPartials = 2048;
constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 24;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

// Fixed-order sum of the partials (one CTA) into *out; NaN when a bounded copy wait of the
// apply expired (the grid's error word is set), so that the caller sees the failure in *dot.
__global__ void noalloc_reduce(int n, const int* __restrict__ err, double* __restrict__ out) {
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += g_noalloc_partials[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = (err != nullptr && *err != 0) ? __longlong_as_double(0x7ff8000000000000LL) : s;
    }
}

// Device address of the static array, looked up once per device with that device current.
static int noalloc_scratch(double** out) {
    static std::mutex mu;
    static void* addr[64] = {nullptr};
    int dev = 0;
    PC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        addr[dev] = p;
    }
    *out = static_cast<double*>(addr[dev]);
    return PC_OK;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_block_apply_dot_noalloc(pc_grid* g, int block, int dtype, const void* x, void* y, double shift,
                                          double* dot, void* stream) {
    if (!g || !x || !y || !dot) return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: null argument");
    if (block < -1 || block > 3) return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: block must be -1..3");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: bad dtype");
    if (x == y) return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: x and y must differ");
    if (!std::isfinite(shift)) return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: non-finite shift");
    if (!g->k.set) return fail(PC_ESTATE, "pc_block_apply_dot_noalloc: call pc_set_k first");
    const bool full = block < 0;
    const int64_t nodes = full ? g->n : g->nb;
    if (nodes > kNoAllocMaxNodes)
        return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: " + std::to_string(nodes) +
                                   " nodes exceed the static-scratch limit of " + std::to_string(kNoAllocMaxNodes));
    {
        const size_t vbytes = (size_t)3 * nodes * (dtype == PC_C64 ? 8 : 16);
        const char* xb = static_cast<const char*>(x);
        const char* yb = static_cast<const char*>(y);
        if (xb < yb + vbytes && yb < xb + vbytes)
            return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: x and y overlap");
    }
    const int X = full ? g->N : g->X, Y = full ? g->N : g->Y;
    ApplyConfig cfg = choose_apply_config(X, Y, g->Z, 1, dtype, false, 0,
                                          false /* no kernel that needs scratch of its own */);
    if (cfg.ctas > kNoAllocPartials) {
        // widest register-staged tiles with every plane of a column in one CTA: at most
        // ceil(X/32) ceil(Y/8) (complex64) or ceil(X/16) ceil(Y/8) (complex128) CTAs, which for
        // 2^24 nodes stays far below the partial-sum capacity
        cfg = ApplyConfig();
        cfg.shape = dtype == PC_C128 ? 1 : 0;
        cfg.tz = g->Z;
        cfg.ctas = ((X + tile_tx(cfg.shape) - 1) / tile_tx(cfg.shape)) * ((Y + tile_ty(cfg.shape) - 1) / tile_ty(cfg.shape));
    }
    if (cfg.ctas > kNoAllocPartials)
        return fail(PC_EINVAL, "pc_block_apply_dot_noalloc: launch needs " + std::to_string(cfg.ctas) +
                                   " partial sums, static scratch holds " + std::to_string(kNoAllocPartials));
    double* scratch = nullptr;
    PC_TRY(noalloc_scratch(&scratch));
    ApplyItem it;
    it.x = x;
    it.y = y;
    it.mat = grid_mat(g, block);
    it.shift = shift;
    it.block = block;
    it.dot_slot = 0;
    it.skip = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    PC_TRY(grid_apply(g, dtype, full, &it, 1, scratch, cfg.ctas, s, &cfg));
    noalloc_reduce<<<1, 256, 0, s>>>(cfg.ctas, g->d_err, dot);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}
