// Elementwise and layout kernels: nodewise mass, block <-> full transfer.
#include "pc_complex.cuh"
#include "pc_internal.h"

namespace pc {

// Full-grid index of position t of block b (canonical quarter-grid order; Sec. 4).
__host__ __device__ __forceinline__ int64_t block_to_full(int64_t t, int N, int b) {
    const int X = N / 2;
    const int64_t a = t % X, bb = (t / X) % X, k = t / ((int64_t)X * X);
    const int p12 = b >> 1, p13 = b & 1;
    const int64_t i = 2 * a + ((k + p13) & 1);
    const int64_t j = 2 * bb + ((k + p12 + p13) & 1);
    return i + (int64_t)N * (j + (int64_t)N * k);
}

// y = M x for ncomp consecutive component arrays of m nodes (3 per vector).
template <typename C, typename R>
__global__ void mass_kernel(const C* __restrict__ x, C* __restrict__ y, const void* __restrict__ mat,
                            int matkind, R rho0, R rho1, int64_t m, int ncomp) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += stride) {
        const R rho = node_rho_hat<R>(mat, matkind, rho0, rho1, m, t);
        for (int a = 0; a < ncomp; ++a) y[a * m + t] = cscale(rho, x[a * m + t]);
    }
}

template <typename C>
__global__ void transfer_kernel(const C* __restrict__ src, C* __restrict__ dst, int N, int b, int dir,
                                int64_t nb, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nb; t += stride) {
        const int64_t l = block_to_full(t, N, b);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (dir == 0) dst[a * nb + t] = src[a * n + l];
            else dst[a * n + l] = src[a * nb + t];
        }
    }
}

static int grid_for(int64_t m) {
    int64_t g = (m + 255) / 256;
    if (g > 16LL * device_sm_count()) g = 16LL * device_sm_count();
    if (g < 1) g = 1;
    return (int)g;
}

int launch_mass(int dtype, const void* x, void* y, const void* mat, int matkind, double rho0,
                double rho1, int64_t m, cudaStream_t s, int nvec) {
    if (dtype == PC_C64)
        { mass_kernel<float2, float><<<grid_for(m), 256, 0, s>>>((const float2*)x, (float2*)y, mat, matkind,
                                                              (float)rho0, (float)rho1, m, 3 * nvec); note_launch(); }
    else
        { mass_kernel<double2, double><<<grid_for(m), 256, 0, s>>>((const double2*)x, (double2*)y, mat,
                                                                matkind, rho0, rho1, m, 3 * nvec); note_launch(); }
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

int launch_transfer(int dtype, const void* src, void* dst, int N, int b, int dir, cudaStream_t s) {
    const int64_t n = (int64_t)N * N * N, nb = n / 4;
    if (dtype == PC_C64)
        { transfer_kernel<float2><<<grid_for(nb), 256, 0, s>>>((const float2*)src, (float2*)dst, N, b, dir, nb, n); note_launch(); }
    else
        { transfer_kernel<double2><<<grid_for(nb), 256, 0, s>>>((const double2*)src, (double2*)dst, N, b, dir, nb,
                                                             n); note_launch(); }
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

}  // namespace pc
