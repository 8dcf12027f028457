// Tall-skinny complex128 products of the outer Krylov-Schur loop: the Gram blocks V^H M W of
// block classical Gram-Schmidt and Cholesky QR (M = the nodal mass, Eq. discrete_GEP_main),
// and the basis updates W <- beta W + alpha V h of the same steps, of the Ritz vectors and of
// the restarts.
//
// The shapes are a few to a few dozen columns of length 3 n_b (83k at N = 48, 3.1M at N = 160),
// so the work is a sum over a long index with a small dense result.  On GB300 these products are
// bound by the FP64 pipe (two FP64 lanes per cycle per SM, the same rate for FP64 tensor
// instructions), not by memory: 4 FMAs per complex multiply-add against 32 bytes of operands.
// The kernels therefore keep every FP64 instruction useful: each thread owns a strip of the
// long index and a register block of the result (RB rows x CB columns of the Gram block, CB
// columns of an update), operands are read once per register block with coalesced 16-byte
// loads, the mass weight is applied once per element of W (not per product), and Gram partial
// sums are reduced in a fixed order (per CTA, then across CTAs) so results are deterministic.
#include <algorithm>

#include "pc_solver.h"

namespace pc {

namespace {

constexpr int kGramThreads = 256;
constexpr int kGramCB = 2;  // columns of W per register block

template <int MATK>
__device__ __forceinline__ double node_weight(const void* __restrict__ mat, int64_t t, int64_t m, double rho0,
                                              double drho) {
    if (MATK == 0) return rho0 + drho * (double)static_cast<const uint8_t*>(mat)[t];
    if (MATK == 1) return rho0 + drho * (double)static_cast<const float*>(mat)[t];
    if (MATK == 2) return static_cast<const double*>(mat)[21 * m + t];
    return 1.0;
}

// Partial sums of out(i, j) = sum_e conj(A[i][e]) w(e) B[j][e] over the nodes [t0, t1) of chunk
// blockIdx.x (all three components), for rows i0 .. i0 + RB - 1 and columns j0 .. j0 + CB - 1.
// MATK: -1 = no weight, 0 = phase ids, 1 = inclusion fractions, 2 = nodewise material.
template <int RB, int MATK>
__global__ void __launch_bounds__(kGramThreads)
    ts_gram_kernel(const double2* __restrict__ A, int rows, const double2* __restrict__ B, int cols, int64_t m,
                   const void* __restrict__ mat, double rho0, double drho, int ngc, int nchunk,
                   double* __restrict__ part) {
    constexpr int CB = kGramCB;
    const int rg = blockIdx.y / ngc, cg = blockIdx.y % ngc;
    const int i0 = rg * RB, j0 = cg * CB;
    const int64_t vs = 3 * m;
    const int64_t t0 = (int64_t)blockIdx.x * m / nchunk, t1 = (int64_t)(blockIdx.x + 1) * m / nchunk;
    double ar[RB][CB], ai[RB][CB];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < CB; ++j) ar[i][j] = ai[i][j] = 0.0;
    for (int64_t t = t0 + threadIdx.x; t < t1; t += kGramThreads) {
        const double w = node_weight<MATK>(mat, t, m, rho0, drho);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t e = c * m + t;
            double2 b[CB];
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                b[j] = (j0 + j < cols) ? B[(int64_t)(j0 + j) * vs + e] : make_double2(0.0, 0.0);
                if (MATK >= 0) b[j] = make_double2(w * b[j].x, w * b[j].y);
            }
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                if (i0 + i < rows) {
                    const double2 a = A[(int64_t)(i0 + i) * vs + e];
#pragma unroll
                    for (int j = 0; j < CB; ++j) {  // conj(a) b
                        ar[i][j] = fma(a.x, b[j].x, fma(a.y, b[j].y, ar[i][j]));
                        ai[i][j] = fma(a.x, b[j].y, fma(-a.y, b[j].x, ai[i][j]));
                    }
                }
            }
        }
    }
    // CTA reduction in a fixed order: warp shuffles, then the warps' sums in warp order
    constexpr int NV = RB * CB * 2;
    __shared__ double red[kGramThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            double vr = ar[i][j], vi = ai[i][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vr += __shfl_down_sync(0xffffffffu, vr, o);
                vi += __shfl_down_sync(0xffffffffu, vi, o);
            }
            if (lane == 0) {
                red[warp][(i * CB + j) * 2 + 0] = vr;
                red[warp][(i * CB + j) * 2 + 1] = vi;
            }
        }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int v = threadIdx.x, ij = v >> 1, ri = v & 1;
        const int gi = i0 + ij / CB, gj = j0 + ij % CB;
        if (gi < rows && gj < cols) {
            double s = 0.0;
            for (int q = 0; q < kGramThreads / 32; ++q) s += red[q][v];
            part[((int64_t)(gi + gj * rows) * 2 + ri) * nchunk + blockIdx.x] = s;
        }
    }
}

// out[e] = sum over chunks of part[e][chunk]: one warp per entry, lane l sums the chunks
// l, l + 32, ... in order, then the lanes' sums are combined by a fixed shuffle tree
// (deterministic for a given chunk count).
__global__ void ts_gram_reduce(const double* __restrict__ part, int nentries, int nchunk, double2* __restrict__ out) {
    const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= nentries) return;
    double re = 0.0, im = 0.0;
    for (int c = lane; c < nchunk; c += 32) {
        re += part[((int64_t)e * 2 + 0) * nchunk + c];
        im += part[((int64_t)e * 2 + 1) * nchunk + c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) out[e] = make_double2(re, im);
}

// C[:, j] = beta C[:, j] + alpha sum_k A[:, k] h(k, j) for the CB columns j0 .. j0 + CB - 1 of
// column group blockIdx.y; h (k x cols, column-major) is staged in shared memory.  With
// beta == 0, C is not read (it may hold anything).
template <int CB>
__global__ void __launch_bounds__(256)
    ts_update_kernel(const double2* __restrict__ A, int k, const double2* __restrict__ h, int cols,
                     double2* __restrict__ C, int64_t vs, double alpha, double beta) {
    extern __shared__ double2 hs[];  // [k][CB]
    const int j0 = blockIdx.y * CB;
    for (int q = threadIdx.x; q < k * CB; q += blockDim.x) {
        const int kk = q / CB, j = q % CB;
        hs[q] = (j0 + j < cols) ? h[kk + (int64_t)(j0 + j) * k] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        double cr[CB], ci[CB];
#pragma unroll
        for (int j = 0; j < CB; ++j) cr[j] = ci[j] = 0.0;
        for (int kk = 0; kk < k; ++kk) {
            const double2 a = A[(int64_t)kk * vs + e];
#pragma unroll
            for (int j = 0; j < CB; ++j) {  // a h
                const double2 hv = hs[kk * CB + j];
                cr[j] = fma(a.x, hv.x, fma(-a.y, hv.y, cr[j]));
                ci[j] = fma(a.x, hv.y, fma(a.y, hv.x, ci[j]));
            }
        }
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            if (j0 + j >= cols) continue;
            double2* cp = C + (int64_t)(j0 + j) * vs + e;
            double2 o = make_double2(alpha * cr[j], alpha * ci[j]);
            if (beta != 0.0) {
                const double2 cv = *cp;
                o.x = fma(beta, cv.x, o.x);
                o.y = fma(beta, cv.y, o.y);
            }
            *cp = o;
        }
    }
}

template <int RB>
int launch_gram_rb(const double2* A, int rows, const double2* B, int cols, int64_t m, const void* mat, int matkind,
                   double rho0, double drho, int ngc, int nrg, int nchunk, double* part, cudaStream_t s) {
    const dim3 grid(nchunk, nrg * ngc);
    if (mat == nullptr)
        ts_gram_kernel<RB, -1><<<grid, kGramThreads, 0, s>>>(A, rows, B, cols, m, mat, rho0, drho, ngc, nchunk, part);
    else if (matkind == 0)
        ts_gram_kernel<RB, 0><<<grid, kGramThreads, 0, s>>>(A, rows, B, cols, m, mat, rho0, drho, ngc, nchunk, part);
    else if (matkind == 2)
        ts_gram_kernel<RB, 2><<<grid, kGramThreads, 0, s>>>(A, rows, B, cols, m, mat, rho0, drho, ngc, nchunk, part);
    else
        ts_gram_kernel<RB, 1><<<grid, kGramThreads, 0, s>>>(A, rows, B, cols, m, mat, rho0, drho, ngc, nchunk, part);
    note_launch();
    return PC_OK;
}

// ---------------------------------------------------------------- batched forms (several spaces)
// The outer loop runs the same product for every active space of a solve (the four parity blocks
// times the Bloch vectors solved together); one launch serves them all, job j in blockIdx.z.
constexpr int kMaxJobs = 64;

struct GramBatch {
    GramJob j[kMaxJobs];
    int64_t off[kMaxJobs + 1];  // prefix sums of the jobs' result entries
    int n;
};

template <int RB, int MATK>
__global__ void __launch_bounds__(kGramThreads)
    ts_gram_batch_kernel(const __grid_constant__ GramBatch B, int64_t m, double rho0, double drho, int ngc,
                         int nchunk, double* __restrict__ part) {
    constexpr int CB = kGramCB;
    const GramJob& J = B.j[blockIdx.z];
    const int rows = J.rows, cols = J.cols;
    const int rg = blockIdx.y / ngc, cg = blockIdx.y % ngc;
    const int i0 = rg * RB, j0 = cg * CB;
    if (i0 >= rows || j0 >= cols) return;  // this job has fewer register blocks than the launch
    const double2* __restrict__ A = J.A;
    const double2* __restrict__ Bm = J.B;
    const void* __restrict__ mat = J.mat;
    const int64_t vs = 3 * m;
    const int64_t t0 = (int64_t)blockIdx.x * m / nchunk, t1 = (int64_t)(blockIdx.x + 1) * m / nchunk;
    double ar[RB][CB], ai[RB][CB];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < CB; ++j) ar[i][j] = ai[i][j] = 0.0;
    for (int64_t t = t0 + threadIdx.x; t < t1; t += kGramThreads) {
        const double w = node_weight<MATK>(mat, t, m, rho0, drho);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t e = c * m + t;
            double2 b[CB];
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                b[j] = (j0 + j < cols) ? Bm[(int64_t)(j0 + j) * vs + e] : make_double2(0.0, 0.0);
                if (MATK >= 0) b[j] = make_double2(w * b[j].x, w * b[j].y);
            }
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                if (i0 + i < rows) {
                    const double2 a = A[(int64_t)(i0 + i) * vs + e];
#pragma unroll
                    for (int j = 0; j < CB; ++j) {  // conj(a) b
                        ar[i][j] = fma(a.x, b[j].x, fma(a.y, b[j].y, ar[i][j]));
                        ai[i][j] = fma(a.x, b[j].y, fma(-a.y, b[j].x, ai[i][j]));
                    }
                }
            }
        }
    }
    constexpr int NV = RB * CB * 2;
    __shared__ double red[kGramThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            double vr = ar[i][j], vi = ai[i][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vr += __shfl_down_sync(0xffffffffu, vr, o);
                vi += __shfl_down_sync(0xffffffffu, vi, o);
            }
            if (lane == 0) {
                red[warp][(i * CB + j) * 2 + 0] = vr;
                red[warp][(i * CB + j) * 2 + 1] = vi;
            }
        }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int v = threadIdx.x, ij = v >> 1, ri = v & 1;
        const int gi = i0 + ij / CB, gj = j0 + ij % CB;
        if (gi < rows && gj < cols) {
            double s = 0.0;
            for (int q = 0; q < kGramThreads / 32; ++q) s += red[q][v];
            part[((B.off[blockIdx.z] + gi + (int64_t)gj * rows) * 2 + ri) * nchunk + blockIdx.x] = s;
        }
    }
}

// Entry e of the concatenated results (job order) = fixed-order sum of its chunk partials.
__global__ void ts_gram_batch_reduce(const __grid_constant__ GramBatch B, const double* __restrict__ part,
                                     int nchunk) {
    const int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= B.off[B.n]) return;
    double re = 0.0, im = 0.0;
    for (int c = lane; c < nchunk; c += 32) {
        re += part[(e * 2 + 0) * nchunk + c];
        im += part[(e * 2 + 1) * nchunk + c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
        int j = 0;
        while (e >= B.off[j + 1]) ++j;
        B.j[j].out[e - B.off[j]] = make_double2(re, im);
    }
}

struct UpdateBatch {
    UpdateJob j[kMaxJobs];
    int n;
};

template <int CB>
__global__ void __launch_bounds__(256)
    ts_update_batch_kernel(const __grid_constant__ UpdateBatch U, int64_t vs) {
    extern __shared__ double2 hs[];  // [k][CB]
    const UpdateJob& J = U.j[blockIdx.z];
    const int k = J.k, cols = J.cols;
    const int j0 = blockIdx.y * CB;
    if (j0 >= cols) return;
    const double2* __restrict__ h = J.h;
    for (int q = threadIdx.x; q < k * CB; q += blockDim.x) {
        const int kk = q / CB, j = q % CB;
        hs[q] = (j0 + j < cols) ? h[kk + (int64_t)(j0 + j) * k] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const double2* __restrict__ A = J.A;
    double2* __restrict__ C = J.C;
    const double alpha = J.alpha, beta = J.beta;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        double cr[CB], ci[CB];
#pragma unroll
        for (int j = 0; j < CB; ++j) cr[j] = ci[j] = 0.0;
        for (int kk = 0; kk < k; ++kk) {
            const double2 a = A[(int64_t)kk * vs + e];
#pragma unroll
            for (int j = 0; j < CB; ++j) {
                const double2 hv = hs[kk * CB + j];
                cr[j] = fma(a.x, hv.x, fma(-a.y, hv.y, cr[j]));
                ci[j] = fma(a.x, hv.y, fma(a.y, hv.x, ci[j]));
            }
        }
#pragma unroll
        for (int j = 0; j < CB; ++j) {
            if (j0 + j >= cols) continue;
            double2* cp = C + (int64_t)(j0 + j) * vs + e;
            double2 o = make_double2(alpha * cr[j], alpha * ci[j]);
            if (beta != 0.0) {
                const double2 cv = *cp;
                o.x = fma(beta, cv.x, o.x);
                o.y = fma(beta, cv.y, o.y);
            }
            *cp = o;
        }
    }
}

}  // namespace

int ts_gram(const double2* A, int rows, const double2* B, int cols, int64_t m, const void* mat, int matkind,
            double rho0, double rho1, double2* d_out, double* d_part, size_t part_cap, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return PC_OK;
    if (!A || !B || !d_out || !d_part || m <= 0) return fail(PC_EINVAL, "ts_gram: bad argument");
    const int RB = rows <= 2 ? 2 : (rows <= 4 ? 4 : 8);
    const int nrg = (rows + RB - 1) / RB, ngc = (cols + kGramCB - 1) / kGramCB;
    // chunks of the node range: about two CTAs per SM over all register blocks, at least 512
    // nodes (two per thread) per chunk so that the per-CTA reduction stays small next to the
    // products, and as many partials as the scratch holds
    const int64_t entries = (int64_t)rows * cols;
    int64_t nchunk = (2LL * device_sm_count() + nrg * ngc - 1) / (nrg * ngc);
    nchunk = std::min<int64_t>(nchunk, std::max<int64_t>(1, m / 512));
    nchunk = std::min<int64_t>(nchunk, (int64_t)(part_cap / (2 * entries)));
    if (nchunk < 1) return fail(PC_EINVAL, "ts_gram: partial-sum scratch too small");
    const double drho = rho1 - rho0;
    if (RB == 2)
        launch_gram_rb<2>(A, rows, B, cols, m, mat, matkind, rho0, drho, ngc, nrg, (int)nchunk, d_part, s);
    else if (RB == 4)
        launch_gram_rb<4>(A, rows, B, cols, m, mat, matkind, rho0, drho, ngc, nrg, (int)nchunk, d_part, s);
    else
        launch_gram_rb<8>(A, rows, B, cols, m, mat, matkind, rho0, drho, ngc, nrg, (int)nchunk, d_part, s);
    ts_gram_reduce<<<(int)((entries + 7) / 8), 256, 0, s>>>(d_part, (int)entries, (int)nchunk, d_out);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

int ts_update(const double2* A, int k, const double2* d_h, int cols, double2* C, int64_t vs, double alpha,
              double beta, cudaStream_t s) {
    if (cols <= 0) return PC_OK;
    if (!C || vs <= 0) return fail(PC_EINVAL, "ts_update: bad argument");
    if (k <= 0) {  // empty product: C <- beta C
        if (beta == 1.0) return PC_OK;
        if (beta == 0.0) {
            for (int j = 0; j < cols; ++j)
                PC_CUDA_TRY(cudaMemsetAsync(C + (int64_t)j * vs, 0, sizeof(double2) * vs, s));
            return PC_OK;
        }
        return fail(PC_EINVAL, "ts_update: empty product with beta other than 0 or 1");
    }
    if (!A || !d_h) return fail(PC_EINVAL, "ts_update: bad argument");
    // column blocks of 2 when cols <= 2 (the Gram-Schmidt updates of a 2-wide Krylov block:
    // no FMAs on padding columns), else of 4
    const int CB = cols <= 2 ? 2 : 4;
    const size_t smem = sizeof(double2) * (size_t)k * CB;
    if (smem > 48 * 1024) return fail(PC_EINVAL, "ts_update: too many basis columns");
    const int ngc = (cols + CB - 1) / CB;
    int64_t gx = (vs + 255) / 256;
    gx = std::min<int64_t>(gx, std::max<int64_t>(1, 8LL * device_sm_count() / ngc));
    if (CB == 2)
        ts_update_kernel<2><<<dim3((unsigned)gx, ngc), 256, smem, s>>>(A, k, d_h, cols, C, vs, alpha, beta);
    else
        ts_update_kernel<4><<<dim3((unsigned)gx, ngc), 256, smem, s>>>(A, k, d_h, cols, C, vs, alpha, beta);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

int ts_gram_batch(const GramJob* jobs, int njobs, int64_t m, int matkind, double rho0, double rho1, double* d_part,
                  size_t part_cap, cudaStream_t s) {
    for (int base = 0; base < njobs; base += kMaxJobs) {
        GramBatch B;
        B.n = 0;
        B.off[0] = 0;
        int maxr = 0, maxc = 0;
        bool weighted = false;
        for (int i = base; i < njobs && B.n < kMaxJobs; ++i) {
            const GramJob& J = jobs[i];
            if (J.rows <= 0 || J.cols <= 0) continue;
            if (!J.A || !J.B || !J.out) return fail(PC_EINVAL, "ts_gram_batch: bad job");
            if (B.n > 0 && (J.mat != nullptr) != weighted) return fail(PC_EINVAL, "ts_gram_batch: mixed weights");
            weighted = J.mat != nullptr;
            B.j[B.n] = J;
            B.off[B.n + 1] = B.off[B.n] + (int64_t)J.rows * J.cols;
            ++B.n;
            maxr = std::max(maxr, J.rows);
            maxc = std::max(maxc, J.cols);
        }
        if (B.n == 0) continue;
        const int RB = maxr <= 2 ? 2 : (maxr <= 4 ? 4 : 8);
        const int nrg = (maxr + RB - 1) / RB, ngc = (maxc + kGramCB - 1) / kGramCB;
        const int64_t entries = B.off[B.n];
        int64_t nchunk = (2LL * device_sm_count() + (int64_t)nrg * ngc * B.n - 1) / ((int64_t)nrg * ngc * B.n);
        nchunk = std::min<int64_t>(nchunk, std::max<int64_t>(1, m / 512));
        nchunk = std::min<int64_t>(nchunk, (int64_t)(part_cap / (2 * entries)));
        if (nchunk < 1) return fail(PC_EINVAL, "ts_gram_batch: partial-sum scratch too small");
        const dim3 grid((unsigned)nchunk, nrg * ngc, B.n);
        const double drho = rho1 - rho0;
        const int mk = weighted ? matkind : -1;
#define PC_GRAM_B(RBV, MKV) \
    ts_gram_batch_kernel<RBV, MKV><<<grid, kGramThreads, 0, s>>>(B, m, rho0, drho, ngc, (int)nchunk, d_part)
#define PC_GRAM_MK(RBV)                  \
    if (mk < 0) PC_GRAM_B(RBV, -1);      \
    else if (mk == 0) PC_GRAM_B(RBV, 0); \
    else if (mk == 2) PC_GRAM_B(RBV, 2); \
    else PC_GRAM_B(RBV, 1);
        if (RB == 2) { PC_GRAM_MK(2) }
        else if (RB == 4) { PC_GRAM_MK(4) }
        else { PC_GRAM_MK(8) }
#undef PC_GRAM_MK
#undef PC_GRAM_B
        note_launch();
        ts_gram_batch_reduce<<<(unsigned)((entries + 7) / 8), 256, 0, s>>>(B, d_part, (int)nchunk);
        note_launch();
        PC_CUDA_TRY(cudaGetLastError());
    }
    return PC_OK;
}

int ts_update_batch(const UpdateJob* jobs, int njobs, int64_t vs, cudaStream_t s) {
    for (int base = 0; base < njobs; base += kMaxJobs) {
        UpdateBatch U;
        U.n = 0;
        int maxk = 0, maxc = 0;
        for (int i = base; i < njobs && U.n < kMaxJobs; ++i) {
            const UpdateJob& J = jobs[i];
            if (J.cols <= 0) continue;
            if (J.k <= 0 || !J.A || !J.h || !J.C) return fail(PC_EINVAL, "ts_update_batch: bad job");
            U.j[U.n++] = J;
            maxk = std::max(maxk, J.k);
            maxc = std::max(maxc, J.cols);
        }
        if (U.n == 0) continue;
        const int CB = maxc <= 2 ? 2 : 4;
        const size_t smem = sizeof(double2) * (size_t)maxk * CB;
        if (smem > 48 * 1024) return fail(PC_EINVAL, "ts_update_batch: too many basis columns");
        const int ngc = (maxc + CB - 1) / CB;
        int64_t gx = (vs + 255) / 256;
        gx = std::min<int64_t>(gx, std::max<int64_t>(1, 8LL * device_sm_count() / ((int64_t)ngc * U.n)));
        if (CB == 2)
            ts_update_batch_kernel<2><<<dim3((unsigned)gx, ngc, U.n), 256, smem, s>>>(U, vs);
        else
            ts_update_batch_kernel<4><<<dim3((unsigned)gx, ngc, U.n), 256, smem, s>>>(U, vs);
        note_launch();
        PC_CUDA_TRY(cudaGetLastError());
    }
    return PC_OK;
}

}  // namespace pc
