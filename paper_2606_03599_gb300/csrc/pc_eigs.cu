// Shift-invert block Krylov-Schur eigensolver over the parity blocks (Sec. 6).
//
// For each space (one of the four parity blocks, Cor. 4.2, or the full space)
// the outer iteration works with Op = (A - sigma M)^-1 M, which is
// self-adjoint in the M inner product: eigenpairs A v = lambda M v map to
// Op v = mu v with mu = 1 / (lambda - sigma) (Eq. shift_invert_system_unified,
// sigma = -delta).  Every application of Op is a batch of PCG solves (one per
// column of the newest Krylov block, all active spaces together).
//
// Basis V is M-orthonormal; Op V_m = V_{m+b} H with H built column by column
// from classical Gram-Schmidt run twice (CGS2) and a twice-applied Cholesky QR
// of each new block.  Rayleigh-Ritz on the leading m x m part of H gives Ritz
// values mu_i; the wanted pairs have the largest mu.  Restarts keep the best
// Ritz vectors and the coupling row of the last block (Krylov-Schur form).
//
// Convergence uses the true FP64 residual of each Ritz vector y (unit M-norm):
// with the Rayleigh quotient lambda = y^H A y / y^H M y,
//     || A y - lambda M y ||_2 / ( max(|lambda|, |sigma|) || M y ||_2 ) <= tol,
// i.e. relative to lambda, and to the scale of the shift for the few eigenvalues below |sigma|
// (acoustic modes next to Gamma).
//
// At a Bloch vector where symbol blocks vanish (Gamma, Sec. 6.2, App. C) the
// zero-derivative modes T_sigma (e_m (x) e_alpha) of those Fourier modes m are
// M-orthonormalised and projected out of every Krylov vector exactly (the
// M-orthogonal complement is invariant under Op), so they are never reported.
//
// The four block spectra are merged by sorting (Eq. block_gep_impl_unified):
// the lowest nev of the union are final once every block either lists an
// eigenvalue at or above the nev-th merged value, or has converged all of its
// requested pairs below it; otherwise that block's request grows.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pc_complex.cuh"
#include "pc_solver.h"

namespace pc {

using cd = std::complex<double>;

// ================================================================== small dense LA (host)
// Hermitian eigen-decomposition: Householder reduction to tridiagonal form, a diagonal unitary
// scaling that makes the off-diagonal real, then the implicit QL iteration with Wilkinson shifts
// on the real symmetric tridiagonal matrix (the textbook tridiagonal QL method).  A: n x n
// column-major (only its Hermitian part is used).  Returns eigenvalues in descending order and the
// matching orthonormal eigenvectors (columns of V).
static void herm_eig_desc(int n, std::vector<cd> A, std::vector<double>& w, std::vector<cd>& V) {
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < j; ++i) {
            cd h = 0.5 * (A[i + j * n] + std::conj(A[j + i * n]));
            A[i + j * n] = h;
            A[j + i * n] = std::conj(h);
        }
    for (int i = 0; i < n; ++i) A[i + i * n] = cd(A[i + i * n].real(), 0.0);
    // Q accumulates the reflectors: A = Q T Q^H
    std::vector<cd> Q((size_t)n * n, cd(0, 0));
    for (int i = 0; i < n; ++i) Q[i + i * n] = 1.0;
    std::vector<cd> v(n), p(n), q(n);
    for (int k = 0; k + 2 < n; ++k) {
        // reflector H = I - tau u u^H mapping A[k+1:, k] to a multiple of e_{k+1}
        double xn = 0;
        for (int i = k + 1; i < n; ++i) xn += std::norm(A[i + k * n]);
        xn = std::sqrt(xn);
        if (xn == 0.0) continue;
        const cd x0 = A[(k + 1) + k * n];
        const double ax0 = std::abs(x0);
        const cd ph = ax0 > 0 ? x0 / ax0 : cd(1, 0);
        const cd alpha = -ph * xn;
        for (int i = 0; i < n; ++i) v[i] = 0;
        for (int i = k + 1; i < n; ++i) v[i] = A[i + k * n];
        v[k + 1] -= alpha;
        double vn = 0;
        for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
        if (vn == 0.0) continue;
        const double tau = 2.0 / vn;
        // A <- H A H with H = I - tau v v^H (A Hermitian): p = tau A v, K = tau/2 v^H p,
        // q = p - K v, A <- A - v q^H - q v^H
        for (int i = k; i < n; ++i) {
            cd s = 0;
            for (int j = k + 1; j < n; ++j) s += A[i + j * n] * v[j];
            p[i] = tau * s;
        }
        cd K = 0;
        for (int i = k + 1; i < n; ++i) K += std::conj(v[i]) * p[i];
        K *= 0.5 * tau;
        for (int i = k; i < n; ++i) q[i] = p[i] - K * (i > k ? v[i] : cd(0, 0));
        for (int j = k; j < n; ++j)
            for (int i = k; i < n; ++i) {
                const cd vi = i > k ? v[i] : cd(0, 0), vj = j > k ? v[j] : cd(0, 0);
                A[i + j * n] -= vi * std::conj(q[j]) + q[i] * std::conj(vj);
            }
        // Q <- Q H
        for (int i = 0; i < n; ++i) {
            cd s = 0;
            for (int j = k + 1; j < n; ++j) s += Q[i + j * n] * v[j];
            s *= tau;
            for (int j = k + 1; j < n; ++j) Q[i + j * n] -= s * std::conj(v[j]);
        }
    }
    // T: real diagonal d, complex subdiagonal A[k+1, k]; D = diag(phases) makes it real
    std::vector<double> d(n), e(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = A[i + i * n].real();
    cd phase = 1.0;
    std::vector<cd> phs(n);
    phs[0] = 1.0;
    for (int k = 0; k + 1 < n; ++k) {
        const cd t = A[(k + 1) + k * n];
        const double at = std::abs(t);
        e[k] = at;
        phase = at > 0 ? phase * (t / at) : phase;
        phs[k + 1] = phase;
    }
    // implicit QL on (d, e), rotations accumulated in Z (real, column-major)
    std::vector<double> Z((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[i + i * n] = 1.0;
    for (int l = 0; l < n; ++l) {
        for (int iter = 0; iter < 60; ++iter) {
            int m = l;
            for (; m + 1 < n; ++m) {
                const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-16 * dd) break;
            }
            if (m == l) break;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, pp = 0.0;
            int i = m - 1;
            bool deflated = false;
            for (; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= pp;
                    e[m] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * b;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - b;
                for (int k = 0; k < n; ++k) {
                    f = Z[k + (i + 1) * n];
                    Z[k + (i + 1) * n] = s * Z[k + i * n] + c * f;
                    Z[k + i * n] = c * Z[k + i * n] - s * f;
                }
            }
            if (deflated) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    // eigenvectors: Q D Z
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] > d[b]; });
    w.resize(n);
    V.assign((size_t)n * n, cd(0, 0));
    std::vector<cd> QD((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) QD[i + j * n] = Q[i + j * n] * phs[j];
    for (int jj = 0; jj < n; ++jj) {
        const int j = idx[jj];
        w[jj] = d[j];
        for (int k = 0; k < n; ++k) {
            const double z = Z[k + j * n];
            if (z == 0.0) continue;
            for (int i = 0; i < n; ++i) V[i + jj * n] += QD[i + k * n] * z;
        }
    }
}

// G = R^H R with R upper triangular (column-major n x n).  False if G is not numerically SPD.
static bool chol_upper(int n, const std::vector<cd>& G, std::vector<cd>& R) {
    R.assign((size_t)n * n, cd(0, 0));
    double scale = 0;
    for (int i = 0; i < n; ++i) scale = std::max(scale, G[i + i * n].real());
    for (int j = 0; j < n; ++j) {
        cd s = G[j + j * n];
        for (int k = 0; k < j; ++k) s -= std::norm(R[k + j * n]);
        if (!(s.real() > 1e-13 * scale)) return false;
        const double d = std::sqrt(s.real());
        R[j + j * n] = d;
        for (int i = j + 1; i < n; ++i) {
            cd t = G[j + i * n];
            for (int k = 0; k < j; ++k) t -= std::conj(R[k + j * n]) * R[k + i * n];
            R[j + i * n] = t / d;
        }
    }
    return true;
}

static void upper_inverse(int n, const std::vector<cd>& R, std::vector<cd>& Ri) {
    Ri.assign((size_t)n * n, cd(0, 0));
    for (int j = 0; j < n; ++j) {
        Ri[j + j * n] = 1.0 / R[j + j * n];
        for (int i = j - 1; i >= 0; --i) {
            cd s = 0;
            for (int k = i + 1; k <= j; ++k) s += R[i + k * n] * Ri[k + j * n];
            Ri[i + j * n] = -s / R[i + i * n];
        }
    }
}

// ================================================================== device kernels
__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Deterministic pseudo-random start vectors: uniform in [-1, 1) for re and im.
__global__ void fill_random(double2* v, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a = splitmix(seed ^ (2 * (uint64_t)i)), b = splitmix(seed ^ (2 * (uint64_t)i + 1));
        v[i] = make_double2((double)(a >> 11) * 0x1.0p-52 - 1.0, (double)(b >> 11) * 0x1.0p-52 - 1.0);
    }
}

// Per-candidate residual statistics of y_i and r_i = (A - lambda_i M) y_i:
// out[5 i + 0..4] partials of sum |r|^2, sum rho^2 |y|^2, Re sum conj(y) r, sum rho |y|^2, Re sum rho conj(y) r.
__global__ void resid_stats(const double2* __restrict__ Y, const double2* __restrict__ Rv, const void* __restrict__ mat,
                            int matkind, double rho0, double rho1, int64_t m, double* __restrict__ part, int npart) {
    const int i = blockIdx.y;
    const double2* y = Y + (int64_t)i * 3 * m;
    const double2* r = Rv + (int64_t)i * 3 * m;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const double rho = node_rho_hat<double>(mat, matkind, rho0, rho1, m, t);
        for (int a = 0; a < 3; ++a) {
            const double2 yv = y[a * m + t], rv = r[a * m + t];
            const double yy = yv.x * yv.x + yv.y * yv.y;
            const double yr = yv.x * rv.x + yv.y * rv.y;
            acc[0] += rv.x * rv.x + rv.y * rv.y;
            acc[1] += rho * rho * yy;
            acc[2] += yr;
            acc[3] += rho * yy;
            acc[4] += rho * yr;
        }
    }
    __shared__ double red[5][32];
    for (int q = 0; q < 5; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        part[((int64_t)i * 5 + threadIdx.x) * npart + blockIdx.x] = s;
    }
}

// Per-system squared norms (partials) of n_sys vectors of vs elements.
template <typename C>
__global__ void sq_norms(const C* __restrict__ v, int64_t vs, double* __restrict__ part, int npart) {
    const int s = blockIdx.y;
    double acc = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        const C x = v[s * vs + e];
        acc += (double)x.x * (double)x.x + (double)x.y * (double)x.y;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
        part[(int64_t)s * npart + blockIdx.x] = sum;
    }
}

// out32_s = in64_s * scale_s (complex128 -> complex64)
__global__ void to_c64_scaled(const double2* __restrict__ in, float2* __restrict__ out, const double* __restrict__ scale,
                              int64_t vs) {
    const int s = blockIdx.y;
    const double f = scale[s];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = in[s * vs + e];
        out[s * vs + e] = make_float2((float)(v.x * f), (float)(v.y * f));
    }
}

// x64_s += d32_s * scale_s (systems of scale 0 are left as they are)
__global__ void axpy_c64_into_c128(const float2* __restrict__ d, double2* __restrict__ x, const double* __restrict__ scale,
                                   int64_t vs) {
    const int s = blockIdx.y;
    const double f = scale[s];
    if (f == 0.0) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = d[s * vs + e];
        double2 o = x[s * vs + e];
        o.x += f * (double)v.x;
        o.y += f * (double)v.y;
        x[s * vs + e] = o;
    }
}

// res = b - res
// res_s = b_s - res_s for the systems of nonzero scale_s (the others keep their residual)
__global__ void sub_from(const double2* __restrict__ b, double2* __restrict__ res, const double* __restrict__ scale,
                         int64_t vs) {
    const int s = blockIdx.y;
    if (scale[s] == 0.0) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 bv = b[s * vs + e], rv = res[s * vs + e];
        res[s * vs + e] = make_double2(bv.x - rv.x, bv.y - rv.y);
    }
}

static int ctas_for(int64_t n) {
    int64_t g = (n + 1023) / 1024;
    if (g > 304) g = 304;
    return (int)(g < 1 ? 1 : g);
}

// ================================================================== solver context
struct Space {
    int block = 0;          // 0..3 or -1
    int kslot = 0;          // Bloch slot of the grid this space solves at
    int64_t m = 0, vs = 0;  // nodes, elements per vector
    double2* V = nullptr;   // basis [mcap][vs]
    int m_exp = 0;          // expanded columns
    std::vector<cd> H;      // (mcap) x (mcap), column-major, ld = mcap
    std::vector<double> theta;
    std::vector<cd> S;      // Ritz vectors of the leading block (m_exp x m_exp)
    int target = 0;
    int nconv = 0;
    std::vector<double> lam, res;  // converged eigenvalues (ascending) and residuals
    bool done = false;
    double2* Z = nullptr;  // null basis [nz][vs], M-orthonormal
    int nz = 0;
};

struct Eigs {
    pc_grid* g = nullptr;
    const pc_options* o = nullptr;
    cudaStream_t s = nullptr;
    double sigma = 0;
    int bs = 4, mmax = 32, mcap = 36;
    std::vector<Space> sp;  // space (kslot, block) at index kslot * (spaces per Bloch vector) + block
    double2 *W = nullptr, *MW = nullptr, *T = nullptr, *RHS = nullptr;
    double2 *Y = nullptr, *AY = nullptr;
    int ycols = 0;  // columns of Y and AY (Ritz candidates checked per batch)
    float* X32 = nullptr;
    float* R32 = nullptr;
    double* dpart = nullptr;
    double* dscale = nullptr;
    cd* dsmall = nullptr;  // device scratch for small GEMM results
    size_t dsmall_cap = 0;
    double* gpart = nullptr;  // partial sums of the Gram kernels
    size_t gpart_cap = 0;
    long long pcg_iters = 0;
    int max_pcg = 0, solves = 0, expansions = 0, cholqr_single = 0, syncs = 0;
    double t_op = 0, t_ritz = 0, t_check = 0;  // wall seconds in the solves, Rayleigh-Ritz, residual checks
    std::vector<void*> allocs;
    ~Eigs() {
        for (void* p : allocs) cudaFree(p);
    }
    template <typename T>
    int alloc(T** p, size_t count) {
        cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(eigensolver)");
        allocs.push_back(*p);
        return PC_OK;
    }
};

static const cuDoubleComplex kOne = {1.0, 0.0}, kZero = {0.0, 0.0};

// dh (device, rows x cols) = A^H M B in the mass inner product of space S.
static int gram_m(Eigs& E, const Space& S, const double2* A, int rows, const double2* B, int cols, cd* dh) {
    pc_grid* g = E.g;
    return ts_gram(A, rows, B, cols, S.m, grid_mat(g, S.block), g->matkind, g->rhohat[0], g->rhohat[1],
                   reinterpret_cast<double2*>(dh), E.gpart, E.gpart_cap, E.s);
}

static int gram_batch(Eigs& E, const std::vector<GramJob>& jobs) {
    if (jobs.empty()) return PC_OK;
    pc_grid* g = E.g;
    return ts_gram_batch(jobs.data(), (int)jobs.size(), E.sp[0].m, g->matkind, g->rhohat[0], g->rhohat[1], E.gpart,
                         E.gpart_cap, E.s);
}

static int update_batch(Eigs& E, const std::vector<UpdateJob>& jobs) {
    if (jobs.empty()) return PC_OK;
    return ts_update_batch(jobs.data(), (int)jobs.size(), E.sp[0].vs, E.s);
}

static int to_host(Eigs& E, const cd* d, size_t n, std::vector<cd>& out) {
    out.resize(n);
    PC_CUDA_TRY(cudaMemcpyAsync(out.data(), d, sizeof(cd) * n, cudaMemcpyDeviceToHost, E.s));
    PC_CUDA_TRY(cudaStreamSynchronize(E.s));
    ++E.syncs;
    return PC_OK;
}

// Cout (vs x cols) = beta Cout + alpha A (vs x k) * Hs (k x cols, host); alpha and beta real.
static int gemm_nn_host(Eigs& E, const double2* A, int k, const std::vector<cd>& Hs, int cols, double2* Cout,
                        int64_t vs, cuDoubleComplex alpha, cuDoubleComplex beta) {
    PC_CUDA_TRY(cudaMemcpyAsync(E.dsmall, Hs.data(), sizeof(cd) * k * cols, cudaMemcpyHostToDevice, E.s));
    return ts_update(A, k, reinterpret_cast<const double2*>(E.dsmall), cols, Cout, vs, alpha.x, beta.x, E.s);
}

static int mass(Eigs& E, const Space& S, const double2* x, double2* y, int nvec) {
    pc_grid* g = E.g;
    return launch_mass(PC_C128, x, y, grid_mat(g, S.block), g->matkind, g->rhohat[0], g->rhohat[1], S.m, E.s, nvec);
}

// W -= Z (Z^H M W)  (exact M-orthogonal projection off the null basis), device-resident
static int project_null(Eigs& E, Space& S, double2* Wv, int cols) {
    if (S.nz == 0) return PC_OK;
    PC_TRY(gram_m(E, S, S.Z, S.nz, Wv, cols, E.dsmall));
    return ts_update(S.Z, S.nz, reinterpret_cast<const double2*>(E.dsmall), cols, Wv, S.vs, -1.0, 1.0, E.s);
}

// M-orthonormalise the cols columns of Wv in place (CholQR2); returns R (cols x cols, upper) with
// Wv_in = Wv_out R.  Rank-deficient columns are replaced by random vectors orthogonalised against
// V[:, 0:nv] (their R columns are set to zero).  One space at a time (start blocks and the rare
// rank-deficient Krylov block); the expansions run the batched form in expand().
static int cholqr2(Eigs& E, Space& S, double2* Wv, int cols, int nv, std::vector<cd>& Rtot, uint64_t seed) {
    Rtot.assign((size_t)cols * cols, cd(0, 0));
    for (int i = 0; i < cols; ++i) Rtot[i + i * cols] = 1.0;
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<cd> G, R, Ri;
        PC_TRY(gram_m(E, S, Wv, cols, Wv, cols, E.dsmall));
        PC_TRY(to_host(E, E.dsmall, (size_t)cols * cols, G));
        if (!chol_upper(cols, G, R)) {
            if (pass == 1) return fail(PC_ENOCONV, "eigensolver: Krylov block lost rank twice");
            // replace the block by fresh random directions (breakdown of the Krylov space)
            fill_random<<<ctas_for(cols * S.vs), 256, 0, E.s>>>(Wv, cols * S.vs, seed);
            note_launch();
            PC_TRY(project_null(E, S, Wv, cols));
            for (int rep = 0; rep < 2 && nv > 0; ++rep) {
                PC_TRY(gram_m(E, S, S.V, nv, Wv, cols, E.dsmall));
                PC_TRY(ts_update(S.V, nv, reinterpret_cast<const double2*>(E.dsmall), cols, Wv, S.vs, -1.0, 1.0,
                                 E.s));
            }
            Rtot.assign((size_t)cols * cols, cd(0, 0));
            pass = -1;  // restart both passes on the new block; R of a replaced block is zero
            continue;
        }
        // a block whose columns are already nearly M-orthogonal (every normalised off-diagonal
        // Gram entry below 0.1, so its scaled condition number is below ~1.25) is orthonormal to
        // working precision after one pass; the second pass is only needed otherwise
        bool well_conditioned = pass == 0;
        for (int j = 0; j < cols && well_conditioned; ++j)
            for (int i = 0; i < j; ++i)
                if (std::abs(G[i + j * cols]) > 0.1 * std::sqrt(G[i + i * cols].real() * G[j + j * cols].real()))
                    well_conditioned = false;
        upper_inverse(cols, R, Ri);
        // Wv <- Wv R^-1  (through T)
        PC_TRY(gemm_nn_host(E, Wv, cols, Ri, cols, E.T, S.vs, kOne, kZero));
        PC_CUDA_TRY(cudaMemcpyAsync(Wv, E.T, sizeof(double2) * cols * S.vs, cudaMemcpyDeviceToDevice, E.s));
        // Rtot <- R Rtot
        std::vector<cd> Rn((size_t)cols * cols, cd(0, 0));
        for (int j = 0; j < cols; ++j)
            for (int i = 0; i < cols; ++i) {
                cd acc = 0;
                for (int k = 0; k < cols; ++k) acc += R[i + k * cols] * Rtot[k + j * cols];
                Rn[i + j * cols] = acc;
            }
        Rtot.swap(Rn);
        if (well_conditioned) {
            ++E.cholqr_single;
            break;
        }
    }
    return PC_OK;
}

// W (stacked [nsys][vs]) = Op applied to the right-hand sides RHS = M V (stacked), i.e. solves of
// (A - sigma M) W = RHS, FP64 PCG or complex64 PCG with FP64 residual refinement.  System i is
// in block blocks[i] at Bloch slot kslots[i]; systems with live[i] == 0 have a zero right-hand
// side (the PCG marks them done at its start) and get no refinement apply.
static int apply_op(Eigs& E, int nsys, const std::vector<int>& blocks, const std::vector<int>& kslots,
                    const std::vector<char>& live, int64_t vs) {
    pc_grid* g = E.g;
    const pc_options& o = *E.o;
    std::vector<PcgResult> res(nsys);
    const int* ks = g->nk > 1 ? kslots.data() : nullptr;
    if (o.precision == PC_PREC_FP64) {
        PC_TRY(pcg_solve(g, PC_C128, nsys, blocks.data(), E.sigma, E.RHS, E.W, o.inner_tol, o.inner_maxit, res.data(),
                         E.s, o.precond_fp32 != 0, ks));
        for (auto& r : res) {
            E.pcg_iters += r.iters;
            E.max_pcg = std::max(E.max_pcg, r.iters);
            if (r.status == PC_EBREAKDOWN)
                return fail(PC_EBREAKDOWN, "PCG breakdown: sigma is not below the spectrum");
            if (r.status == PC_ENAN) return fail(PC_ENAN, "PCG met NaN");
        }
        for (int i = 0; i < nsys; ++i) E.solves += live[i] ? 1 : 0;
        return PC_OK;
    }
    // mixed precision: x = 0, res = rhs; repeat { d = PCG32(res/|res|); x += |res| d; res = rhs - (A - sigma M) x }
    // over the systems whose FP64 residual is still above inner_tol |rhs|.  A complex64 sweep
    // reduces its system's residual by about its own PCG tolerance, so each sweep asks for a
    // quarter of the reduction the worst remaining system still needs, within [tol32, 0.1]: the
    // last sweep of a solve then stops after a few iterations instead of running to tol32.
    const int nc = ctas_for(vs);
    const dim3 vg(nc, nsys);
    PC_CUDA_TRY(cudaMemsetAsync(E.W, 0, sizeof(double2) * nsys * vs, E.s));
    PC_CUDA_TRY(cudaMemcpyAsync(E.MW, E.RHS, sizeof(double2) * nsys * vs, cudaMemcpyDeviceToDevice, E.s));
    std::vector<double> bnorm(nsys), rnorm(nsys), part((size_t)nsys * nc);
    const double tol32 = 1e-4;
    std::vector<ApplyItem> items;
    for (int sweep = 0; sweep < 40; ++sweep) {
        sq_norms<double2><<<vg, 256, 0, E.s>>>(E.MW, vs, E.dpart, nc);
        note_launch();
        PC_CUDA_TRY(cudaMemcpyAsync(part.data(), E.dpart, sizeof(double) * nsys * nc, cudaMemcpyDeviceToHost, E.s));
        PC_CUDA_TRY(cudaStreamSynchronize(E.s));
        ++E.syncs;
        std::vector<double> sc(nsys, 0.0);
        std::vector<char> act(nsys, 0);
        double worst = 0.0;  // largest |res| / |rhs| of the systems still running
        for (int i = 0; i < nsys; ++i) {
            double a = 0;
            for (int c = 0; c < nc; ++c) a += part[(size_t)i * nc + c];
            rnorm[i] = std::sqrt(a);
            if (sweep == 0) bnorm[i] = rnorm[i];
            if (!std::isfinite(rnorm[i])) return fail(PC_ENAN, "refinement met NaN");
            act[i] = live[i] && rnorm[i] > o.inner_tol * bnorm[i];
            if (act[i]) {
                sc[i] = 1.0 / rnorm[i];
                worst = std::max(worst, rnorm[i] / bnorm[i]);
            }
        }
        if (worst == 0.0) break;
        const double tol_sweep = std::min(0.1, std::max(tol32, 0.25 * o.inner_tol / worst));
        PC_CUDA_TRY(cudaMemcpyAsync(E.dscale, sc.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, E.s));
        to_c64_scaled<<<vg, 256, 0, E.s>>>(E.MW, (float2*)E.R32, E.dscale, vs);  // zero for the others
        note_launch();
        PC_TRY(pcg_solve(g, PC_C64, nsys, blocks.data(), E.sigma, E.R32, E.X32, tol_sweep, o.inner_maxit, res.data(),
                         E.s, false, ks));
        for (auto& r : res) {
            E.pcg_iters += r.iters;
            E.max_pcg = std::max(E.max_pcg, r.iters);
            if (r.status == PC_EBREAKDOWN) return fail(PC_EBREAKDOWN, "PCG breakdown: sigma is not below the spectrum");
        }
        items.clear();
        for (int i = 0; i < nsys; ++i) {
            sc[i] = act[i] ? rnorm[i] : 0.0;
            if (!act[i]) continue;
            ApplyItem it;
            it.x = E.W + i * vs;
            it.y = E.MW + i * vs;
            it.mat = grid_mat(g, blocks[i]);
            it.shift = E.sigma;
            it.block = blocks[i];
            it.dot_slot = -1;
            it.skip = nullptr;
            it.kslot = kslots[i];
            items.push_back(it);
        }
        PC_CUDA_TRY(cudaMemcpyAsync(E.dscale, sc.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, E.s));
        axpy_c64_into_c128<<<vg, 256, 0, E.s>>>((const float2*)E.X32, E.W, E.dscale, vs);
        note_launch();
        // residual in FP64 of the systems of this sweep: MW = RHS - (A - sigma M) W
        PC_TRY(grid_apply(g, PC_C128, blocks[0] < 0, items.data(), (int)items.size(), nullptr, 0, E.s, nullptr));
        sub_from<<<vg, 256, 0, E.s>>>(E.RHS, E.MW, E.dscale, vs);
        note_launch();
        PC_CUDA_TRY(cudaGetLastError());
    }
    for (int i = 0; i < nsys; ++i) E.solves += live[i] ? 1 : 0;
    return PC_OK;
}

// Rayleigh-Ritz on the leading m_exp x m_exp block of H (descending mu).
static void ritz(Eigs& E, Space& S) {
    const int m = S.m_exp;
    std::vector<cd> Hm((size_t)m * m);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) Hm[i + j * m] = S.H[i + j * E.mcap];
    herm_eig_desc(m, Hm, S.theta, S.S);
}

// True residuals of the leading ncand[c] Ritz pairs of spaces chk[c] (all in one apply); returns
// their Rayleigh quotients and residuals per space.  Candidates go through Y / AY in groups of at
// most E.ycols columns.
static int check_pairs(Eigs& E, const std::vector<int>& chk, const std::vector<int>& ncand,
                       std::vector<std::vector<double>>& lam, std::vector<std::vector<double>>& rel) {
    pc_grid* g = E.g;
    const int64_t vs = E.sp[0].vs, m = E.sp[0].m;
    const int nc = ctas_for(m);
    lam.assign(chk.size(), {});
    rel.assign(chk.size(), {});
    size_t c0 = 0;
    while (c0 < chk.size()) {
        size_t c1 = c0;
        int cols = 0;
        while (c1 < chk.size() && (cols + ncand[c1] <= E.ycols || c1 == c0)) cols += ncand[c1++];
        // Ritz vectors Y = V S_k of every space of the group (one upload, one launch)
        std::vector<cd> hs;
        std::vector<size_t> so;
        for (size_t c = c0; c < c1; ++c) {
            const Space& S = E.sp[chk[c]];
            so.push_back(hs.size());
            for (int j = 0; j < ncand[c]; ++j)
                for (int i = 0; i < S.m_exp; ++i) hs.push_back(S.S[i + j * S.m_exp]);
        }
        if (hs.size() > E.dsmall_cap) return fail(PC_EINVAL, "eigensolver: small-matrix scratch too small");
        PC_CUDA_TRY(cudaMemcpyAsync(E.dsmall, hs.data(), sizeof(cd) * hs.size(), cudaMemcpyHostToDevice, E.s));
        std::vector<UpdateJob> uj;
        std::vector<ApplyItem> items;
        std::vector<double> lr;
        int col = 0;
        for (size_t c = c0; c < c1; ++c) {
            const Space& S = E.sp[chk[c]];
            uj.push_back({S.V, S.m_exp, reinterpret_cast<const double2*>(E.dsmall + so[c - c0]), ncand[c],
                          E.Y + (int64_t)col * vs, 1.0, 0.0});
            for (int i = 0; i < ncand[c]; ++i) {
                ApplyItem it;
                it.x = E.Y + (int64_t)(col + i) * vs;
                it.y = E.AY + (int64_t)(col + i) * vs;
                it.mat = grid_mat(g, S.block);
                it.shift = E.sigma + 1.0 / S.theta[i];
                it.block = S.block;
                it.dot_slot = -1;
                it.skip = nullptr;
                it.kslot = S.kslot;
                items.push_back(it);
                lr.push_back(it.shift);
            }
            col += ncand[c];
        }
        PC_TRY(update_batch(E, uj));
        PC_TRY(grid_apply(g, PC_C128, E.sp[chk[c0]].block < 0, items.data(), (int)items.size(), nullptr, 0, E.s,
                          nullptr));
        col = 0;
        for (size_t c = c0; c < c1; ++c) {
            const Space& S = E.sp[chk[c]];
            resid_stats<<<dim3(nc, ncand[c]), 256, 0, E.s>>>(E.Y + (int64_t)col * vs, E.AY + (int64_t)col * vs,
                                                             grid_mat(g, S.block), g->matkind, g->rhohat[0],
                                                             g->rhohat[1], m, E.dpart + (size_t)col * 5 * nc, nc);
            note_launch();
            col += ncand[c];
        }
        PC_CUDA_TRY(cudaGetLastError());
        std::vector<double> part((size_t)cols * 5 * nc);
        PC_CUDA_TRY(cudaMemcpyAsync(part.data(), E.dpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, E.s));
        PC_CUDA_TRY(cudaStreamSynchronize(E.s));
        ++E.syncs;
        col = 0;
        for (size_t c = c0; c < c1; ++c) {
            auto& L = lam[c];
            auto& Rl = rel[c];
            L.resize(ncand[c]);
            Rl.resize(ncand[c]);
            for (int i = 0; i < ncand[c]; ++i, ++col) {
                double q[5];
                for (int k = 0; k < 5; ++k) {
                    double a = 0;
                    for (int t = 0; t < nc; ++t) a += part[((size_t)col * 5 + k) * nc + t];
                    q[k] = a;
                }
                const double d = q[2] / q[3];  // Rayleigh-quotient correction of lambda
                L[i] = lr[col] + d;
                const double r2 = std::max(0.0, q[0] - 2.0 * d * q[4] + d * d * q[1]);
                // relative to the eigenvalue, or to the shift's scale for eigenvalues below |sigma|
                // (the acoustic modes next to Gamma, where |lambda| / ||A|| is below what an
                // inexact shift-invert solve resolves; for lambda >= |sigma| this is ||r|| / |lambda|)
                Rl[i] = std::sqrt(r2) / (std::max(std::fabs(L[i]), std::fabs(E.sigma)) * std::sqrt(q[1]));
            }
        }
        c0 = c1;
    }
    return PC_OK;
}

// Krylov-Schur restart keeping the best `keep` Ritz vectors.
static int restart(Eigs& E, Space& S, int keep) {
    const int m = S.m_exp, bs = E.bs, ld = E.mcap;
    std::vector<cd> Sk((size_t)m * keep);
    for (int j = 0; j < keep; ++j)
        for (int i = 0; i < m; ++i) Sk[i + j * m] = S.S[i + j * m];
    PC_TRY(gemm_nn_host(E, S.V, m, Sk, keep, E.T, S.vs, kOne, kZero));
    PC_CUDA_TRY(cudaMemcpyAsync(S.V, E.T, sizeof(double2) * keep * S.vs, cudaMemcpyDeviceToDevice, E.s));
    PC_CUDA_TRY(cudaMemcpyAsync(S.V + (int64_t)keep * S.vs, S.V + (int64_t)m * S.vs, sizeof(double2) * bs * S.vs,
                                cudaMemcpyDeviceToDevice, E.s));
    std::vector<cd> Hn((size_t)ld * ld, cd(0, 0));
    for (int i = 0; i < keep; ++i) Hn[i + i * ld] = S.theta[i];
    for (int r = 0; r < bs; ++r)
        for (int j = 0; j < keep; ++j) {
            cd acc = 0;
            for (int k = 0; k < m; ++k) acc += S.H[(m + r) + k * ld] * S.S[k + j * m];
            Hn[(keep + r) + j * ld] = acc;
        }
    S.H.swap(Hn);
    S.m_exp = keep;
    return PC_OK;
}

// Upper-triangular product R_a R_b (n x n, column-major).
static std::vector<cd> upper_mul(int n, const std::vector<cd>& Ra, const std::vector<cd>& Rb) {
    std::vector<cd> out((size_t)n * n, cd(0, 0));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            cd acc = 0;
            for (int k = 0; k < n; ++k) acc += Ra[i + k * n] * Rb[k + j * n];
            out[i + j * n] = acc;
        }
    return out;
}

// One expansion of every active space: solves (one batched PCG over all of them), projection off
// the null bases, CGS2 and the first CholQR Gram (batched, one copy to the host), the CholQR update
// (batched, a second pass only for ill-conditioned blocks), Rayleigh-Ritz, the true residuals of
// the candidate pairs (one batched apply) and restarts.
static int expand(Eigs& E, std::vector<int>& active, double tol) {
    pc_grid* g = E.g;
    const int bs = E.bs, ld = E.mcap;
    const int64_t vs = E.sp[active[0]].vs;
    const int nA = (int)active.size();
    // Every space keeps its own systems (space i: systems i bs .. i bs + bs - 1) whether it is
    // active or not, so the batched PCG sees the same systems at every expansion and replays one
    // captured graph for the whole solve; finished spaces get a zero right-hand side, which the
    // PCG retires at its start.
    const int nS = (int)E.sp.size(), nsys = bs * nS;
    std::vector<int> blocks(nsys), kslots(nsys);
    std::vector<char> live(nsys, 0);
    for (int i = 0; i < nS; ++i)
        for (int j = 0; j < bs; ++j) {
            blocks[i * bs + j] = E.sp[i].block;
            kslots[i * bs + j] = E.sp[i].kslot;
        }
    for (int a = 0; a < nA; ++a)
        for (int j = 0; j < bs; ++j) live[active[a] * bs + j] = 1;
    for (int i = 0; i < nS; ++i) {
        Space& S = E.sp[i];
        double2* rhs = E.RHS + (int64_t)i * bs * vs;
        if (live[i * bs]) PC_TRY(mass(E, S, S.V + (int64_t)S.m_exp * vs, rhs, bs));
        else PC_CUDA_TRY(cudaMemsetAsync(rhs, 0, sizeof(double2) * bs * vs, E.s));
    }
    const auto t_op0 = std::chrono::steady_clock::now();
    PC_TRY(apply_op(E, nsys, blocks, kslots, live, vs));
    E.t_op += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_op0).count();
    E.expansions += nA;
    auto Wv = [&](int a) { return E.W + (int64_t)active[a] * bs * vs; };
    auto dsm = [&](size_t off) { return reinterpret_cast<double2*>(E.dsmall + off); };
    // device scratch layout: [null coefficients][CGS2 coefficients, both passes][Gram][R^-1]
    std::vector<size_t> oz(nA), oh(nA), og(nA), oi(nA);
    size_t off = 0;
    for (int a = 0; a < nA; ++a) {
        oz[a] = off;
        off += (size_t)E.sp[active[a]].nz * bs;
    }
    const size_t h0 = off;
    for (int a = 0; a < nA; ++a) {
        oh[a] = off;
        off += (size_t)2 * (E.sp[active[a]].m_exp + bs) * bs;
    }
    for (int a = 0; a < nA; ++a) {
        og[a] = off;
        off += (size_t)bs * bs;
    }
    const size_t h1 = off;
    for (int a = 0; a < nA; ++a) {
        oi[a] = off;
        off += (size_t)bs * bs;
    }
    if (off > E.dsmall_cap) return fail(PC_EINVAL, "eigensolver: small-matrix scratch too small");
    {  // exact projection off the null bases
        std::vector<GramJob> gj;
        std::vector<UpdateJob> uj;
        for (int a = 0; a < nA; ++a) {
            Space& S = E.sp[active[a]];
            if (S.nz == 0) continue;
            gj.push_back({S.Z, S.nz, Wv(a), bs, grid_mat(g, S.block), dsm(oz[a])});
            uj.push_back({S.Z, S.nz, dsm(oz[a]), bs, Wv(a), -1.0, 1.0});
        }
        PC_TRY(gram_batch(E, gj));
        PC_TRY(update_batch(E, uj));
    }
    for (int rep = 0; rep < 2; ++rep) {  // CGS2 against the basis
        std::vector<GramJob> gj;
        std::vector<UpdateJob> uj;
        for (int a = 0; a < nA; ++a) {
            Space& S = E.sp[active[a]];
            const int nv = S.m_exp + bs;
            const size_t o = oh[a] + (size_t)rep * nv * bs;
            gj.push_back({S.V, nv, Wv(a), bs, grid_mat(g, S.block), dsm(o)});
            uj.push_back({S.V, nv, dsm(o), bs, Wv(a), -1.0, 1.0});
        }
        PC_TRY(gram_batch(E, gj));
        PC_TRY(update_batch(E, uj));
    }
    {
        std::vector<GramJob> gj;
        for (int a = 0; a < nA; ++a) {
            Space& S = E.sp[active[a]];
            gj.push_back({Wv(a), bs, Wv(a), bs, grid_mat(g, S.block), dsm(og[a])});
        }
        PC_TRY(gram_batch(E, gj));
    }
    std::vector<cd> hh;
    PC_TRY(to_host(E, E.dsmall + h0, h1 - h0, hh));
    // host: CGS2 coefficients, Cholesky factors of the new blocks
    std::vector<std::vector<cd>> hcoef(nA), Rtot(nA);
    std::vector<char> ok(nA, 1), second(nA, 0);
    std::vector<cd> hri(off - h1, cd(0, 0));
    for (int a = 0; a < nA; ++a) {
        Space& S = E.sp[active[a]];
        const int nv = S.m_exp + bs;
        hcoef[a].resize((size_t)nv * bs);
        for (size_t i = 0; i < hcoef[a].size(); ++i)
            hcoef[a][i] = hh[oh[a] - h0 + i] + hh[oh[a] - h0 + (size_t)nv * bs + i];
        std::vector<cd> G(hh.begin() + (og[a] - h0), hh.begin() + (og[a] - h0) + (size_t)bs * bs), R, Ri;
        if (!chol_upper(bs, G, R)) {
            ok[a] = 0;  // rank-deficient block: the one-space path below replaces it
            continue;
        }
        bool wc = true;
        for (int j = 0; j < bs && wc; ++j)
            for (int i = 0; i < j; ++i)
                if (std::abs(G[i + j * bs]) > 0.1 * std::sqrt(G[i + i * bs].real() * G[j + j * bs].real())) wc = false;
        second[a] = wc ? 0 : 1;
        if (wc) ++E.cholqr_single;
        upper_inverse(bs, R, Ri);
        std::copy(Ri.begin(), Ri.end(), hri.begin() + (oi[a] - h1));
        Rtot[a] = R;
    }
    PC_CUDA_TRY(cudaMemcpyAsync(E.dsmall + h1, hri.data(), sizeof(cd) * hri.size(), cudaMemcpyHostToDevice, E.s));
    {  // V[:, nv:nv+bs] = W R^-1
        std::vector<UpdateJob> uj;
        for (int a = 0; a < nA; ++a) {
            if (!ok[a]) continue;
            Space& S = E.sp[active[a]];
            const int nv = S.m_exp + bs;
            uj.push_back({Wv(a), bs, dsm(oi[a]), bs, S.V + (int64_t)nv * vs, 1.0, 0.0});
        }
        PC_TRY(update_batch(E, uj));
    }
    bool any2 = false;
    for (int a = 0; a < nA; ++a) any2 = any2 || (ok[a] && second[a]);
    if (any2) {  // second CholQR pass of the ill-conditioned blocks
        std::vector<GramJob> gj;
        for (int a = 0; a < nA; ++a) {
            if (!ok[a] || !second[a]) continue;
            Space& S = E.sp[active[a]];
            double2* Vn = S.V + (int64_t)(S.m_exp + bs) * vs;
            gj.push_back({Vn, bs, Vn, bs, grid_mat(g, S.block), dsm(og[a])});
        }
        PC_TRY(gram_batch(E, gj));
        PC_TRY(to_host(E, E.dsmall + h0, h1 - h0, hh));
        std::vector<UpdateJob> uj;
        for (int a = 0; a < nA; ++a) {
            if (!ok[a] || !second[a]) continue;
            std::vector<cd> G(hh.begin() + (og[a] - h0), hh.begin() + (og[a] - h0) + (size_t)bs * bs), R, Ri;
            if (!chol_upper(bs, G, R)) return fail(PC_ENOCONV, "eigensolver: Krylov block lost rank twice");
            upper_inverse(bs, R, Ri);
            std::copy(Ri.begin(), Ri.end(), hri.begin() + (oi[a] - h1));
            Rtot[a] = upper_mul(bs, R, Rtot[a]);
            Space& S = E.sp[active[a]];
            uj.push_back({S.V + (int64_t)(S.m_exp + bs) * vs, bs, dsm(oi[a]), bs, Wv(a), 1.0, 0.0});
        }
        PC_CUDA_TRY(cudaMemcpyAsync(E.dsmall + h1, hri.data(), sizeof(cd) * hri.size(), cudaMemcpyHostToDevice, E.s));
        PC_TRY(update_batch(E, uj));
        for (int a = 0; a < nA; ++a) {
            if (!ok[a] || !second[a]) continue;
            Space& S = E.sp[active[a]];
            PC_CUDA_TRY(cudaMemcpyAsync(S.V + (int64_t)(S.m_exp + bs) * vs, Wv(a), sizeof(double2) * bs * vs,
                                        cudaMemcpyDeviceToDevice, E.s));
        }
    }
    for (int a = 0; a < nA; ++a) {  // rank-deficient blocks, one space at a time
        if (ok[a]) continue;
        Space& S = E.sp[active[a]];
        const int nv = S.m_exp + bs;
        PC_TRY(cholqr2(E, S, Wv(a), bs, nv, Rtot[a], 0xC0FFEEull + 7919ull * (uint64_t)E.expansions + (uint64_t)a));
        PC_CUDA_TRY(cudaMemcpyAsync(S.V + (int64_t)nv * vs, Wv(a), sizeof(double2) * bs * vs,
                                    cudaMemcpyDeviceToDevice, E.s));
    }
    // Rayleigh-Ritz and the candidates for a true-residual check
    const auto t_rr0 = std::chrono::steady_clock::now();
    std::vector<int> chk, nck;
    for (int a = 0; a < nA; ++a) {
        Space& S = E.sp[active[a]];
        const int nv = S.m_exp + bs, c0 = S.m_exp;
        for (int j = 0; j < bs; ++j) {
            for (int i = 0; i < nv; ++i) S.H[i + (c0 + j) * ld] = hcoef[a][i + j * nv];
            for (int i = 0; i < bs; ++i) S.H[(nv + i) + (c0 + j) * ld] = Rtot[a][i + j * bs];
        }
        S.m_exp += bs;
        ritz(E, S);
        // residual estimates of the Ritz pairs: || H[m:m+bs, 0:m] s_i ||
        const int m = S.m_exp;
        int ncand = std::min(m, S.target + 1);
        std::vector<double> est(ncand);
        for (int i = 0; i < ncand; ++i) {
            double acc = 0;
            for (int r = 0; r < bs; ++r) {
                cd v = 0;
                for (int k = 0; k < m; ++k) v += S.H[(m + r) + k * ld] * S.S[k + i * m];
                acc += std::norm(v);
            }
            est[i] = std::sqrt(acc) / std::fabs(S.theta[i]);
        }
        int ntest = 0;
        while (ntest < ncand && est[ntest] < 1e-3) ++ntest;
        if (ntest >= std::min(S.target, m) && ntest > 0) {
            chk.push_back(active[a]);
            nck.push_back(ntest);
        }
    }
    const auto t_ck0 = std::chrono::steady_clock::now();
    E.t_ritz += std::chrono::duration<double>(t_ck0 - t_rr0).count();
    if (!chk.empty()) {
        std::vector<std::vector<double>> lam, rel;
        PC_TRY(check_pairs(E, chk, nck, lam, rel));
        E.t_check += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_ck0).count();
        for (size_t c = 0; c < chk.size(); ++c) {
            Space& S = E.sp[chk[c]];
            int nc = 0;
            while (nc < nck[c] && rel[c][nc] <= tol) ++nc;
            S.nconv = nc;
            if (nc >= S.target) {
                S.lam.assign(lam[c].begin(), lam[c].begin() + nc);
                S.res.assign(rel[c].begin(), rel[c].begin() + nc);
                S.done = true;
            }
        }
    }
    for (int a = 0; a < nA; ++a) {
        Space& S = E.sp[active[a]];
        if (!S.done && S.m_exp + bs > E.mmax) {
            int keep = std::max(S.target + bs, E.mmax / 2);
            keep = std::min(keep, S.m_exp - bs);
            PC_TRY(restart(E, S, keep));
        }
    }
    return PC_OK;
}

// Null basis of a space from the vanishing symbol blocks of its Bloch slot:
// T_sigma (e_m (x) e_alpha), M-orthonormalised.
static int build_null(Eigs& E, Space& S) {
    pc_grid* g = E.g;
    Precond* P = g->pre;
    S.nz = 0;
    if (!P || S.kslot >= (int)P->null_slot.size() || P->null_slot[S.kslot].empty()) return PC_OK;
    const std::vector<int>& modes = P->null_slot[S.kslot];
    const int nm = (int)modes.size();
    const int blocks_needed = S.block < 0 ? 4 : 1;
    S.nz = 3 * nm * blocks_needed;
    PC_TRY(E.alloc(&S.Z, (size_t)S.nz * S.vs));
    PC_CUDA_TRY(cudaMemsetAsync(S.Z, 0, sizeof(double2) * S.nz * S.vs, E.s));
    const int64_t nb = g->nb;
    double2* delta = E.T;  // [3 nb] mode-space vector, then block vector in E.T + 3 nb
    int col = 0;
    for (int bi = 0; bi < blocks_needed; ++bi) {
        const int b = S.block < 0 ? bi : S.block;
        for (int mi = 0; mi < nm; ++mi)
            for (int a = 0; a < 3; ++a, ++col) {
                PC_CUDA_TRY(cudaMemsetAsync(delta, 0, sizeof(double2) * 3 * nb, E.s));
                const double2 one = make_double2(1.0, 0.0);
                PC_CUDA_TRY(cudaMemcpyAsync(delta + a * nb + modes[mi], &one, sizeof(double2),
                                            cudaMemcpyHostToDevice, E.s));
                PC_CUDA_TRY(cudaStreamSynchronize(E.s));
                double2* dst = S.Z + (int64_t)col * S.vs;
                if (S.block < 0) {
                    PC_TRY(block_fourier(g, b, PC_C128, 1, delta, E.T + 3 * nb, E.s, S.kslot));
                    PC_TRY(launch_transfer(PC_C128, E.T + 3 * nb, dst, g->N, b, 1, E.s));
                } else {
                    PC_TRY(block_fourier(g, b, PC_C128, 1, delta, dst, E.s, S.kslot));
                }
            }
    }
    // M-orthonormalise the null columns
    std::vector<cd> G, R, Ri;
    PC_TRY(gram_m(E, S, S.Z, S.nz, S.Z, S.nz, E.dsmall));
    PC_TRY(to_host(E, E.dsmall, (size_t)S.nz * S.nz, G));
    if (!chol_upper(S.nz, G, R)) return fail(PC_ECUDA, "null basis is rank deficient");
    upper_inverse(S.nz, R, Ri);
    PC_TRY(gemm_nn_host(E, S.Z, S.nz, Ri, S.nz, E.AY, S.vs, kOne, kZero));
    PC_CUDA_TRY(cudaMemcpyAsync(S.Z, E.AY, sizeof(double2) * S.nz * S.vs, cudaMemcpyDeviceToDevice, E.s));
    return PC_OK;
}

// Lowest nev eigenvalues at nk Bloch vectors of one grid, solved in lockstep: the grid's slots
// 0 .. nk - 1 hold the vectors, every (slot, block) pair is a space, and one expansion advances all
// unfinished spaces together.  evals / block_of: [nk][nev]; info: nk entries (see pc_eigs_multi).
static int run_eigs(pc_grid* g, int nk, const double* kappas, int nev, double sigma, const pc_options* opt,
                    double* evals, void* evecs, int* block_of, pc_eigs_info* info) {
    if (g->matkind == 2 && opt->precision == PC_PREC_MIXED)
        return fail(PC_EINVAL, "pc_eigs: a nodewise material is solved in PC_PREC_FP64 only");
    auto t0 = std::chrono::steady_clock::now();
    PC_TRY(grid_set_kslots(g, nk, kappas));
    if (nk > 1 && !precond_multi_k(g))
        return fail(PC_EINVAL, "pc_eigs_multi: this grid size solves one Bloch vector at a time");
    if (!g->sol) g->sol = new Solver();
    Eigs E;
    E.g = g;
    E.o = opt;
    E.sigma = std::isnan(sigma) ? pc_default_sigma(g) : sigma;
    E.bs = std::max(1, std::min(opt->block_size, 16));
    {
        // the basis must hold a space's wanted pairs plus room to expand: at least its initial
        // target (its share of nev plus the guard pairs) + 2 blocks + 8
        const int share0 = opt->full_space ? nev : (nev + 3) / 4;
        const int target0 = share0 + (opt->full_space ? std::max(0, opt->guard) : 1);
        E.mmax = std::max({opt->max_basis, 3 * E.bs, target0 + 2 * E.bs + 8});
    }
    E.mcap = E.mmax + 2 * E.bs;
    const bool own_stream = opt->stream == nullptr;
    if (own_stream) PC_CUDA_TRY(cudaStreamCreateWithFlags(&E.s, cudaStreamNonBlocking));
    else E.s = (cudaStream_t)opt->stream;
    struct StreamGuard {
        cudaStream_t s;
        bool own;
        ~StreamGuard() {
            if (own) cudaStreamDestroy(s);
        }
    } sg{E.s, own_stream};

    const bool full = opt->full_space != 0;
    const int nper = full ? 1 : 4;  // spaces per Bloch vector
    const int nspace = nper * nk;
    const int64_t m = full ? g->n : g->nb, vs = 3 * m;
    if (opt->autotune) {
        // stencil launch shapes for the batches this solve runs (inner PCG, and the FP64 residual
        // refinement of the mixed path); tuned once per layout and cached
        const bool mixed = opt->precision == PC_PREC_MIXED;
        PC_TRY(autotune_layout(g, mixed ? PC_C64 : PC_C128, full, E.bs * nspace, E.s, opt->verbose));
        if (mixed) PC_TRY(autotune_layout(g, PC_C128, full, E.bs * nspace, E.s, opt->verbose));
    }
    E.sp.resize(nspace);
    const int share = full ? nev : (nev + 3) / 4;
    const int guard = std::max(0, opt->guard);
    const int ymax = std::max(E.mmax, share + guard + 16);
    // Ritz candidates checked per batched apply: every space's at once while that stays within
    // about 2 GB of vectors, else in groups
    const int64_t cols_2gb = std::max<int64_t>(1, ((int64_t)2 << 30) / (vs * (int64_t)sizeof(double2)));
    E.ycols = (int)std::max<int64_t>(ymax, std::min<int64_t>((int64_t)nspace * ymax, cols_2gb));
    PC_TRY(E.alloc(&E.W, (size_t)E.bs * nspace * vs));
    PC_TRY(E.alloc(&E.RHS, (size_t)E.bs * nspace * vs));
    PC_TRY(E.alloc(&E.MW, (size_t)std::max(E.bs * nspace, ymax) * vs));
    PC_TRY(E.alloc(&E.T, (size_t)std::max<int64_t>(E.mcap, 8) * vs));
    PC_TRY(E.alloc(&E.Y, (size_t)E.ycols * vs));
    PC_TRY(E.alloc(&E.AY, (size_t)std::max(E.ycols, ymax) * vs));
    PC_TRY(E.alloc(&E.dpart, (size_t)std::max(E.ycols * 5, E.bs * nspace) * 304));
    PC_TRY(E.alloc(&E.dscale, (size_t)E.bs * nspace));
    E.dsmall_cap = (size_t)2 * E.mcap * std::max(E.mcap, ymax) +
                   (size_t)nspace * (2 * E.mcap * E.bs + 2 * E.bs * E.bs + 48 * E.bs) +
                   (size_t)E.ycols * E.mcap;
    PC_TRY(E.alloc(&E.dsmall, E.dsmall_cap));
    E.gpart_cap = (size_t)2 * E.mcap * std::max(E.mcap, 16) * 160 + (size_t)nspace * 2 * E.mcap * E.bs * 160;
    PC_TRY(E.alloc(&E.gpart, E.gpart_cap));
    if (opt->precision == PC_PREC_MIXED) {
        PC_TRY(E.alloc(&E.X32, (size_t)2 * E.bs * nspace * vs));
        PC_TRY(E.alloc(&E.R32, (size_t)2 * E.bs * nspace * vs));
    }
    std::vector<int> zero_modes(nk, 0);
    for (int i = 0; i < nspace; ++i) {
        Space& S = E.sp[i];
        const int b = i % nper;
        S.block = full ? -1 : b;
        S.kslot = i / nper;
        S.m = m;
        S.vs = vs;
        S.target = share + (full ? guard : 1);
        PC_TRY(E.alloc(&S.V, (size_t)E.mcap * vs));
        S.H.assign((size_t)E.mcap * E.mcap, cd(0, 0));
        PC_TRY(build_null(E, S));
        zero_modes[S.kslot] += S.nz;
        // the start block depends on the block only, so every Bloch vector starts as a solve of
        // that vector alone would
        fill_random<<<ctas_for(E.bs * vs), 256, 0, E.s>>>(S.V, E.bs * vs, 0x5EED0000ull + (uint64_t)(b + 1) * 1000003ull);
        note_launch();
        PC_CUDA_TRY(cudaGetLastError());
        PC_TRY(project_null(E, S, S.V, E.bs));
        std::vector<cd> R;
        PC_TRY(cholqr2(E, S, S.V, E.bs, 0, R, 0xABCDEFull + b));
        S.m_exp = 0;
    }
    const int max_exp = std::max(1, opt->max_restarts) * std::max(1, (E.mmax / E.bs));
    int status = PC_OK;
    std::vector<std::vector<double>> merged(nk);
    std::vector<std::vector<int>> mblock(nk);
    std::vector<char> kdone(nk, 0);
    for (int outer = 0;; ++outer) {
        // merge the Bloch vectors whose spaces have all finished; reopen the ones that may hide a
        // lower eigenvalue
        for (int ks = 0; ks < nk; ++ks) {
            if (kdone[ks]) continue;
            bool all_done = true;
            for (int b = 0; b < nper; ++b) all_done = all_done && E.sp[ks * nper + b].done;
            if (!all_done) continue;
            std::vector<std::pair<double, int>> all;
            for (int b = 0; b < nper; ++b) {
                const Space& S = E.sp[ks * nper + b];
                for (double l : S.lam) all.push_back({l, S.block});
            }
            std::sort(all.begin(), all.end());
            bool ok = (int)all.size() >= nev;
            if (ok && !full) {
                const double cut = all[nev - 1].first;
                for (int b = 0; b < nper; ++b) {
                    Space& S = E.sp[ks * nper + b];
                    if (S.lam.empty() || S.lam.back() < cut) {  // may hide more eigenvalues below the cut
                        S.target += 2;
                        S.done = false;
                        ok = false;
                    }
                }
            } else if (!ok) {
                for (int b = 0; b < nper; ++b) {
                    E.sp[ks * nper + b].target += 2;
                    E.sp[ks * nper + b].done = false;
                }
            }
            if (ok) {
                for (int i = 0; i < nev; ++i) {
                    merged[ks].push_back(all[i].first);
                    mblock[ks].push_back(all[i].second);
                }
                kdone[ks] = 1;
            }
        }
        std::vector<int> active;
        for (int i = 0; i < nspace; ++i)
            if (!E.sp[i].done) active.push_back(i);
        if (active.empty()) break;  // every Bloch vector merged
        if (E.expansions >= max_exp * nspace) {
            status = PC_ENOCONV;
            break;
        }
        PC_TRY(expand(E, active, opt->tol));
        if (opt->verbose) {
            for (int i : active)
                std::fprintf(stderr, "[pc_eigs] k %d space %d m=%d target=%d nconv=%d done=%d\n", E.sp[i].kslot,
                             E.sp[i].block, E.sp[i].m_exp, E.sp[i].target, E.sp[i].nconv, (int)E.sp[i].done);
        }
    }
    if (opt->verbose)
        std::fprintf(stderr, "[pc_eigs] Bloch vectors=%d expansions=%d single-pass CholQR=%d solves=%d pcg=%lld "
                     "host syncs=%d; seconds in solves %.3f, Rayleigh-Ritz %.3f, residual checks %.3f, total %.3f\n",
                     nk, E.expansions, E.cholqr_single, E.solves, E.pcg_iters, E.syncs, E.t_op, E.t_ritz, E.t_check,
                     std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
    const double to_si = g->C0 / (g->rho0 * g->L * g->L);
    std::vector<double> maxres(nk, 0.0);
    for (int ks = 0; ks < nk; ++ks) {
        double* ev = evals + (size_t)ks * nev;
        int* bo = block_of ? block_of + (size_t)ks * nev : nullptr;
        if (kdone[ks]) {
            for (int i = 0; i < nev; ++i) {
                ev[i] = merged[ks][i] * to_si;
                if (bo) bo[i] = mblock[ks][i];
            }
            for (int b = 0; b < nper; ++b) {
                const Space& S = E.sp[ks * nper + b];
                for (size_t i = 0; i < S.res.size(); ++i)
                    if (std::find(merged[ks].begin(), merged[ks].end(), S.lam[i]) != merged[ks].end())
                        maxres[ks] = std::max(maxres[ks], S.res[i]);
            }
        } else {
            // best effort: whatever converged, then NaN
            std::vector<std::pair<double, int>> all;
            for (int b = 0; b < nper; ++b)
                for (double l : E.sp[ks * nper + b].lam) all.push_back({l, E.sp[ks * nper + b].block});
            std::sort(all.begin(), all.end());
            for (int i = 0; i < nev; ++i) {
                ev[i] = i < (int)all.size() ? all[i].first * to_si : NAN;
                if (bo) bo[i] = i < (int)all.size() ? all[i].second : -2;
            }
        }
    }
    if (evecs) {
        // recompute Ritz vectors for the merged values and write them in full-space layout,
        // [Bloch vector][nev][3][n]; the vectors of a Bloch vector that did not converge stay zero
        const size_t vn = (size_t)3 * g->n;
        PC_CUDA_TRY(cudaMemsetAsync(evecs, 0, sizeof(double2) * (size_t)nk * nev * vn, E.s));
        for (int ks = 0; ks < nk; ++ks) {
            if (!kdone[ks]) continue;
            double2* out = static_cast<double2*>(evecs) + (size_t)ks * nev * vn;
            std::vector<char> used(nev, 0);  // equal eigenvalues of one block get distinct slots
            for (int b = 0; b < nper; ++b) {
                Space& S = E.sp[ks * nper + b];
                ritz(E, S);
                const int ncand = (int)S.lam.size();
                if (ncand == 0) continue;
                const int mm = S.m_exp;
                std::vector<cd> Sk((size_t)mm * ncand);
                for (int j = 0; j < ncand; ++j)
                    for (int r = 0; r < mm; ++r) Sk[r + j * mm] = S.S[r + j * mm];
                PC_TRY(gemm_nn_host(E, S.V, mm, Sk, ncand, E.Y, S.vs, kOne, kZero));
                for (int j = 0; j < ncand; ++j) {
                    int slot = -1;
                    for (int q = 0; q < nev && slot < 0; ++q)
                        if (!used[q] && mblock[ks][q] == S.block && merged[ks][q] == S.lam[j]) slot = q;
                    if (slot < 0) continue;
                    used[slot] = 1;
                    double2* dst = out + (size_t)slot * vn;
                    if (S.block < 0)
                        PC_CUDA_TRY(cudaMemcpyAsync(dst, E.Y + (int64_t)j * S.vs, sizeof(double2) * S.vs,
                                                    cudaMemcpyDeviceToDevice, E.s));
                    else
                        PC_TRY(launch_transfer(PC_C128, E.Y + (int64_t)j * S.vs, dst, g->N, S.block, 1, E.s));
                }
            }
        }
    }
    PC_CUDA_TRY(cudaStreamSynchronize(E.s));
    if (info) {
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int ks = 0; ks < nk; ++ks) {
            pc_eigs_info& I = info[ks];
            I.status = kdone[ks] ? PC_OK : PC_ENOCONV;
            I.outer_iters = E.expansions;
            I.inner_solves = E.solves;
            I.pcg_iters = E.pcg_iters;
            I.max_pcg_iters = E.max_pcg;
            I.zero_modes = zero_modes[ks];
            I.max_rel_resid = maxres[ks];
            I.seconds = secs;
        }
    }
    if (status != PC_OK) return fail(status, "pc_eigs: outer iteration cap reached");
    return PC_OK;
}

}  // namespace pc

using namespace pc;

namespace pc {
void release_solver_state(pc_grid* g) {
    delete g->sol;
    g->sol = nullptr;
    delete g->pre;
    g->pre = nullptr;
}
}  // namespace pc

extern "C" {

int pc_options_default(pc_options* o) {
    if (!o) return fail(PC_EINVAL, "pc_options_default: null");
    o->tol = 1e-8;
    o->inner_tol = 1e-10;
    o->precision = PC_PREC_FP64;
    o->full_space = 0;
    o->block_size = 2;
    o->max_basis = 24;
    o->max_restarts = 60;
    o->inner_maxit = 400;
    o->guard = 3;
    o->verbose = 0;
    o->stream = nullptr;
    o->autotune = 0;
    o->precond_fp32 = 1;
    o->kbatch = 0;
    return PC_OK;
}

double pc_default_sigma(const pc_grid* g) {
    if (!g) return NAN;
    return -0.30 * g->sigma_cmax / g->sigma_rmax;
}

int pc_block_fourier(pc_grid* g, int block, int dtype, int inverse, const void* w, void* what, void* stream) {
    if (!g || !w || !what) return fail(PC_EINVAL, "pc_block_fourier: null argument");
    if (block < 0 || block > 3) return fail(PC_EINVAL, "pc_block_fourier: block must be 0..3");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_block_fourier: bad dtype");
    if (!g->k.set) return fail(PC_ESTATE, "pc_block_fourier: call pc_set_k first");
    return block_fourier(g, block, dtype, inverse ? 1 : 0, w, what, (cudaStream_t)stream);
}

int pc_block_precond(pc_grid* g, int block, int dtype, int fp32_transforms, double sigma, const void* r, void* z,
                     void* stream) {
    if (!g || !r || !z) return fail(PC_EINVAL, "pc_block_precond: null argument");
    if (block < -1 || block > 3) return fail(PC_EINVAL, "pc_block_precond: block must be -1..3");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_block_precond: bad dtype");
    if (!std::isfinite(sigma)) return fail(PC_EINVAL, "pc_block_precond: non-finite sigma");
    if (!g->k.set) return fail(PC_ESTATE, "pc_block_precond: call pc_set_k first");
    return precond_once(g, block, dtype, fp32_transforms != 0, sigma, r, z, (cudaStream_t)stream);
}

int pc_shift_invert_pcg(pc_grid* g, int block, int dtype, double sigma, const void* rhs, void* x, double tol, int maxit,
                        pc_pcg_info* info, void* stream) {
    if (!g || !rhs || !x) return fail(PC_EINVAL, "pc_shift_invert_pcg: null argument");
    if (block < -1 || block > 3) return fail(PC_EINVAL, "pc_shift_invert_pcg: block must be -1..3");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_shift_invert_pcg: bad dtype");
    if (!std::isfinite(sigma)) return fail(PC_EINVAL, "pc_shift_invert_pcg: non-finite sigma");
    if (!g->k.set) return fail(PC_ESTATE, "pc_shift_invert_pcg: call pc_set_k first");
    PcgResult r;
    int rc = pcg_solve(g, dtype, 1, &block, sigma, rhs, x, tol, maxit, &r, (cudaStream_t)stream);
    if (rc != PC_OK) return rc;
    PC_TRY(grid_device_status(g, (cudaStream_t)stream));
    if (info) {
        info->iters = r.iters;
        info->status = r.status;
        info->rel_resid = r.rel_resid;
    }
    if (r.status == PC_ENOCONV) return fail(PC_ENOCONV, "pc_shift_invert_pcg: iteration cap reached");
    if (r.status == PC_EBREAKDOWN) return fail(PC_EBREAKDOWN, "pc_shift_invert_pcg: p^H (A - sigma M) p <= 0");
    if (r.status == PC_ENAN) return fail(PC_ENAN, "pc_shift_invert_pcg: NaN in a reduction");
    return PC_OK;
}

static int check_eigs_args(const pc_grid* g, int nev, double sigma, const pc_options* o, const char* who) {
    if (nev < 1) return fail(PC_EINVAL, std::string(who) + ": nev must be >= 1");
    if (!(o->tol > 0) || !(o->inner_tol > 0)) return fail(PC_EINVAL, std::string(who) + ": tolerances must be positive");
    if (o->precision != PC_PREC_FP64 && o->precision != PC_PREC_MIXED)
        return fail(PC_EINVAL, std::string(who) + ": precision must be PC_PREC_FP64 or PC_PREC_MIXED");
    if (!std::isnan(sigma) && !std::isfinite(sigma)) return fail(PC_EINVAL, std::string(who) + ": bad sigma");
    const int64_t dim = o->full_space ? 3 * g->n : 3 * g->nb;
    if (nev > dim / 8) return fail(PC_EINVAL, std::string(who) + ": nev too large for this grid");
    return PC_OK;
}

int pc_eigs(pc_grid* g, const double kappa[3], int nev, double sigma, const pc_options* opt, double* evals,
            void* evecs, int* block_of, pc_eigs_info* info) {
    if (!g || !kappa || !evals) return fail(PC_EINVAL, "pc_eigs: null argument");
    pc_options def;
    pc_options_default(&def);
    const pc_options* o = opt ? opt : &def;
    PC_TRY(check_eigs_args(g, nev, sigma, o, "pc_eigs"));
    const int rc = run_eigs(g, 1, kappa, nev, sigma, o, evals, evecs, block_of, info);
    const int st = grid_device_status(g, (cudaStream_t)o->stream);
    return st != PC_OK ? st : rc;
}

int pc_eigs_multi(pc_grid* g, int nk, const double* kappas, int nev, double sigma, const pc_options* opt,
                  double* evals, void* evecs, int* block_of, pc_eigs_info* info) {
    if (!g || !kappas || !evals) return fail(PC_EINVAL, "pc_eigs_multi: null argument");
    if (nk < 1 || nk > kMaxKSlots) return fail(PC_EINVAL, "pc_eigs_multi: nk must be in 1..32");
    pc_options def;
    pc_options_default(&def);
    const pc_options* o = opt ? opt : &def;
    PC_TRY(check_eigs_args(g, nev, sigma, o, "pc_eigs_multi"));
    const int rc = run_eigs(g, nk, kappas, nev, sigma, o, evals, evecs, block_of, info);
    const int st = grid_device_status(g, (cudaStream_t)o->stream);
    return st != PC_OK ? st : rc;
}

int pc_eigs_multi_max(const pc_grid* g) {
    if (!g) return fail(PC_EINVAL, "pc_eigs_multi_max: null grid");
    const bool own = g->X == g->Y && g->Z == 2 * g->X && bloch_dft_supported(g->X, nullptr, nullptr);
    return own ? kMaxKSlots : 1;
}

}  // extern "C"
