// Adjoint (Hellmann-Feynman) kernel: gradients of eigenvalues with respect to the
// nodewise stiffness and density.
//
// For an eigenpair A x = lambda M x with x^H M x = 1 and A = B C B^H (Eq.
// discrete_GEP_main), a change dC, dM of the nodewise material moves the
// eigenvalue by d lambda = x^H (B dC B^H - lambda dM) x = sum_i e_i^H dC_i e_i -
// lambda sum_i rho'_i |x(i)|^2 with e = B^H x the Voigt strain at node i.  Per
// node and per independent entry of the symmetric 6x6 stiffness (upper
// triangle, Voigt order [11,22,33,23,13,12]):
//     d lambda / d C_i[p][q] = Re(conj(e_p) e_q) * (2 if p != q else 1),
//     d lambda / d rho_i      = -lambda sum_alpha |x_alpha(i)|^2.
// The strain is evaluated exactly as in the apply kernel (Bloch-phased backward
// body-diagonal differences, reconstruction, lattice mixing, engineering shear).
#include <cmath>

#include "pc_complex.cuh"
#include "pc_solver.h"

namespace pc {

struct GradParams {
    double Mmix[9];  // (A_hat^-1)_{s m} / (4 h_s)
    double ph[3][2];
    int X, Y, Z, N;
    int block;       // 0..3 or -1
    double scaleC;   // 1 / (rho0 L^2): hat strain products -> d lambda_SI / d C_SI
    double scaleR;   // 1 / rho0
};

__device__ __forceinline__ int wrapg(int v, int n, int& w) {
    w = 0;
    while (v < 0) { v += n; --w; }
    while (v >= n) { v -= n; ++w; }
    return v;
}

// One thread per node of the layout; loops over the vectors so that each output
// entry has a single writer (no atomics, deterministic).
__global__ void eig_grad_kernel(GradParams P, int nvec, const double2* __restrict__ X, const double* __restrict__ lam_si,
                                const double* __restrict__ w, double* __restrict__ dC, double* __restrict__ drho,
                                int64_t n_full) {
    const int64_t plane = (int64_t)P.X * P.Y, m = plane * P.Z;
    const bool full = P.block < 0;
    const int p12 = full ? 0 : (P.block >> 1), p13 = full ? 0 : (P.block & 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % P.X), b = (int)((t / P.X) % P.Y), k = (int)(t / plane);
        // full-grid index of this node
        int64_t l;
        if (full) l = t;
        else {
            const int64_t i = 2 * a + ((k + p13) & 1), j = 2 * b + ((k + p12 + p13) & 1);
            l = i + (int64_t)P.N * (j + (int64_t)P.N * k);
        }
        double g21[21];
        for (int q = 0; q < 21; ++q) g21[q] = 0.0;
        double gr = 0.0;
        // backward neighbour positions (same for every vector)
        int64_t nb[4];
        double2 ph[4];
        for (int ll = 0; ll < 4; ++ll) {
            const int s2 = (ll < 2) ? 1 : -1, s3 = (ll & 1) ? -1 : 1;
            int da, db;
            if (full) { da = -1; db = -s2; }
            else {
                const int i0 = (k + p13) & 1, j0 = (k + p12 + p13) & 1;
                da = i0 - 1;
                db = j0 - ((s2 + 1) >> 1);
            }
            int wa, wb, wk;
            const int aa = wrapg(a + da, P.X, wa), bb = wrapg(b + db, P.Y, wb), kk = wrapg(k - s3, P.Z, wk);
            nb[ll] = aa + (int64_t)P.X * (bb + (int64_t)P.Y * kk);
            double2 e = make_double2(1.0, 0.0);
            const int wv[3] = {wa, wb, wk};
            for (int s = 0; s < 3; ++s)
                for (int r = 0; r < (wv[s] < 0 ? -wv[s] : wv[s]); ++r)
                    e = cmul(e, make_double2(P.ph[s][0], wv[s] < 0 ? -P.ph[s][1] : P.ph[s][1]));
            ph[ll] = e;
        }
        for (int v = 0; v < nvec; ++v) {
            const double2* x = X + (int64_t)v * 3 * m;
            double2 H[3][3];
            double xx = 0.0;
            for (int al = 0; al < 3; ++al) {
                const double2 x0 = x[al * m + t];
                xx += x0.x * x0.x + x0.y * x0.y;
                double2 g[4];
                for (int ll = 0; ll < 4; ++ll) g[ll] = csub(cmul(ph[ll], x[al * m + nb[ll]]), x0);
                const double2 u = cadd(g[0], g[1]), vv = cadd(g[2], g[3]);
                const double2 ww = csub(g[0], g[1]), z = csub(g[2], g[3]);
                H[0][al] = cadd(u, vv);
                H[1][al] = csub(u, vv);
                H[2][al] = cadd(ww, z);
            }
            double2 G[3][3];  // G[m][alpha] = sum_s Mmix_{s m} H_{s alpha}  (the hat strain is i G)
            for (int mm = 0; mm < 3; ++mm)
                for (int al = 0; al < 3; ++al) {
                    double2 acc = cscale(P.Mmix[0 * 3 + mm], H[0][al]);
                    acc = cfma(P.Mmix[1 * 3 + mm], H[1][al], acc);
                    G[mm][al] = cfma(P.Mmix[2 * 3 + mm], H[2][al], acc);
                }
            double2 e[6];
            e[0] = G[0][0];
            e[1] = G[1][1];
            e[2] = G[2][2];
            e[3] = cadd(G[2][1], G[1][2]);
            e[4] = cadd(G[2][0], G[0][2]);
            e[5] = cadd(G[1][0], G[0][1]);
            const double wv = w[v] * P.scaleC;
            int q = 0;
            for (int p = 0; p < 6; ++p)
                for (int r = p; r < 6; ++r, ++q) {
                    const double re = e[p].x * e[r].x + e[p].y * e[r].y;
                    g21[q] += wv * (p == r ? re : 2.0 * re);
                }
            gr += -w[v] * lam_si[v] * xx * P.scaleR;
        }
        for (int q = 0; q < 21; ++q) dC[(int64_t)q * n_full + l] += g21[q];
        drho[l] += gr;
    }
}

}  // namespace pc

using namespace pc;

extern "C" int pc_eig_grad(pc_grid* g, int block, int nvec, const void* X, const double* lambdas, const double* weights,
                           double* dC, double* drho, void* stream) {
    if (!g || (!X && nvec > 0) || !lambdas || !weights || !dC || !drho)
        return fail(PC_EINVAL, "pc_eig_grad: null argument");
    if (block < -1 || block > 3) return fail(PC_EINVAL, "pc_eig_grad: block must be -1..3");
    if (nvec < 0 || nvec > 4096) return fail(PC_EINVAL, "pc_eig_grad: nvec must be in 0..4096");
    if (!g->k.set) return fail(PC_ESTATE, "pc_eig_grad: call pc_set_k (or pc_eigs) first");
    if (nvec == 0) return PC_OK;
    for (int v = 0; v < nvec; ++v)
        if (!std::isfinite(lambdas[v]) || !std::isfinite(weights[v]))
            return fail(PC_EINVAL, "pc_eig_grad: non-finite eigenvalue or weight");
    GradParams P;
    const double q = g->N / 4.0;
    for (int e = 0; e < 9; ++e) P.Mmix[e] = g->Ainv[e] * q;
    for (int l = 0; l < 3; ++l) {
        P.ph[l][0] = std::cos(g->k.phi[l]);
        P.ph[l][1] = std::sin(g->k.phi[l]);
    }
    P.N = g->N;
    P.block = block;
    P.X = block < 0 ? g->N : g->X;
    P.Y = block < 0 ? g->N : g->Y;
    P.Z = g->Z;
    P.scaleC = 1.0 / (g->rho0 * g->L * g->L);
    P.scaleR = 1.0 / g->rho0;
    cudaStream_t s = (cudaStream_t)stream;
    double *dl = nullptr, *dw = nullptr;
    PC_CUDA_TRY(cudaMallocAsync(&dl, sizeof(double) * 2 * nvec, s));
    dw = dl + nvec;
    PC_CUDA_TRY(cudaMemcpyAsync(dl, lambdas, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
    PC_CUDA_TRY(cudaMemcpyAsync(dw, weights, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
    const int64_t m = (int64_t)P.X * P.Y * P.Z;
    int64_t gb = (m + 127) / 128;
    if (gb > 16LL * device_sm_count()) gb = 16LL * device_sm_count();
    eig_grad_kernel<<<(int)gb, 128, 0, s>>>(P, nvec, static_cast<const double2*>(X), dl, dw, dC, drho, g->n);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());
    PC_CUDA_TRY(cudaFreeAsync(dl, s));
    return PC_OK;
}
