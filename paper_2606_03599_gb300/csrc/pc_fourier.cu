// Block Bloch Fourier transform T_sigma (Sec. 5.2) and the reference-medium
// preconditioner built on it (Sec. 5.3-5.4), plus the per-k Fourier symbol
// tables and the Fourier-SVD detection of zero-derivative modes (Sec. 6.2).
//
// For w on block b (quarter grid (a, b', k), i = 2a + i0(k), j = 2b' + j0(k)),
//   what(p,q,r) = (T_sigma^H w)(m) = n_b^-1/2 sum_nodes w e^{-i(i alpha_p + j beta_q + k gamma_r)}
// over the representatives p < N/2, q < N/2, r < N (Eqs. psi_pqr_unified,
// f_sigma_unified, Tsigma_unified: T_sigma^H w = 2 (T^H w) on the
// representatives for w supported on the block).  Splitting k = 2k' + par,
// i0 and j0 depend on par only, so
//   what(r)      = n_b^-1/2 [T_0(r) W_0(r) + T_1(r) W_1(r)]
//   what(r + Z2) = n_b^-1/2 [T_0(r) W_0(r) - T_1(r) W_1(r)],  r < Z2 = N/2,
// with T_par(p,q,r) = e^{-i par gamma_r} e^{-i (i0(par) alpha_p + j0(par) beta_q)}
// and W_par the plain 3D DFT over (k', b', a) of the parity-par planes after
// the pre-twiddle e^{-i (a phi1/X + b' phi2/Y + k' phi3/Z2)}.  The inverse runs
// the same steps backwards with conjugate factors.
//
// Preconditioner (Sec. 5.4 with a constant reference material): z = T_sigma
// diag_m (A_ref(m) - sigma rho_ref I_3)^-1 T_sigma^H r with
// A_ref(m) = B_hat(m) C_ref B_hat(m)^H (Eq. Bhat_xi_m_def), C_ref and rho_ref the
// volume averages of the material.  The symbol of the body-diagonal shifts is
// the same for every block (all points of an orbit share it), so one table of
// A_ref(m) serves all four blocks.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <vector>

#include "pc_complex.cuh"
#include "pc_fourier.h"
#include "pc_internal.h"

namespace pc {

// ------------------------------------------------------------------ device helpers
template <typename C> struct CR;
template <> struct CR<float2> { using R = float; };
template <> struct CR<double2> { using R = double; };

template <typename C> __device__ __forceinline__ C conjc(C a) { a.y = -a.y; return a; }
// Phase tables in the working precision of the transform (complex64 transforms read tables
// rounded once on the host: no per-use FP64 conversion, which runs on GB300's narrow FP64 pipe).
template <typename C> struct TabT;
template <> struct TabT<float2> { using T = float2; };
template <> struct TabT<double2> { using T = double2; };
template <typename C> __device__ __forceinline__ C ld(const typename TabT<C>::T* t, int i) { return t[i]; }

// Sum over the CTA (any blockDim multiple of 32 up to 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

template <typename C> __device__ __forceinline__ C cvt_c(float2 v);
template <typename C> __device__ __forceinline__ C cvt_c(double2 v);
template <> __device__ __forceinline__ float2 cvt_c<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 cvt_c<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt_c<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 cvt_c<double2>(float2 v) { return make_double2(v.x, v.y); }

// Pack: w[comp][k][b][a] * pre-twiddle -> W[comp][par][k'][b][a]; optional scale.  The work
// buffer W may be of lower precision than w (complex64 preconditioning of complex128 vectors).
template <typename C, typename Ci = C>
__global__ void fourier_pack(const Ci* __restrict__ w, C* __restrict__ W, const typename TabT<C>::T* __restrict__ twa,
                             const typename TabT<C>::T* __restrict__ twb, const typename TabT<C>::T* __restrict__ twk, int X, int Y,
                             int Z, int nsys, int64_t sys_stride_in, int64_t sys_stride_out, double scale,
                             int conj_tw) {
    const int64_t plane = (int64_t)X * Y, nb = plane * Z;
    const int64_t total = (int64_t)nsys * 3 * nb;
    using R = typename CR<C>::R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e32 = (uint32_t)e, nb32 = (uint32_t)nb;  // every index here is below 2^32
        const uint32_t q3 = e32 / nb32;  // s * 3 + comp
        const int64_t s = q3 / 3u;
        const int comp = (int)(q3 - 3u * (uint32_t)s);
        const int64_t t = e32 - q3 * nb32;
        int a, b, k;
        split3(t, X, Y, a, b, k);
        const int par = k & 1, kk = k >> 1;
        C tw = cmul(cmul(ld<C>(twa, a), ld<C>(twb, b)), ld<C>(twk, kk));
        if (conj_tw) tw = conjc(tw);
        C v = cmul(cvt_c<C>(w[s * sys_stride_in + comp * nb + t]), tw);
        v = cscale((R)scale, v);
        W[s * sys_stride_out + comp * nb + par * (nb / 2) + (int64_t)kk * plane + (int64_t)b * X + a] = v;
    }
}

// Unpack: W[comp][par][k'][b][a] * post-twiddle -> z[comp][k][b][a]; optional fused
// Re<r, z> partial sums per system (one partial per CTA, partial index blockIdx.x).
template <typename C>
__global__ void fourier_unpack(const C* __restrict__ W, C* __restrict__ z, const typename TabT<C>::T* __restrict__ twa,
                               const typename TabT<C>::T* __restrict__ twb, const typename TabT<C>::T* __restrict__ twk, int X, int Y,
                               int Z, int64_t sys_stride_in, int64_t sys_stride_out, double scale, int conj_tw) {
    const int64_t plane = (int64_t)X * Y, nb = plane * Z;
    const int s = blockIdx.y;
    using R = typename CR<C>::R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * nb;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)((uint32_t)e / (uint32_t)nb);
        const int64_t t = e - comp * nb;
        int a, b, k;
        split3(t, X, Y, a, b, k);
        const int par = k & 1, kk = k >> 1;
        C tw = cmul(cmul(ld<C>(twa, a), ld<C>(twb, b)), ld<C>(twk, kk));
        if (conj_tw) tw = conjc(tw);
        C v = W[s * sys_stride_in + comp * nb + par * (nb / 2) + (int64_t)kk * plane + (int64_t)b * X + a];
        z[s * sys_stride_out + e] = cscale((R)scale, cmul(v, tw));
    }
}

// Unpack with fused partial sums of Re<r_s, z_s> (one partial per CTA) and per-system skip flags.
// z and r (type Co) may be of higher precision than the work buffer W.
template <typename C, typename Co = C>
__global__ void fourier_unpack_dot(const C* __restrict__ W, Co* __restrict__ z, const Co* __restrict__ r,
                                   const typename TabT<C>::T* __restrict__ twa, const typename TabT<C>::T* __restrict__ twb,
                                   const typename TabT<C>::T* __restrict__ twk, int X, int Y, int Z, int64_t sys_stride,
                                   const int* __restrict__ skip, double* __restrict__ part, int npart) {
    const int64_t plane = (int64_t)X * Y, nb = plane * Z;
    const int s = blockIdx.y;
    if (skip && skip[s]) return;
    using Ro = decltype(z[0].x);
    Ro acc = 0;  // per-thread sums in the output precision (complex64: FP32), FP64 across threads
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * nb;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)((uint32_t)e / (uint32_t)nb);
        const int64_t t = e - comp * nb;
        int a, b, k;
        split3(t, X, Y, a, b, k);
        const int par = k & 1, kk = k >> 1;
        C tw = conjc(cmul(cmul(ld<C>(twa, a), ld<C>(twb, b)), ld<C>(twk, kk)));
        const Co v = cvt_c<Co>(
            cmul(W[s * sys_stride + comp * nb + par * (nb / 2) + (int64_t)kk * plane + (int64_t)b * X + a], tw));
        z[s * sys_stride + e] = v;
        const Co rv = r[s * sys_stride + e];
        acc = cdotre(rv, v, acc);
    }
    const double sum = block_sum((double)acc);
    if (threadIdx.x == 0) part[(int64_t)s * npart + blockIdx.x] = sum;
}

// Twiddle T_par(p,q,r) for r < Z2.
template <typename C>
__device__ __forceinline__ C t_par(const typename TabT<C>::T* ea, const typename TabT<C>::T* eb, const typename TabT<C>::T* eg, int p, int q, int r,
                                   int par, int p12, int p13) {
    const int i0 = (par + p13) & 1, j0 = (par + p12 + p13) & 1;
    C t = make_c<C>(1, 0);
    if (par) t = ld<C>(eg, r);
    if (i0) t = cmul(t, ld<C>(ea, p));
    if (j0) t = cmul(t, ld<C>(eb, q));
    return t;
}

// Butterfly between parity halves: forward (W -> what, mode order [comp][r][q][p]) or inverse.
template <typename C>
__global__ void fourier_butterfly(const C* __restrict__ in, C* __restrict__ out, const typename TabT<C>::T* __restrict__ ea,
                                  const typename TabT<C>::T* __restrict__ eb, const typename TabT<C>::T* __restrict__ eg, int X, int Y,
                                  int Z, int p12, int p13, double scale, int inverse) {
    const int64_t plane = (int64_t)X * Y, nb = plane * Z, half = nb / 2;
    using R = typename CR<C>::R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * half;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)((uint32_t)e / (uint32_t)half);
        const int64_t u = e - comp * half;
        int p, q, r;
        split3(u, X, Y, p, q, r);
        const C T0 = t_par<C>(ea, eb, eg, p, q, r, 0, p12, p13);
        const C T1 = t_par<C>(ea, eb, eg, p, q, r, 1, p12, p13);
        const int64_t i_lo = comp * nb + (int64_t)r * plane + (int64_t)q * X + p;  // mode r (or parity 0 plane)
        const int64_t i_hi = i_lo + half;                                          // mode r+Z2 (or parity 1)
        if (!inverse) {
            C w0 = cmul(T0, in[i_lo]), w1 = cmul(T1, in[i_hi]);
            out[i_lo] = cscale((R)scale, cadd(w0, w1));
            out[i_hi] = cscale((R)scale, csub(w0, w1));
        } else {
            C lo = in[i_lo], hi = in[i_hi];
            out[i_lo] = cscale((R)scale, cmul(conjc(T0), cadd(lo, hi)));
            out[i_hi] = cscale((R)scale, cmul(conjc(T1), csub(lo, hi)));
        }
    }
}

// Preconditioner core on the parity-split spectrum W (in place, one CTA row per system):
// forward butterfly, per-mode (A_ref(m) - sigma rho_ref)^-1 in the working precision R,
// inverse butterfly.  Aref holds 9 reals per mode (diag, then a01, a02, a12 as re/im).
template <typename C, typename R>
__global__ void precond_symbol_solve(C* __restrict__ W, const R* __restrict__ Aref, const typename TabT<C>::T* __restrict__ ea,
                                     const typename TabT<C>::T* __restrict__ eb, const typename TabT<C>::T* __restrict__ eg,
                                     const int* __restrict__ sys_block, const int* __restrict__ skip, int X, int Y,
                                     int Z, int64_t sys_stride, double shift_rho_d, double scale_d) {
    const int s = blockIdx.y;
    if (skip && skip[s]) return;
    const int b = sys_block[s];
    const int p12 = b >> 1, p13 = b & 1;
    const int64_t plane = (int64_t)X * Y, nb = plane * Z, half = nb / 2;
    const R shift_rho = (R)shift_rho_d, scale = (R)scale_d;
    C* Ws = W + s * sys_stride;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < half; u += (int64_t)gridDim.x * blockDim.x) {
        int p, q, r;
        split3(u, X, Y, p, q, r);
        const C T0 = t_par<C>(ea, eb, eg, p, q, r, 0, p12, p13);
        const C T1 = t_par<C>(ea, eb, eg, p, q, r, 1, p12, p13);
        C lo[3], hi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C w0 = cmul(T0, Ws[c * nb + u]), w1 = cmul(T1, Ws[c * nb + half + u]);
            lo[c] = cadd(w0, w1);
            hi[c] = csub(w0, w1);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t mode = u + h * half;  // [r][q][p] with r in [0, Z)
            const R* A = Aref + 9 * mode;
            // Hermitian [[d0,a01,a02],[a01*,d1,a12],[a02*,a12*,d2]] shifted by -sigma rho_ref; solve by its adjugate
            const R d0 = A[0] + shift_rho, d1 = A[1] + shift_rho, d2 = A[2] + shift_rho;
            const C a01 = make_c<C>(A[3], A[4]), a02 = make_c<C>(A[5], A[6]), a12 = make_c<C>(A[7], A[8]);
            const R c00 = d1 * d2 - (a12.x * a12.x + a12.y * a12.y);
            const R c11 = d0 * d2 - (a02.x * a02.x + a02.y * a02.y);
            const R c22 = d0 * d1 - (a01.x * a01.x + a01.y * a01.y);
            const C c01 = csub(cmul(a02, conjc(a12)), cscale(d2, a01));  // adj(0,1)
            const C c02 = csub(cmul(a01, a12), cscale(d1, a02));         // adj(0,2)
            const C c12 = csub(cmul(conjc(a01), a02), cscale(d0, a12));  // adj(1,2)
            const R det = d0 * c00 + (a01.x * c01.x + a01.y * c01.y) + (a02.x * c02.x + a02.y * c02.y);
            const R inv = scale / det;
            C* v = h ? hi : lo;
            const C v0 = v[0], v1 = v[1], v2 = v[2];
            C z0 = cadd(cadd(cscale(c00, v0), cmul(c01, v1)), cmul(c02, v2));
            C z1 = cadd(cadd(cmul(conjc(c01), v0), cscale(c11, v1)), cmul(c12, v2));
            C z2 = cadd(cadd(cmul(conjc(c02), v0), cmul(conjc(c12), v1)), cscale(c22, v2));
            v[0] = cscale(inv, z0);
            v[1] = cscale(inv, z1);
            v[2] = cscale(inv, z2);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Ws[c * nb + u] = cmul(conjc(T0), cadd(lo[c], hi[c]));
            Ws[c * nb + half + u] = cmul(conjc(T1), csub(lo[c], hi[c]));
        }
    }
}

__global__ void table_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// Reference symbol A_ref(m) = B_hat(m) C_ref B_hat(m)^H for every mode (p, q, r), r < Z, and
// the zero-derivative flag ||eta(m)|| == 0 (B_hat(m) = 0: rank-0 symbol, Sec. 6.2).
__global__ void symbol_table(double* __restrict__ Aref, int* __restrict__ nnull, int* __restrict__ null_modes,
                             const double2* __restrict__ ea, const double2* __restrict__ eb,
                             const double2* __restrict__ egf, SymbolParams sp) {
    const int X = sp.X, Y = sp.Y, Z = sp.Z;
    const int64_t plane = (int64_t)X * Y, total = plane * Z;
    for (int64_t mode = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; mode < total;
         mode += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(mode % X), q = (int)((mode / X) % Y), r = (int)(mode / plane);
        // s_l = e^{i (alpha_p + s2 beta_q + s3 gamma_r)}  (Eq. Sd_phase_maintext); tables hold e^{-i .}
        const double2 a = make_double2(ea[p].x, -ea[p].y);
        const double2 bq = make_double2(eb[q].x, -eb[q].y);
        const double2 g = make_double2(egf[r].x, -egf[r].y);
        auto cm = [](double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); };
        auto cj = [](double2 x) { return make_double2(x.x, -x.y); };
        double2 s[4];
        s[0] = cm(cm(a, bq), g);
        s[1] = cm(cm(a, bq), cj(g));
        s[2] = cm(cm(a, cj(bq)), g);
        s[3] = cm(cm(a, cj(bq)), cj(g));
        const double sg[3][4] = {{1, 1, 1, 1}, {1, 1, -1, -1}, {1, -1, 1, -1}};
        double2 delta[3];
        for (int t = 0; t < 3; ++t) {
            double2 acc = make_double2(0, 0);
            for (int l = 0; l < 4; ++l) {
                acc.x += sg[t][l] * (s[l].x - 1.0);
                acc.y += sg[t][l] * s[l].y;
            }
            delta[t] = make_double2(acc.x * sp.q, acc.y * sp.q);  // (1/(4 h_s)) sum_l c_{s l}(s_l - 1)
        }
        // eta_m = sum_s Ainv_{s m} (-i delta_s)
        double2 eta[3];
        double en = 0;
        for (int m = 0; m < 3; ++m) {
            double2 acc = make_double2(0, 0);
            for (int t = 0; t < 3; ++t) {
                acc.x += sp.Ainv[t * 3 + m] * delta[t].y;   // -i (x + iy) = y - i x
                acc.y += -sp.Ainv[t * 3 + m] * delta[t].x;
            }
            eta[m] = acc;
            en = fmax(en, fabs(acc.x) + fabs(acc.y));
        }
        // B_hat (3x6) rows: [e1 0 0 0 e3 e2], [0 e2 0 e3 0 e1], [0 0 e3 e2 e1 0]
        double2 B[3][6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 6; ++j) B[i][j] = make_double2(0, 0);
        B[0][0] = eta[0]; B[0][4] = eta[2]; B[0][5] = eta[1];
        B[1][1] = eta[1]; B[1][3] = eta[2]; B[1][5] = eta[0];
        B[2][2] = eta[2]; B[2][3] = eta[1]; B[2][4] = eta[0];
        // T = B C  (3x6), A = T B^H
        double2 T[3][6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 6; ++j) {
                double2 acc = make_double2(0, 0);
                for (int k = 0; k < 6; ++k) {
                    acc.x += B[i][k].x * sp.Cref[k * 6 + j];
                    acc.y += B[i][k].y * sp.Cref[k * 6 + j];
                }
                T[i][j] = acc;
            }
        double2 Am[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double2 acc = make_double2(0, 0);
                for (int k = 0; k < 6; ++k) acc = make_double2(acc.x + T[i][k].x * B[j][k].x + T[i][k].y * B[j][k].y,
                                                               acc.y + T[i][k].y * B[j][k].x - T[i][k].x * B[j][k].y);
                Am[i][j] = acc;
            }
        double* o = Aref + 9 * mode;
        o[0] = Am[0][0].x; o[1] = Am[1][1].x; o[2] = Am[2][2].x;
        o[3] = Am[0][1].x; o[4] = Am[0][1].y;
        o[5] = Am[0][2].x; o[6] = Am[0][2].y;
        o[7] = Am[1][2].x; o[8] = Am[1][2].y;
        if (en <= sp.null_tol) {
            int slot = atomicAdd(nnull, 1);
            if (slot < 64) null_modes[slot] = (int)mode;
        }
    }
}

int precond_partials(const pc_grid* g) {
    if (g->X == g->Y && g->Z == 2 * g->X && bloch_dft_supported(g->X, nullptr, nullptr))
        return std::max(bloch_dft_partials(g->X), unpack_ctas(3 * g->nb));
    return unpack_ctas(3 * g->nb);
}

// CTAs per system of the unpack-with-dot kernel (also the count of its partial sums).
int unpack_ctas(int64_t vs) {
    int64_t g = (vs + 1023) / 1024;
    if (g > 304) g = 304;
    return (int)(g < 1 ? 1 : g);
}

static int nblocks_for(int64_t work) {
    int64_t g = (work + 255) / 256;
    const int64_t cap = 8LL * device_sm_count();
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace pc

Precond::~Precond() {
    for (auto& pl : plans) cufftDestroy(pl.h);
    cudaFree(d_tabs);
    cudaFree(d_tabs32);
    cudaFree(d_Aref);
    cudaFree(d_Aref32);
    cudaFree(d_null);
    cudaFree(d_work);
    cudaFree(d_wn);
    cudaFree(d_wn32);
    cudaFree(d_blockids);
}

namespace pc {
// ------------------------------------------------------------------ host side

int precond_create(pc_grid* g) {
    if (g->pre) return PC_OK;
    Precond* P = new Precond();
    g->pre = P;
    const int X = g->X, Y = g->Y, Z = g->Z;
    // tables per slot: ea[X], eb[Y], egh[Z2], egf[Z], twa[X], twb[Y], twk[Z2]
    P->tab_len = X + Y + Z / 2 + Z + X + Y + Z / 2;
    // roots of the own quarter-grid DFT (Bloch-independent) and the block ids
    P->own_dft = g->X == g->Y && g->Z == 2 * g->X && bloch_dft_supported(g->X, nullptr, nullptr);
    {
        const int n = g->X;
        std::vector<double2> w(n);
        std::vector<float2> w32(n);
        for (int j = 0; j < n; ++j) {
            w[j] = make_double2(std::cos(2 * M_PI * j / n), -std::sin(2 * M_PI * j / n));
            w32[j] = make_float2((float)w[j].x, (float)w[j].y);
        }
        PC_CUDA_TRY(cudaMalloc(&P->d_wn, sizeof(double2) * n));
        PC_CUDA_TRY(cudaMalloc(&P->d_wn32, sizeof(float2) * n));
        PC_CUDA_TRY(cudaMemcpy(P->d_wn, w.data(), sizeof(double2) * n, cudaMemcpyHostToDevice));
        PC_CUDA_TRY(cudaMemcpy(P->d_wn32, w32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
        P->wn = P->d_wn;
        P->wn32 = P->d_wn32;
        const int ids[4] = {0, 1, 2, 3};
        PC_CUDA_TRY(cudaMalloc(&P->d_blockids, sizeof(ids)));
        PC_CUDA_TRY(cudaMemcpy(P->d_blockids, ids, sizeof(ids), cudaMemcpyHostToDevice));
    }
    // reference medium: volume averages of rho and C over the grid
    const double th = g->mean_theta;
    P->rho_ref = (1 - th) * g->rhohat[0] + th * g->rhohat[1];
    for (int e = 0; e < 36; ++e) P->Cref[e] = (1 - th) * g->Chat[0][e] + th * g->Chat[1][e];
    return PC_OK;
}

bool precond_multi_k(const pc_grid* g) { return g->pre != nullptr && g->pre->own_dft; }

// Room for nk slots of tables (grown, never shrunk); the slot-0 pointers follow the allocation.
static int precond_slots(pc_grid* g, int nk) {
    Precond* P = g->pre;
    if (P->nslots < nk) {
        cudaFree(P->d_tabs);
        cudaFree(P->d_tabs32);
        cudaFree(P->d_Aref);
        cudaFree(P->d_Aref32);
        cudaFree(P->d_null);
        P->d_tabs = nullptr;
        P->d_tabs32 = nullptr;
        P->d_Aref = nullptr;
        P->d_Aref32 = nullptr;
        P->d_null = nullptr;
        P->nslots = 0;
        PC_CUDA_TRY(cudaMalloc(&P->d_tabs, sizeof(double2) * P->tab_len * nk));
        PC_CUDA_TRY(cudaMalloc(&P->d_tabs32, sizeof(float2) * P->tab_len * nk));
        PC_CUDA_TRY(cudaMalloc(&P->d_Aref, sizeof(double) * 9 * g->nb * nk));
        PC_CUDA_TRY(cudaMalloc(&P->d_Aref32, sizeof(float) * 9 * g->nb * nk));
        PC_CUDA_TRY(cudaMalloc(&P->d_null, sizeof(int) * 65 * nk));
        P->nslots = nk;
    }
    const int X = g->X, Y = g->Y, Z2 = g->Z / 2, Z = g->Z;
    P->ea32 = P->d_tabs32;
    P->eb32 = P->ea32 + X;
    P->egh32 = P->eb32 + Y;
    P->twa32 = P->egh32 + Z2 + Z;
    P->twb32 = P->twa32 + X;
    P->twk32 = P->twb32 + Y;
    P->ea = P->d_tabs;
    P->eb = P->ea + X;
    P->egh = P->eb + Y;
    P->egf = P->egh + Z2;
    P->twa = P->egf + Z;
    P->twb = P->twa + X;
    P->twk = P->twb + Y;
    return PC_OK;
}

// Phase tables, reference symbol and null modes of one slot.
static int precond_fill_slot(pc_grid* g, int slot) {
    Precond* P = g->pre;
    const int X = g->X, Y = g->Y, Z = g->Z, Z2 = Z / 2, N = g->N;
    const size_t to = (size_t)slot * P->tab_len;
    std::vector<double2> h(P->tab_len);
    double2* ea = h.data();
    double2* eb = ea + X;
    double2* egh = eb + Y;
    double2* egf = egh + Z2;
    double2* twa = egf + Z;
    double2* twb = twa + X;
    double2* twk = twb + Y;
    const double* phi = g->ks[slot].phi;
    auto ex = [](double ang) { return make_double2(std::cos(ang), -std::sin(ang)); };  // e^{-i ang}
    for (int p = 0; p < X; ++p) ea[p] = ex((phi[0] + 2 * M_PI * p) / N);
    for (int q = 0; q < Y; ++q) eb[q] = ex((phi[1] + 2 * M_PI * q) / N);
    for (int r = 0; r < Z2; ++r) egh[r] = ex((phi[2] + 2 * M_PI * r) / N);
    for (int r = 0; r < Z; ++r) egf[r] = ex((phi[2] + 2 * M_PI * r) / N);
    for (int a = 0; a < X; ++a) twa[a] = ex(a * phi[0] / X);
    for (int b = 0; b < Y; ++b) twb[b] = ex(b * phi[1] / Y);
    for (int k = 0; k < Z2; ++k) twk[k] = ex(k * phi[2] / Z2);
    PC_CUDA_TRY(cudaMemcpy(P->d_tabs + to, h.data(), sizeof(double2) * P->tab_len, cudaMemcpyHostToDevice));
    std::vector<float2> h32(P->tab_len);
    for (int i = 0; i < P->tab_len; ++i) h32[i] = make_float2((float)h[i].x, (float)h[i].y);
    PC_CUDA_TRY(cudaMemcpy(P->d_tabs32 + to, h32.data(), sizeof(float2) * P->tab_len, cudaMemcpyHostToDevice));
    SymbolParams sp;
    sp.X = X; sp.Y = Y; sp.Z = Z;
    sp.q = N / 4.0;
    for (int e = 0; e < 9; ++e) sp.Ainv[e] = g->Ainv[e];
    for (int e = 0; e < 36; ++e) sp.Cref[e] = P->Cref[e];
    sp.null_tol = 1e-9;
    double* aref = P->d_Aref + (size_t)slot * 9 * g->nb;
    int* dn = P->d_null + (size_t)slot * 65;
    PC_CUDA_TRY(cudaMemset(dn, 0, sizeof(int) * 65));
    symbol_table<<<nblocks_for(g->nb), 256>>>(aref, dn, dn + 1, P->ea + to, P->eb + to, P->egf + to, sp);
    note_launch();
    table_to_f32<<<nblocks_for(9 * g->nb), 256>>>(aref, P->d_Aref32 + (size_t)slot * 9 * g->nb, 9 * g->nb);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());
    int hn[65];
    PC_CUDA_TRY(cudaMemcpy(hn, dn, sizeof(hn), cudaMemcpyDeviceToHost));
    P->null_slot[slot].assign(hn + 1, hn + 1 + (hn[0] < 64 ? hn[0] : 64));
    return PC_OK;
}

int precond_set_k(pc_grid* g) {
    PC_TRY(precond_create(g));
    Precond* P = g->pre;
    PC_TRY(precond_slots(g, g->nk));
    P->null_slot.assign(g->nk, std::vector<int>());
    for (int slot = 0; slot < g->nk; ++slot) PC_TRY(precond_fill_slot(g, slot));
    P->null_modes = P->null_slot[0];
    return PC_OK;
}

static int get_plan(Precond* P, pc_grid* g, int dtype, int nsys, cufftHandle* out) {
    for (auto& pl : P->plans)
        if (pl.dtype == dtype && pl.nsys == nsys) {
            *out = pl.h;
            return PC_OK;
        }
    cufftHandle h;
    int n[3] = {g->Z / 2, g->Y, g->X};
    const int batch = 6 * nsys;
    const int dist = (g->Z / 2) * g->Y * g->X;
    cufftResult rc = cufftPlanMany(&h, 3, n, nullptr, 1, dist, nullptr, 1, dist,
                                   dtype == PC_C64 ? CUFFT_C2C : CUFFT_Z2Z, batch);
    if (rc != CUFFT_SUCCESS) return fail(PC_ECUDA, "cufftPlanMany failed (" + std::to_string((int)rc) + ")");
    P->plans.push_back({dtype, nsys, h});
    *out = h;
    return PC_OK;
}

static int exec_fft(cufftHandle h, int dtype, void* data, int dir, cudaStream_t s) {
    cufftSetStream(h, s);
    cufftResult rc;
    if (dtype == PC_C64)
        rc = cufftExecC2C(h, (cufftComplex*)data, (cufftComplex*)data, dir);
    else
        rc = cufftExecZ2Z(h, (cufftDoubleComplex*)data, (cufftDoubleComplex*)data, dir);
    if (rc != CUFFT_SUCCESS) return fail(PC_ECUDA, "cufftExec failed (" + std::to_string((int)rc) + ")");
    return PC_OK;
}

int precond_workspace(pc_grid* g, int dtype, int nsys, void** W) {
    Precond* P = g->pre;
    const size_t need = (size_t)nsys * 3 * g->nb * (dtype == PC_C64 ? 8 : 16);
    if (P->work_bytes < need) {
        cudaFree(P->d_work);
        P->d_work = nullptr;
        P->work_bytes = 0;
        PC_CUDA_TRY(cudaMalloc(&P->d_work, need));
        P->work_bytes = need;
    }
    *W = P->d_work;
    return PC_OK;
}

// z_s = P_ref r_s for nsys systems (vectors contiguous with stride 3 n_b), blocks in d_sys_block.
int precond_apply(pc_grid* g, int dtype, int nsys, const void* r, void* z, const int* d_sys_block,
                  const int* d_skip, double sigma, cudaStream_t s, double* d_part, int* npart_out, bool fp32_inner,
                  const int* d_sys_k) {
    if (!g->pre || !g->k.set) return fail(PC_ESTATE, "preconditioner: pc_set_k first");
    if (d_sys_k && !g->pre->own_dft) return fail(PC_EINVAL, "preconditioner: several Bloch slots need the own DFT");
    Precond* P = g->pre;
    const bool lower = dtype == PC_C128 && fp32_inner;  // complex128 vectors, complex64 transforms
    const int wdt = lower ? PC_C64 : dtype;
    void* W;
    PC_TRY(precond_workspace(g, wdt, nsys, &W));
    if (P->own_dft) {
        if (lower && !d_part) return fail(PC_EINVAL, "preconditioner: complex64 transforms need the fused dot");
        PC_TRY(own_precond(g->X, wdt, dtype, nsys, r, z, W, P, d_sys_block, d_sys_k, d_skip, -sigma * P->rho_ref,
                           1.0 / (double)g->nb, d_part, s));
        if (npart_out) *npart_out = bloch_dft_partials(g->X);
        return PC_OK;
    }
    cufftHandle plan;
    PC_TRY(get_plan(P, g, wdt, nsys, &plan));
    const int64_t vs = 3 * g->nb;
    const double inv_nb = 1.0 / (double)g->nb;
    const double shift_rho = -sigma * P->rho_ref;
    if (lower) {
        fourier_pack<float2, double2><<<nblocks_for(nsys * vs), 256, 0, s>>>(
            (const double2*)r, (float2*)W, P->twa32, P->twb32, P->twk32, g->X, g->Y, g->Z, nsys, vs, vs, 1.0, 0);
        note_launch();
        PC_TRY(exec_fft(plan, wdt, W, CUFFT_FORWARD, s));
        precond_symbol_solve<float2, float><<<dim3(nblocks_for(g->nb / 2), nsys), 256, 0, s>>>(
            (float2*)W, P->d_Aref32, P->ea32, P->eb32, P->egh32, d_sys_block, d_skip, g->X, g->Y, g->Z, vs, shift_rho, inv_nb);
        note_launch();
        PC_TRY(exec_fft(plan, wdt, W, CUFFT_INVERSE, s));
        if (!d_part) return fail(PC_EINVAL, "preconditioner: complex64 transforms need the fused dot");
        fourier_unpack_dot<float2, double2><<<dim3(unpack_ctas(vs), nsys), 256, 0, s>>>(
            (const float2*)W, (double2*)z, (const double2*)r, P->twa32, P->twb32, P->twk32, g->X, g->Y, g->Z, vs, d_skip,
            d_part, unpack_ctas(vs));
        note_launch();
    } else if (dtype == PC_C64) {
        fourier_pack<float2><<<nblocks_for(nsys * vs), 256, 0, s>>>((const float2*)r, (float2*)W, P->twa32, P->twb32,
                                                                  P->twk32, g->X, g->Y, g->Z, nsys, vs, vs, 1.0, 0);
        note_launch();
        PC_TRY(exec_fft(plan, dtype, W, CUFFT_FORWARD, s));
        precond_symbol_solve<float2, float><<<dim3(nblocks_for(g->nb / 2), nsys), 256, 0, s>>>(
            (float2*)W, P->d_Aref32, P->ea32, P->eb32, P->egh32, d_sys_block, d_skip, g->X, g->Y, g->Z, vs, shift_rho, inv_nb);
        note_launch();
        PC_TRY(exec_fft(plan, dtype, W, CUFFT_INVERSE, s));
        if (d_part)
            { fourier_unpack_dot<float2><<<dim3(unpack_ctas(vs), nsys), 256, 0, s>>>(
                (const float2*)W, (float2*)z, (const float2*)r, P->twa32, P->twb32, P->twk32, g->X, g->Y, g->Z, vs, d_skip,
                d_part, unpack_ctas(vs)); note_launch(); }
        else
            { fourier_unpack<float2><<<dim3(nblocks_for(vs), nsys), 256, 0, s>>>((const float2*)W, (float2*)z, P->twa32,
                                                                              P->twb32, P->twk32, g->X, g->Y, g->Z, vs,
                                                                              vs, 1.0, 1); note_launch(); }
    } else {
        fourier_pack<double2><<<nblocks_for(nsys * vs), 256, 0, s>>>((const double2*)r, (double2*)W, P->twa,
                                                                    P->twb, P->twk, g->X, g->Y, g->Z, nsys, vs, vs,
                                                                    1.0, 0);
        note_launch();
        PC_TRY(exec_fft(plan, dtype, W, CUFFT_FORWARD, s));
        precond_symbol_solve<double2, double><<<dim3(nblocks_for(g->nb / 2), nsys), 256, 0, s>>>(
            (double2*)W, P->d_Aref, P->ea, P->eb, P->egh, d_sys_block, d_skip, g->X, g->Y, g->Z, vs, shift_rho,
            inv_nb);
        note_launch();
        PC_TRY(exec_fft(plan, dtype, W, CUFFT_INVERSE, s));
        if (d_part)
            { fourier_unpack_dot<double2><<<dim3(unpack_ctas(vs), nsys), 256, 0, s>>>(
                (const double2*)W, (double2*)z, (const double2*)r, P->twa, P->twb, P->twk, g->X, g->Y, g->Z, vs,
                d_skip, d_part, unpack_ctas(vs)); note_launch(); }
        else
            { fourier_unpack<double2><<<dim3(nblocks_for(vs), nsys), 256, 0, s>>>((const double2*)W, (double2*)z,
                                                                               P->twa, P->twb, P->twk, g->X, g->Y,
                                                                               g->Z, vs, vs, 1.0, 1); note_launch(); }
    }
    if (npart_out) *npart_out = unpack_ctas(vs);
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

// Block Fourier transform of one vector (forward: what = T^H w; inverse: w = T what).
int block_fourier(pc_grid* g, int block, int dtype, int inverse, const void* in, void* out, cudaStream_t s,
                  int kslot) {
    if (!g->pre || !g->k.set) return fail(PC_ESTATE, "pc_block_fourier: pc_set_k first");
    if (kslot < 0 || kslot >= g->nk) return fail(PC_EINVAL, "block transform: Bloch slot out of range");
    Precond* P = g->pre;
    void* W;
    PC_TRY(precond_workspace(g, dtype, 1, &W));
    const double sc = 1.0 / std::sqrt((double)g->nb);
    if (P->own_dft)
        return own_block_fourier(g->X, dtype, inverse, in, out, W, P, P->d_blockids + block, kslot, sc, s);
    if (kslot != 0) return fail(PC_EINVAL, "block transform: Bloch slots other than 0 need the own DFT");
    cufftHandle plan;
    PC_TRY(get_plan(P, g, dtype, 1, &plan));
    const int64_t vs = 3 * g->nb;
    const int p12 = block >> 1, p13 = block & 1;
    const int gb = nblocks_for(vs);
    if (dtype == PC_C64) {
        if (!inverse) {
            fourier_pack<float2><<<gb, 256, 0, s>>>((const float2*)in, (float2*)W, P->twa32, P->twb32, P->twk32, g->X,
                                                     g->Y, g->Z, 1, vs, vs, 1.0, 0);
            note_launch();
            PC_TRY(exec_fft(plan, dtype, W, CUFFT_FORWARD, s));
            fourier_butterfly<float2><<<gb, 256, 0, s>>>((const float2*)W, (float2*)out, P->ea32, P->eb32, P->egh32,
                                                          g->X, g->Y, g->Z, p12, p13, sc, 0);
            note_launch();
        } else {
            fourier_butterfly<float2><<<gb, 256, 0, s>>>((const float2*)in, (float2*)W, P->ea32, P->eb32, P->egh32,
                                                          g->X, g->Y, g->Z, p12, p13, 1.0, 1);
            note_launch();
            PC_TRY(exec_fft(plan, dtype, W, CUFFT_INVERSE, s));
            fourier_unpack<float2><<<dim3(gb, 1), 256, 0, s>>>((const float2*)W, (float2*)out, P->twa32, P->twb32,
                                                                P->twk32, g->X, g->Y, g->Z, vs, vs, sc, 1);
            note_launch();
        }
    } else {
        if (!inverse) {
            fourier_pack<double2><<<gb, 256, 0, s>>>((const double2*)in, (double2*)W, P->twa, P->twb, P->twk,
                                                      g->X, g->Y, g->Z, 1, vs, vs, 1.0, 0);
            note_launch();
            PC_TRY(exec_fft(plan, dtype, W, CUFFT_FORWARD, s));
            fourier_butterfly<double2><<<gb, 256, 0, s>>>((const double2*)W, (double2*)out, P->ea, P->eb, P->egh,
                                                           g->X, g->Y, g->Z, p12, p13, sc, 0);
            note_launch();
        } else {
            fourier_butterfly<double2><<<gb, 256, 0, s>>>((const double2*)in, (double2*)W, P->ea, P->eb, P->egh,
                                                           g->X, g->Y, g->Z, p12, p13, 1.0, 1);
            note_launch();
            PC_TRY(exec_fft(plan, dtype, W, CUFFT_INVERSE, s));
            fourier_unpack<double2><<<dim3(gb, 1), 256, 0, s>>>((const double2*)W, (double2*)out, P->twa, P->twb,
                                                                 P->twk, g->X, g->Y, g->Z, vs, vs, sc, 1);
            note_launch();
        }
    }
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

}  // namespace pc
