// Quarter-grid Bloch transform of the parity blocks (Sec. 5.2, Eqs. psi_pqr_unified,
// f_sigma_unified, Tsigma_unified) and the reference-medium preconditioner built on it (Sec. 5.4),
// as three own kernels per application instead of library FFTs.
//
// A block vector lives on the quarter grid (a, b, k), a, b < n = N/2, k < N.  Splitting k = 2k' +
// par, the block transform is, per component and parity, the plain 3D DFT of size n x n x n of the
// pre-twiddled parity planes, followed by the parity butterfly with T_par (see pc_fourier.cu).  All
// three axes have the same length n, so one factorisation n = n1 n2 serves every axis:
//
//   X[k1 + n1 k2] = sum_{i2 < n2} w_n^{i2 k1} [sum_{i1 < n1} x[i1 n2 + i2] w_n1^{i1 k1}] w_n2^{i2 k2}
//
// (Cooley-Tukey with two direct DFTs of lengths n1, n2 <= 16, w_m = e^{-2 pi i / m}; the direct DFTs
// pair their inputs and take their roots as compile-time constants, pc_small_dft.cuh).  Both stages
// work in place in shared memory on groups of n1 (stage A) or n2 (stage B) values that no other
// thread touches, so a stage needs no barrier inside; the spectrum comes out digit-permuted
// (mode k1 + n1 k2 at position k1 n2 + k2) and the inverse stages take that order back to the natural
// one.  Global reads and writes stay in natural order (the permutation is applied on the shared-
// memory side).
//
//   K1 plane_fwd  : per (system, component, parity, k') plane: pre-twiddle, 2D DFT over (a, b);
//   K2 pencil     : per (system, q, tile of p): DFT over k' of the six (component, parity) pencils,
//                   then either the parity butterfly, the per-mode 3x3 reference-symbol solve and the
//                   inverse butterfly (preconditioner), or only the butterfly (forward transform) or
//                   only its inverse (inverse transform); then the inverse DFT over k' where needed;
//   K3 plane_inv  : per plane: inverse 2D DFT, post-twiddle, optional scale, with the inner product
//                   Re <r, z> of the preconditioner fused (one partial per plane).
// The transforms are unnormalised (the preconditioner's symbol solve carries 1 / n_b, the block
// transform its 1 / sqrt(n_b)), as the factors of Eq. Tsigma_unified require.
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "pc_complex.cuh"
#include "pc_fourier.h"
#include "pc_internal.h"
#include "pc_small_dft.cuh"

namespace pc {

namespace {

constexpr int kDftMaxFactor = 16;
constexpr int kDftMaxN = 96;
constexpr int kPlaneThreads = 128;   // one plane per CTA of the plane kernels
constexpr int kPencilThreads = 256;
// Threads per CTA for compile-time factors: the large planes and pencils (n >= 40) hold 25-60 KB of
// shared memory per CTA, so few CTAs fit on an SM; more threads per CTA keep the SM's warps up.
template <int N1, int N2>
constexpr int plane_nt() { return N1 > 0 && N1 * N2 >= 40 ? 512 : kPlaneThreads; }
template <int N1, int N2>
constexpr int pencil_nt() { return N1 > 0 && N1 * N2 >= 40 ? 512 : kPencilThreads; }
constexpr int kPencilTileMax = 16;  // p positions per pencil CTA: the largest divisor of n up to this

template <typename C> struct RTy;
template <> struct RTy<float2> { using R = float; };
template <> struct RTy<double2> { using R = double; };

template <typename C> __device__ __forceinline__ C conj_c(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __device__ __forceinline__ C scale_c(R r, C a) { a.x *= r; a.y *= r; return a; }
template <typename Co, typename Ci> __device__ __forceinline__ Co conv_c(Ci v) {
    Co o;
    o.x = (decltype(o.x))v.x;
    o.y = (decltype(o.y))v.y;
    return o;
}

// Geometry of one batch of lines along an axis of a shared-memory array: element e of line l sits at
// base(l) + e * es with base(l) = (l % lo) * ls_lo + (l / lo) * ls_hi.
struct Lines {
    int count, lo, ls_lo, ls_hi, es;
    bool line_fast;  // consecutive threads take consecutive lines (else consecutive inner indices)
    __device__ __forceinline__ int base(int l) const { return (l % lo) * ls_lo + (l / lo) * ls_hi; }
};

// Stage A (forward): for every line and i2 < n2, the n1 values at i1 n2 + i2 -> their n1-point DFT
// times w_n^{i2 k1}, in place.  Inverse (A^-1, the last inverse stage): conjugate twiddle first, then
// the conjugate n1-point DFT.
template <int L1, bool INV, typename C>
__device__ __forceinline__ void stage_a(C* buf, const Lines ln, int n1, int n2, const C* wn, int n) {
    const int groups = ln.count * n2;
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int l = ln.line_fast ? g % ln.count : g / n2;
        const int i2 = ln.line_fast ? g / ln.count : g % n2;
        const int b0 = ln.base(l) + i2 * ln.es;
        C v[kDftMaxFactor];
#pragma unroll
        for (int i = 0; i < L1; ++i) v[i] = buf[b0 + i * n2 * ln.es];
        if (INV) {
#pragma unroll
            for (int k = 1; k < L1; ++k) v[k] = cmul(v[k], conj_c(wn[(i2 * k) % n]));
        }
        small_dft_ct<L1, INV>(v);
        if (!INV) {
#pragma unroll
            for (int k = 1; k < L1; ++k) v[k] = cmul(v[k], wn[(i2 * k) % n]);
        }
#pragma unroll
        for (int i = 0; i < L1; ++i) buf[b0 + i * n2 * ln.es] = v[i];
    }
}

// Stage B: for every line and k1 < n1, the n2 contiguous values at k1 n2 + i2 -> their n2-point DFT
// (conjugate when INV), in place.
template <int L2, bool INV, typename C>
__device__ __forceinline__ void stage_b(C* buf, const Lines ln, int n1, int n2, const C* wn) {
    const int groups = ln.count * n1;
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        const int l = ln.line_fast ? g % ln.count : g / n1;
        const int k1 = ln.line_fast ? g / ln.count : g % n1;
        const int b0 = ln.base(l) + k1 * n2 * ln.es;
        C v[kDftMaxFactor];
#pragma unroll
        for (int i = 0; i < L2; ++i) v[i] = buf[b0 + i * ln.es];
        small_dft_ct<L2, INV>(v);
#pragma unroll
        for (int i = 0; i < L2; ++i) buf[b0 + i * ln.es] = v[i];
    }
}

template <bool INV, typename C>
__device__ void dispatch_a(C* buf, const Lines ln, int n1, int n2, const C* wn, int n) {
    switch (n1) {
#define PC_CASE(L) case L: stage_a<L, INV>(buf, ln, n1, n2, wn, n); break;
        PC_CASE(1) PC_CASE(2) PC_CASE(3) PC_CASE(4) PC_CASE(5) PC_CASE(6) PC_CASE(7) PC_CASE(8)
        PC_CASE(9) PC_CASE(10) PC_CASE(11) PC_CASE(12) PC_CASE(13) PC_CASE(14) PC_CASE(15) PC_CASE(16)
#undef PC_CASE
        default: break;
    }
}
template <bool INV, typename C>
__device__ void dispatch_b(C* buf, const Lines ln, int n1, int n2, const C* wn) {
    switch (n2) {
#define PC_CASE(L) case L: stage_b<L, INV>(buf, ln, n1, n2, wn); break;
        PC_CASE(1) PC_CASE(2) PC_CASE(3) PC_CASE(4) PC_CASE(5) PC_CASE(6) PC_CASE(7) PC_CASE(8)
        PC_CASE(9) PC_CASE(10) PC_CASE(11) PC_CASE(12) PC_CASE(13) PC_CASE(14) PC_CASE(15) PC_CASE(16)
#undef PC_CASE
        default: break;
    }
}

// Forward transform of the lines (natural order in, digit-permuted out) and its inverse.  N1 > 0:
// the factors are compile-time constants (N1, N2) (only the stages of that size are compiled into
// the kernel); N1 = 0: runtime factors.
template <int N1, int N2, typename C>
__device__ __forceinline__ void dft_fwd(C* buf, const Lines ln, int n1, int n2, const C* wn, int n) {
    if constexpr (N1 > 0) stage_a<N1, false>(buf, ln, N1, N2, wn, N1 * N2);
    else dispatch_a<false>(buf, ln, n1, n2, wn, n);
    __syncthreads();
    if constexpr (N1 > 0) stage_b<N2, false>(buf, ln, N1, N2, wn);
    else dispatch_b<false>(buf, ln, n1, n2, wn);
    __syncthreads();
}
template <int N1, int N2, typename C>
__device__ __forceinline__ void dft_inv(C* buf, const Lines ln, int n1, int n2, const C* wn, int n) {
    if constexpr (N1 > 0) stage_b<N2, true>(buf, ln, N1, N2, wn);
    else dispatch_b<true>(buf, ln, n1, n2, wn);
    __syncthreads();
    if constexpr (N1 > 0) stage_a<N1, true>(buf, ln, N1, N2, wn, N1 * N2);
    else dispatch_a<true>(buf, ln, n1, n2, wn, n);
    __syncthreads();
}

// Planes per CTA of the plane kernels (one: many small CTAs keep every SM busy at the solver's sizes).
__host__ __device__ __forceinline__ int planes_per_cta(int) { return 1; }

// p positions per pencil CTA: the largest divisor of n that is at most kPencilTileMax (no ragged tile).
__host__ __device__ constexpr int pencil_tile(int n) {
    int t = 1;
    for (int d = 1; d <= kPencilTileMax && d <= n; ++d)
        if (n % d == 0) t = d;
    return t;
}

// position of mode m = k1 + n1 k2 in the digit-permuted order
__device__ __forceinline__ int perm_pos(int m, int n1, int n2) { return (m % n1) * n2 + m / n1; }

// Twiddle T_par(p, q, r) of the parity butterfly (as in pc_fourier.cu), r < n.
template <typename C, typename TT>
__device__ __forceinline__ C t_par2(const TT* ea, const TT* eb, const TT* eg, int p, int q, int r, int par, int p12,
                                    int p13) {
    const int i0 = (par + p13) & 1, j0 = (par + p12 + p13) & 1;
    C t;
    t.x = 1;
    t.y = 0;
    if (par) t = conv_c<C>(eg[r]);
    if (i0) t = cmul(t, conv_c<C>(ea[p]));
    if (j0) t = cmul(t, conv_c<C>(eb[q]));
    return t;
}

// K1: one plane per CTA (plane id = ((sys * 3 + comp) * 2 + par) * n + k' = blockIdx.x): w (type Ci)
// pre-twiddled into the work buffer W (type C), 2D DFT over (a, b).  W layout [sys][comp][par][k'][q][p].
// The loads run four per thread before their shared-memory stores, so several are in flight.
template <int N1, int N2, typename C, typename Ci>
__global__ void __launch_bounds__(plane_nt<N1, N2>())
    bdft_plane_fwd(const Ci* __restrict__ w, C* __restrict__ W, const C* __restrict__ wn_g, const C* __restrict__ twa,
                   const C* __restrict__ twb, const C* __restrict__ twk, int n_rt, int n1, int n2, int nplanes,
                   int64_t sys_stride_in, int64_t sys_stride_out, const int* __restrict__ skip, int conj_tw,
                   const int* __restrict__ sys_k, int64_t tab_stride) {
    extern __shared__ __align__(16) unsigned char smem_bdft[];
    const int n = N1 > 0 ? N1 * N2 : n_rt;
    if (N1 > 0) {  // compile-time factors: every index division below is by a constant
        n1 = N1;
        n2 = N2;
    }
    const int nn = n * n;
    const int pl = blockIdx.x;
    if (pl >= nplanes) return;
    const int kp = pl % n, rest = pl / n;
    const int par = rest & 1, comp = (rest >> 1) % 3, sys = rest / 6;
    if (skip && skip[sys]) return;  // the whole CTA: nothing of this system is written
    C* buf = reinterpret_cast<C*>(smem_bdft);
    C* wn = buf + nn;
    const int64_t nb = (int64_t)2 * n * nn, plane = nn;
    for (int j = threadIdx.x; j < n; j += blockDim.x) wn[j] = wn_g[j];
    const int64_t to = sys_k ? (int64_t)sys_k[sys] * tab_stride : 0;
    const C* ta = twa + to;
    const C* tb = twb + to;
    const C tk = twk[to + kp];
    const Ci* src = w + sys * sys_stride_in + comp * nb + (int64_t)(2 * kp + par) * plane;
#pragma unroll 4
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int b = t / n, a = t - b * n;
        C tw = cmul(cmul(ta[a], tb[b]), tk);
        if (conj_tw) tw = conj_c(tw);
        buf[t] = cmul(conv_c<C>(src[t]), tw);
    }
    __syncthreads();
    const Lines rows{n, n, n, nn, 1, false};
    dft_fwd<N1, N2>(buf, rows, n1, n2, wn, n);
    const Lines cols{n, n, 1, nn, n, true};
    dft_fwd<N1, N2>(buf, cols, n1, n2, wn, n);
    C* dst = W + sys * sys_stride_out + comp * nb + par * (nb / 2) + (int64_t)kp * plane;
#pragma unroll 4
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int q = t / n, p = t - q * n;
        dst[t] = buf[perm_pos(q, n1, n2) * n + perm_pos(p, n1, n2)];
    }
}

// K3: one plane per CTA: inverse 2D DFT of W's plane, post-twiddle (conjugate of the pre-twiddle),
// scale, into z (type Co); with part non-null also the partial Re <r, z> of the plane (partial index
// = plane id within its system, 6 n per system).
template <int N1, int N2, typename C, typename Co>
__global__ void __launch_bounds__(plane_nt<N1, N2>())
    bdft_plane_inv(const C* __restrict__ W, Co* __restrict__ z, const Co* __restrict__ r, const C* __restrict__ wn_g,
                   const C* __restrict__ twa, const C* __restrict__ twb, const C* __restrict__ twk, int n_rt, int n1,
                   int n2, int nplanes, int64_t sys_stride_in, int64_t sys_stride_out, double scale,
                   const int* __restrict__ skip, double* __restrict__ part, int npart, const int* __restrict__ sys_k,
                   int64_t tab_stride) {
    extern __shared__ __align__(16) unsigned char smem_bdft[];
    using R = typename RTy<C>::R;
    const int n = N1 > 0 ? N1 * N2 : n_rt;
    if (N1 > 0) {
        n1 = N1;
        n2 = N2;
    }
    const int nn = n * n;
    const int pl = blockIdx.x;
    if (pl >= nplanes) return;
    const int kp = pl % n, rest = pl / n;
    const int par = rest & 1, comp = (rest >> 1) % 3, sys = rest / 6;
    if (skip && skip[sys]) return;
    C* buf = reinterpret_cast<C*>(smem_bdft);
    C* wn = buf + nn;
    const int64_t nb = (int64_t)2 * n * nn, plane = nn;
    for (int j = threadIdx.x; j < n; j += blockDim.x) wn[j] = wn_g[j];
    const C* src = W + sys * sys_stride_in + comp * nb + par * (nb / 2) + (int64_t)kp * plane;
#pragma unroll 4
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int q = t / n, p = t - q * n;
        buf[perm_pos(q, n1, n2) * n + perm_pos(p, n1, n2)] = src[t];
    }
    __syncthreads();
    const Lines cols{n, n, 1, nn, n, true};
    dft_inv<N1, N2>(buf, cols, n1, n2, wn, n);
    const Lines rows{n, n, n, nn, 1, false};
    dft_inv<N1, N2>(buf, rows, n1, n2, wn, n);
    const R sc = (R)scale;
    using Ro = decltype(z[0].x);
    Ro acc = 0;  // per-thread sum in the output precision, FP64 across threads
    const int64_t to = sys_k ? (int64_t)sys_k[sys] * tab_stride : 0;
    const C* ta = twa + to;
    const C* tb = twb + to;
    const C tk = twk[to + kp];
    const int64_t base = sys * sys_stride_out + comp * nb + (int64_t)(2 * kp + par) * plane;
#pragma unroll 4
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        const int b = t / n, a = t - b * n;
        const C tw = conj_c(cmul(cmul(ta[a], tb[b]), tk));
        const Co v = conv_c<Co>(scale_c(sc, cmul(buf[t], tw)));
        z[base + t] = v;
        if (part) acc = cdotre(r[base + t], v, acc);
    }
    if (part) {
        __shared__ double red[plane_nt<N1, N2>() / 32];
        double v = (double)acc;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
            part[(int64_t)sys * npart + (pl - sys * 6 * n)] = t;
        }
    }
}

// K2: per (system, q, tile of pencil_tile(n) p positions): DFT over k' of the six (component, parity)
// pencils, then by `mode`: 0 = preconditioner (butterfly, (A_ref - sigma rho_ref)^-1 scaled, inverse
// butterfly, inverse DFT over k'); 1 = forward block transform (butterfly, scaled, written to `out` in
// mode order [comp][r < 2n][q][p]); 2 = inverse block transform (reads `out`'s layout from W, inverse
// butterfly, inverse DFT over k', written to W).
template <int N1, int N2, typename C, typename R, typename TT>
__global__ void __launch_bounds__(pencil_nt<N1, N2>())
    bdft_pencil(C* __restrict__ W, C* __restrict__ out, const C* __restrict__ wn_g, const R* __restrict__ Aref,
                const TT* __restrict__ ea, const TT* __restrict__ eb, const TT* __restrict__ eg,
                const int* __restrict__ sys_block, const int* __restrict__ skip, int n_rt, int n1, int n2,
                int64_t sys_stride, double shift_rho_d, double scale_d, int mode, const int* __restrict__ sys_k,
                int64_t tab_stride, int64_t aref_stride) {
    const int n = N1 > 0 ? N1 * N2 : n_rt;
    if (N1 > 0) {
        n1 = N1;
        n2 = N2;
    }
    extern __shared__ __align__(16) unsigned char smem_bdft[];
    constexpr int PTc = N1 > 0 ? pencil_tile(N1 * N2) : 1;
    const int PT = N1 > 0 ? PTc : pencil_tile(n);
    C* buf = reinterpret_cast<C*>(smem_bdft);  // [pencil = comp * 2 + par][k'][pl]
    C* wn = buf + 6 * n * PT;
    const int tiles = n / PT;
    int id = blockIdx.x;
    const int tile = id % tiles;
    id /= tiles;
    const int q = id % n;
    const int sys = id / n;
    if (skip && skip[sys]) return;
    const int b = sys_block[sys];
    const int p12 = b >> 1, p13 = b & 1;
    if (sys_k) {  // this system's Bloch slot
        const int ks = sys_k[sys];
        ea += ks * tab_stride;
        eb += ks * tab_stride;
        eg += ks * tab_stride;
        if (Aref) Aref += ks * aref_stride;
    }
    const int p0 = tile * PT, pw = min(PT, n - p0);
    const int64_t nb = (int64_t)2 * n * n * n, plane = (int64_t)n * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) wn[j] = wn_g[j];
    C* Ws = W + sys * sys_stride;
    const Lines pencils{6 * PT, PT, 1, n * PT, PT, true};
    const R shift_rho = (R)shift_rho_d, scale = (R)scale_d;
    if (mode != 2) {
#pragma unroll 4
        for (int e = threadIdx.x; e < 6 * n * PT; e += blockDim.x) {
            const int pl = e % PT, kp = (e / PT) % n, pen = e / (PT * n);
            C v;
            v.x = 0;
            v.y = 0;
            if (pl < pw) v = Ws[(pen >> 1) * nb + (pen & 1) * (nb / 2) + (int64_t)kp * plane + (int64_t)q * n + p0 + pl];
            buf[e] = v;
        }
        __syncthreads();
        dft_fwd<N1, N2>(buf, pencils, n1, n2, wn, n);
    } else {
        // modes r < 2n of `out`'s layout: mode r and r + n of the same (p, q) pair up in the butterfly
        C* Os = out + sys * sys_stride;
        for (int e = threadIdx.x; e < 3 * n * PT; e += blockDim.x) {
            const int pl = e % PT, r = (e / PT) % n, comp = e / (PT * n);
            C lo, hi;
            lo.x = lo.y = hi.x = hi.y = 0;
            if (pl < pw) {
                lo = Os[comp * nb + (int64_t)r * plane + (int64_t)q * n + p0 + pl];
                hi = Os[comp * nb + (int64_t)(r + n) * plane + (int64_t)q * n + p0 + pl];
            }
            const int p = p0 + (pl < pw ? pl : 0);
            const C T0 = t_par2<C>(ea, eb, eg, p, q, r, 0, p12, p13);
            const C T1 = t_par2<C>(ea, eb, eg, p, q, r, 1, p12, p13);
            const int pos = perm_pos(r, n1, n2);
            buf[((comp * 2 + 0) * n + pos) * PT + pl] = scale_c(scale, cmul(conj_c(T0), cadd(lo, hi)));
            buf[((comp * 2 + 1) * n + pos) * PT + pl] = scale_c(scale, cmul(conj_c(T1), csub(lo, hi)));
        }
        __syncthreads();
    }
    if (mode == 0 || mode == 1) {
        for (int u = threadIdx.x; u < n * PT; u += blockDim.x) {
            const int pl = u % PT, r = u / PT;
            if (pl >= pw) continue;
            const int p = p0 + pl;
            const int pos = perm_pos(r, n1, n2);
            const C T0 = t_par2<C>(ea, eb, eg, p, q, r, 0, p12, p13);
            const C T1 = t_par2<C>(ea, eb, eg, p, q, r, 1, p12, p13);
            C lo[3], hi[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const C w0 = cmul(T0, buf[((c * 2 + 0) * n + pos) * PT + pl]);
                const C w1 = cmul(T1, buf[((c * 2 + 1) * n + pos) * PT + pl]);
                lo[c] = cadd(w0, w1);
                hi[c] = csub(w0, w1);
            }
            if (mode == 1) {
                C* Os = out + sys * sys_stride;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Os[c * nb + (int64_t)r * plane + (int64_t)q * n + p] = scale_c(scale, lo[c]);
                    Os[c * nb + (int64_t)(r + n) * plane + (int64_t)q * n + p] = scale_c(scale, hi[c]);
                }
                continue;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t mode_i = (int64_t)(r + h * n) * plane + (int64_t)q * n + p;  // [r][q][p], r < 2n
                const R* A = Aref + 9 * mode_i;
                const R d0 = A[0] + shift_rho, d1 = A[1] + shift_rho, d2 = A[2] + shift_rho;
                C a01, a02, a12;
                a01.x = A[3]; a01.y = A[4];
                a02.x = A[5]; a02.y = A[6];
                a12.x = A[7]; a12.y = A[8];
                const R c00 = d1 * d2 - (a12.x * a12.x + a12.y * a12.y);
                const R c11 = d0 * d2 - (a02.x * a02.x + a02.y * a02.y);
                const R c22 = d0 * d1 - (a01.x * a01.x + a01.y * a01.y);
                const C c01 = csub(cmul(a02, conj_c(a12)), cscale(d2, a01));
                const C c02 = csub(cmul(a01, a12), cscale(d1, a02));
                const C c12 = csub(cmul(conj_c(a01), a02), cscale(d0, a12));
                const R det = d0 * c00 + (a01.x * c01.x + a01.y * c01.y) + (a02.x * c02.x + a02.y * c02.y);
                const R inv = scale / det;
                C* v = h ? hi : lo;
                const C v0 = v[0], v1 = v[1], v2 = v[2];
                const C z0 = cadd(cadd(cscale(c00, v0), cmul(c01, v1)), cmul(c02, v2));
                const C z1 = cadd(cadd(cmul(conj_c(c01), v0), cscale(c11, v1)), cmul(c12, v2));
                const C z2 = cadd(cadd(cmul(conj_c(c02), v0), cmul(conj_c(c12), v1)), cscale(c22, v2));
                v[0] = cscale(inv, z0);
                v[1] = cscale(inv, z1);
                v[2] = cscale(inv, z2);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                buf[((c * 2 + 0) * n + pos) * PT + pl] = cmul(conj_c(T0), cadd(lo[c], hi[c]));
                buf[((c * 2 + 1) * n + pos) * PT + pl] = cmul(conj_c(T1), csub(lo[c], hi[c]));
            }
        }
        if (mode == 1) return;
        __syncthreads();
    }
    dft_inv<N1, N2>(buf, pencils, n1, n2, wn, n);
    for (int e = threadIdx.x; e < 6 * n * PT; e += blockDim.x) {
        const int pl = e % PT, kp = (e / PT) % n, pen = e / (PT * n);
        if (pl < pw) Ws[(pen >> 1) * nb + (pen & 1) * (nb / 2) + (int64_t)kp * plane + (int64_t)q * n + p0 + pl] = buf[e];
    }
}

template <typename C>
size_t plane_smem(int n) { return sizeof(C) * ((size_t)planes_per_cta(n) * n * n + n); }
template <typename C>
size_t pencil_smem(int n) { return sizeof(C) * ((size_t)6 * n * pencil_tile(n) + n); }

// Dynamic shared memory beyond 48 KB is granted once per kernel (the largest size asked so far).
template <typename K>
int allow_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return PC_OK;
    static std::mutex mu;
    static std::map<const void*, size_t> granted;
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = granted[reinterpret_cast<const void*>(kern)];
    if (bytes > have) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(block DFT)");
        have = bytes;
    }
    return PC_OK;
}


// Launch of the three kernels for compile-time factors (N1, N2) (N1 = 0: runtime factors).
template <int N1, int N2, typename C, typename V, typename TT>
static int precond_launch(int n, int n1, int n2, int nsys, const V* r, V* z, C* W, const C* wn, const C* twa,
                          const C* twb, const C* twk, const TT* ea, const TT* eb, const TT* eg,
                          const typename RTy<C>::R* Aref, const int* sys_block, const int* sys_k, int64_t tab_stride,
                          const int* skip, double shift_rho, double scale, double* part, cudaStream_t s) {
    using R = typename RTy<C>::R;
    const int64_t vs = (int64_t)6 * n * n * n;
    const int64_t aref_stride = (int64_t)9 * 2 * n * n * n;
    const size_t sp = plane_smem<C>(n), sq = pencil_smem<C>(n);
    PC_TRY(allow_smem(bdft_plane_fwd<N1, N2, C, V>, sp));
    PC_TRY(allow_smem(bdft_pencil<N1, N2, C, R, TT>, sq));
    PC_TRY(allow_smem(bdft_plane_inv<N1, N2, C, V>, sp));
    const int planes = nsys * 6 * n, pctas = (planes + planes_per_cta(n) - 1) / planes_per_cta(n);
    bdft_plane_fwd<N1, N2, C, V><<<pctas, (plane_nt<N1, N2>()), sp, s>>>(r, W, wn, twa, twb, twk, n, n1, n2, planes, vs, vs,
                                                               skip, 0, sys_k, tab_stride);
    note_launch();
    const int tiles = n / pencil_tile(n);
    bdft_pencil<N1, N2, C, R, TT><<<nsys * n * tiles, (pencil_nt<N1, N2>()), sq, s>>>(
        W, nullptr, wn, Aref, ea, eb, eg, sys_block, skip, n, n1, n2, vs, shift_rho, scale, 0, sys_k, tab_stride,
        aref_stride);
    note_launch();
    bdft_plane_inv<N1, N2, C, V><<<pctas, (plane_nt<N1, N2>()), sp, s>>>(W, z, r, wn, twa, twb, twk, n, n1, n2, planes, vs,
                                                               vs, 1.0, skip, part, bloch_dft_partials(n), sys_k,
                                                               tab_stride);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

template <int N1, int N2, typename C>
static int fourier_launch(int n, int n1, int n2, int inverse, const C* in, C* out, C* W, const C* wn, const C* twa,
                          const C* twb, const C* twk, const C* ea, const C* eb, const C* eg, const int* d_block,
                          double scale, cudaStream_t s) {
    using R = typename RTy<C>::R;
    const int64_t vs = (int64_t)6 * n * n * n;
    const size_t sp = plane_smem<C>(n), sq = pencil_smem<C>(n);
    PC_TRY(allow_smem(bdft_plane_fwd<N1, N2, C, C>, sp));
    PC_TRY(allow_smem(bdft_pencil<N1, N2, C, R, C>, sq));
    PC_TRY(allow_smem(bdft_plane_inv<N1, N2, C, C>, sp));
    const int planes = 6 * n, pctas = (planes + planes_per_cta(n) - 1) / planes_per_cta(n);
    const int tiles = n / pencil_tile(n);
    if (!inverse) {
        bdft_plane_fwd<N1, N2, C, C><<<pctas, (plane_nt<N1, N2>()), sp, s>>>(in, W, wn, twa, twb, twk, n, n1, n2, planes, vs,
                                                                   vs, nullptr, 0, nullptr, 0);
        note_launch();
        bdft_pencil<N1, N2, C, R, C><<<n * tiles, (pencil_nt<N1, N2>()), sq, s>>>(
            W, out, wn, nullptr, ea, eb, eg, d_block, nullptr, n, n1, n2, vs, 0.0, scale, 1, nullptr, 0, 0);
        note_launch();
    } else {
        bdft_pencil<N1, N2, C, R, C><<<n * tiles, (pencil_nt<N1, N2>()), sq, s>>>(
            W, const_cast<C*>(in), wn, nullptr, ea, eb, eg, d_block, nullptr, n, n1, n2, vs, 0.0, 1.0, 2, nullptr, 0, 0);
        note_launch();
        bdft_plane_inv<N1, N2, C, C><<<pctas, (plane_nt<N1, N2>()), sp, s>>>(W, out, nullptr, wn, twa, twb, twk, n, n1, n2,
                                                                   planes, vs, vs, scale, nullptr, nullptr, 0, nullptr,
                                                                   0);
        note_launch();
    }
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

// Compile-time factorisations of the block lengths n = N/2 of the solver's grids (N = 8 .. 160 and the
// paper's 60); any other supported n runs the runtime-factor kernels.
#define PC_DFT_SIZES(X) X(2, 2) X(2, 4) X(3, 4) X(4, 4) X(4, 6) X(5, 6) X(4, 8) X(6, 8) X(8, 8) X(8, 10)

}  // namespace

bool bloch_dft_supported(int n, int* n1, int* n2) {
    if (n < 1 || n > kDftMaxN) return false;
    int best = 1;
    for (int a = 1; a * a <= n; ++a)
        if (n % a == 0) best = a;
    if (n / best > kDftMaxFactor) return false;
    if (n1) *n1 = best;
    if (n2) *n2 = n / best;
    return true;
}

int bloch_dft_partials(int n) { return 6 * n; }

template <typename C, typename V, typename TT>
static int own_precond_t(int n, int nsys, const V* r, V* z, C* W, const C* wn, const C* twa, const C* twb,
                         const C* twk, const TT* ea, const TT* eb, const TT* eg, const typename RTy<C>::R* Aref,
                         const int* sys_block, const int* sys_k, int64_t tab_stride, const int* skip,
                         double shift_rho, double scale, double* part, cudaStream_t s) {
    int n1, n2;
    if (!bloch_dft_supported(n, &n1, &n2)) return fail(PC_EINVAL, "block DFT: unsupported size");
#define PC_DFT_CASE(A, B)                                                                                   \
    if (n1 == A && n2 == B)                                                                                 \
        return precond_launch<A, B>(n, n1, n2, nsys, r, z, W, wn, twa, twb, twk, ea, eb, eg, Aref, sys_block, \
                                    sys_k, tab_stride, skip, shift_rho, scale, part, s);
    PC_DFT_SIZES(PC_DFT_CASE)
#undef PC_DFT_CASE
    return precond_launch<0, 0>(n, n1, n2, nsys, r, z, W, wn, twa, twb, twk, ea, eb, eg, Aref, sys_block, sys_k,
                                tab_stride, skip, shift_rho, scale, part, s);
}

int own_precond(int n, int wdt, int vdt, int nsys, const void* r, void* z, void* W, const Precond* P,
                const int* sys_block, const int* sys_k, const int* skip, double shift_rho, double scale,
                double* part, cudaStream_t s) {
    const int64_t ts = P->tab_len;
    if (wdt == PC_C64 && vdt == PC_C64)
        return own_precond_t<float2, float2, float2>(n, nsys, (const float2*)r, (float2*)z, (float2*)W, P->wn32,
                                                     P->twa32, P->twb32, P->twk32, P->ea32, P->eb32, P->egh32,
                                                     P->d_Aref32, sys_block, sys_k, ts, skip, shift_rho, scale, part,
                                                     s);
    if (wdt == PC_C64 && vdt == PC_C128)
        return own_precond_t<float2, double2, float2>(n, nsys, (const double2*)r, (double2*)z, (float2*)W, P->wn32,
                                                      P->twa32, P->twb32, P->twk32, P->ea32, P->eb32, P->egh32,
                                                      P->d_Aref32, sys_block, sys_k, ts, skip, shift_rho, scale, part,
                                                      s);
    return own_precond_t<double2, double2, double2>(n, nsys, (const double2*)r, (double2*)z, (double2*)W, P->wn,
                                                    P->twa, P->twb, P->twk, P->ea, P->eb, P->egh, P->d_Aref,
                                                    sys_block, sys_k, ts, skip, shift_rho, scale, part, s);
}

// Block transform of one vector of block b: forward (what = T^H w, modes [comp][r < 2n][q][p]) or
// inverse (w = T what).  d_block: device int holding b.  scale: 1 / sqrt(n_b).
template <typename C>
static int own_fourier_t(int n, int inverse, const C* in, C* out, C* W, const C* wn, const C* twa, const C* twb,
                         const C* twk, const C* ea, const C* eb, const C* eg, const int* d_block, double scale,
                         cudaStream_t s) {
    int n1, n2;
    if (!bloch_dft_supported(n, &n1, &n2)) return fail(PC_EINVAL, "block DFT: unsupported size");
#define PC_DFT_CASE(A, B)                                                                                           \
    if (n1 == A && n2 == B)                                                                                         \
        return fourier_launch<A, B>(n, n1, n2, inverse, in, out, W, wn, twa, twb, twk, ea, eb, eg, d_block, scale, s);
    PC_DFT_SIZES(PC_DFT_CASE)
#undef PC_DFT_CASE
    return fourier_launch<0, 0>(n, n1, n2, inverse, in, out, W, wn, twa, twb, twk, ea, eb, eg, d_block, scale, s);
}

int own_block_fourier(int n, int dtype, int inverse, const void* in, void* out, void* W, const Precond* P,
                      const int* d_block, int kslot, double scale, cudaStream_t s) {
    const size_t o = (size_t)kslot * P->tab_len;  // the slot's tables
    if (dtype == PC_C64)
        return own_fourier_t<float2>(n, inverse, (const float2*)in, (float2*)out, (float2*)W, P->wn32, P->twa32 + o,
                                     P->twb32 + o, P->twk32 + o, P->ea32 + o, P->eb32 + o, P->egh32 + o, d_block,
                                     scale, s);
    return own_fourier_t<double2>(n, inverse, (const double2*)in, (double2*)out, (double2*)W, P->wn, P->twa + o,
                                  P->twb + o, P->twk + o, P->ea + o, P->eb + o, P->egh + o, d_block, scale, s);
}

}  // namespace pc
