// Direct L-point DFTs (L <= 16) with compile-time roots, the innermost step of the quarter-grid
// Bloch transform (pc_bloch_dft.cu).
//
// Forward X_k = sum_j v_j w^{jk}, w = e^{-2 pi i / L} (the inverse uses conj(w)).  The inputs pair
// up as a_j = v_j + v_{L-j}, b_j = v_j - v_{L-j} (1 <= j <= (L-1)/2), because
//     v_j w^{jk} + v_{L-j} w^{-jk} = cos(2 pi jk / L) a_j - i sin(2 pi jk / L) b_j,
// so with A_k = v_0 + sum_j cos(.) a_j (+ (-1)^k v_{L/2} for even L) and B_k = sum_j sin(.) b_j the
// two outputs k and L - k are A_k -+ i B_k (forward) and A_k +- i B_k (inverse): each pair costs
// 4 (L-1)/2 real FMAs and no root loads.  The cosines and sines are constant expressions (series
// below), and products with exact 0 or +-1 are not emitted.
#pragma once

#include "pc_complex.cuh"

namespace pc {
namespace sdft {

constexpr double kPi = 3.14159265358979323846;

// Maclaurin series of sin and cos, for |x| <= pi / 4 (terms through x^29: below 1e-35).
constexpr double series_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 15; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double series_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 15; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// cos(2 pi m / L) (s = false) or sin(2 pi m / L) (s = true): the turn fraction m / L is split into a
// quadrant q and a remainder angle alpha = (pi / 2) rem / L in [0, pi / 2); alpha above pi / 4 is
// taken as the complement, so quarter-turn multiples come out exactly 0 or +-1.
constexpr double root(int m, int L, bool s) {
    int M = m % L;
    if (M < 0) M += L;
    const int q = (4 * M) / L, rem = 4 * M - q * L;
    double ca = 0.0, sa = 0.0;
    if (2 * rem <= L) {
        const double a = 0.5 * kPi * rem / L;
        ca = series_cos(a);
        sa = series_sin(a);
    } else {
        const double b = 0.5 * kPi * (L - rem) / L;
        ca = series_sin(b);
        sa = series_cos(b);
    }
    double c = ca, sn = sa;  // rotate (cos alpha, sin alpha) by q quarter turns
    if (q == 1) {
        c = -sa;
        sn = ca;
    } else if (q == 2) {
        c = -ca;
        sn = -sa;
    } else if (q == 3) {
        c = sa;
        sn = -ca;
    }
    return s ? sn : c;
}

// A += cos(2 pi JK / L) a_J and B += sin(2 pi JK / L) b_J for J = J0 .. (L - 1) / 2.
template <int L, int K, int J, typename C, typename R>
PC_HD void pair_terms(const C (&a)[8], const C (&b)[8], R& ax, R& ay, R& bx, R& by) {
    if constexpr (J <= (L - 1) / 2) {
        constexpr double c = root(J * K, L, false), s = root(J * K, L, true);
        if constexpr (c == 1.0) {
            ax += a[J].x;
            ay += a[J].y;
        } else if constexpr (c == -1.0) {
            ax -= a[J].x;
            ay -= a[J].y;
        } else if constexpr (c != 0.0) {
            ax += (R)c * a[J].x;
            ay += (R)c * a[J].y;
        }
        if constexpr (s == 1.0) {
            bx += b[J].x;
            by += b[J].y;
        } else if constexpr (s == -1.0) {
            bx -= b[J].x;
            by -= b[J].y;
        } else if constexpr (s != 0.0) {
            bx += (R)s * b[J].x;
            by += (R)s * b[J].y;
        }
        pair_terms<L, K, J + 1>(a, b, ax, ay, bx, by);
    }
}

// Outputs K and L - K for K = K0 .. L / 2.
template <int L, bool INV, int K, typename C>
PC_HD void outputs(const C* v, const C (&a)[8], const C (&b)[8], C* out) {
    if constexpr (K <= L / 2) {
        using R = decltype(v[0].x);
        R ax = v[0].x, ay = v[0].y, bx = 0, by = 0;
        if constexpr (L % 2 == 0) {  // the unpaired middle input, weight (-1)^K
            if constexpr (K % 2 == 0) {
                ax += v[L / 2].x;
                ay += v[L / 2].y;
            } else {
                ax -= v[L / 2].x;
                ay -= v[L / 2].y;
            }
        }
        pair_terms<L, K, 1>(a, b, ax, ay, bx, by);
        // forward: X_K = A - i B, X_{L-K} = A + i B; inverse: the signs of B swap
        const R sg = INV ? (R)-1 : (R)1;
        out[K].x = ax + sg * by;
        out[K].y = ay - sg * bx;
        if constexpr (K != 0 && 2 * K != L) {
            out[L - K].x = ax - sg * by;
            out[L - K].y = ay + sg * bx;
        }
        outputs<L, INV, K + 1>(v, a, b, out);
    }
}

}  // namespace sdft

// In-place L-point DFT of v[0 .. L) (forward, or inverse without the 1 / L factor).
template <int L, bool INV, typename C>
PC_HD void small_dft_ct(C* v) {
    if constexpr (L == 1) {
        return;
    } else if constexpr (L == 2) {
        const C s = cadd(v[0], v[1]), d = csub(v[0], v[1]);
        v[0] = s;
        v[1] = d;
    } else {
        C a[8], b[8];
#pragma unroll
        for (int j = 1; j <= (L - 1) / 2; ++j) {
            a[j] = cadd(v[j], v[L - j]);
            b[j] = csub(v[j], v[L - j]);
        }
        C out[16];
        sdft::outputs<L, INV, 0>(v, a, b, out);
#pragma unroll
        for (int k = 0; k < L; ++k) v[k] = out[k];
    }
}

}  // namespace pc
