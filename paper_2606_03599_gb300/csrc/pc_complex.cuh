// Device complex arithmetic for the two storage types.
//
// complex64 values are float2 (re, im) and use the packed FP32x2 instructions of
// sm_100-class GPUs (one instruction updates the real and imaginary parts), so a
// complex add or a real-times-complex FMA costs one issue slot.  complex128
// values are double2 with plain FP64 arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pc {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

// Every helper is __host__ __device__ so that the stencil tile logic can also be
// executed by the host-side emulator; the packed FP32x2 instructions are used on
// the device, ordinary FP32 operations with the same rounding per component on the host.
#define PC_HD __host__ __device__ __forceinline__

PC_HD float2 cmk(float a, float b) { return make_float2(a, b); }
PC_HD double2 cmk(double a, double b) { return make_double2(a, b); }

// a + b
PC_HD float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
PC_HD double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
// a - b  (fma with -1 is exact)
PC_HD float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
PC_HD double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// r * a  (real scalar)
PC_HD float2 cscale(float r, float2 a) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    return __fmul2_rn(make_float2(r, r), a);
#else
    return make_float2(r * a.x, r * a.y);
#endif
}
PC_HD double2 cscale(double r, double2 a) { return make_double2(r * a.x, r * a.y); }
// acc + r * a
PC_HD float2 cfma(float r, float2 a, float2 acc) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    return __ffma2_rn(make_float2(r, r), a, acc);
#else
    return make_float2(fmaf(r, a.x, acc.x), fmaf(r, a.y, acc.y));
#endif
}
PC_HD double2 cfma(double r, double2 a, double2 acc) {
    return make_double2(fma(r, a.x, acc.x), fma(r, a.y, acc.y));
}
// complex product a * b
PC_HD float2 cmul(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
    float2 t = __fmul2_rn(make_float2(a.x, a.x), b);                      // (ar br, ar bi)
    return __ffma2_rn(make_float2(-a.y, a.y), make_float2(b.y, b.x), t);  // + (-ai bi, ai br)
#else
    return make_float2(fmaf(-a.y, b.y, a.x * b.x), fmaf(a.y, b.x, a.x * b.y));
#endif
}
PC_HD double2 cmul(double2 a, double2 b) {
    return make_double2(fma(-a.y, b.y, a.x * b.x), fma(a.y, b.x, a.x * b.y));
}
template <typename C> PC_HD C make_c(double re, double im);
template <> PC_HD float2 make_c<float2>(double re, double im) { return make_float2((float)re, (float)im); }
template <> PC_HD double2 make_c<double2>(double re, double im) { return make_double2(re, im); }

PC_HD float2 czero(float) { return make_float2(0.f, 0.f); }
PC_HD double2 czero(double) { return make_double2(0.0, 0.0); }

// True on every active lane of the warp when v holds on all of them (a warp-uniform branch
// condition: both sides of a per-thread branch would otherwise be issued for the whole warp).
PC_HD bool warp_all(bool v) {
#if defined(__CUDA_ARCH__)
    return __all_sync(__activemask(), v);
#else
    return v;
#endif
}

// (a, b, k) of the linear index t = a + X (b + Y k) in 32-bit unsigned arithmetic (every
// per-vector index of the library is below 2^32; 64-bit division is a long software sequence).
PC_HD void split3(int64_t t, int X, int Y, int& a, int& b, int& k) {
    const uint32_t u = (uint32_t)t, q = u / (uint32_t)X;
    a = (int)(u - q * (uint32_t)X);
    k = (int)(q / (uint32_t)Y);
    b = (int)(q - (uint32_t)k * (uint32_t)Y);
}

// True on every active lane when v holds on at least one of them.
PC_HD bool warp_any(bool v) {
#if defined(__CUDA_ARCH__)
    return __any_sync(__activemask(), v);
#else
    return v;
#endif
}

// acc + Re(conj(a) * b)
PC_HD float cdotre(float2 a, float2 b, float acc) { return fmaf(a.x, b.x, fmaf(a.y, b.y, acc)); }
PC_HD double cdotre(double2 a, double2 b, double acc) { return fma(a.x, b.x, fma(a.y, b.y, acc)); }

}  // namespace pc
