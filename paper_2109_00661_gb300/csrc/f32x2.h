// Paired FP32 arithmetic and the hardware approximations shared by the FP32
// forward kernel (forward.cu) and its adjoint (adjoint.cu).
//
// Two values (two Hankel abscissae of one frequency in both kernels) travel
// in one 64-bit register pair and are advanced with the sm_100+ paired FP32
// instructions (add/sub/mul/fma .rn.f32x2): one issue slot per operation on
// both.  The special functions (sqrt, rsqrt, rcp, ex2, sin, cos) are the hardware
// approximations, one scalar instruction per value (relative error about
// 2^-22; sin and cos have an absolute error of the same size on the phases
// both kernels pass them).
#pragma once

#include <cuda_runtime.h>

namespace aem {
namespace f32x2 {

typedef unsigned long long u64;

constexpr u64 kZero2 = 0ull;                   // (0, 0)
constexpr u64 kOne2 = 0x3f8000003f800000ull;   // (1, 1)
constexpr u64 kHalf2 = 0x3f0000003f000000ull;  // (0.5, 0.5)

// Measurement builds (off by default; build.py passes them through its
// AEM_NVCC_DEFINES environment variable):
//   AEM_F32_ACCURATE_MATH=1  the round-to-nearest square root, reciprocal and
//     reciprocal square root and the library's exp2f / sincosf (full range reduction) in
//     place of the hardware approximations, to separate the approximations'
//     share of the FP32 error from the FP32 arithmetic's;
//   AEM_F32_REDUCE_PHASE=1   the Moebius step's phase reduced modulo 2 pi
//     (Cody & Waite 1980: k = round(x / 2 pi) by the 1.5 * 2^23 shifter, then
//     x - k C1 - k C2 with C1 + C2 = 2 pi, C1 the nearest float) before the
//     hardware sine and cosine.
#ifndef AEM_F32_ACCURATE_MATH
#define AEM_F32_ACCURATE_MATH 0
#endif
#ifndef AEM_F32_REDUCE_PHASE
#define AEM_F32_REDUCE_PHASE 0
#endif
//   AEM_F32_POLY_SINCOS=1    the Moebius step's sine and cosine on the FMA
//     pipe: the phase reduced modulo 2 pi as above, then polynomials in x^2
//     on [-pi, pi] (sin x = x P5(x^2), cos x = Q6(x^2); least-squares fits at
//     4000 Chebyshev nodes, absolute error 1e-7 / 1.2e-8 in exact arithmetic,
//     about 6e-7 evaluated in FP32, the hardware approximation's order),
//     paired, 17 FMA-pipe operations per pair of abscissae in place of four
//     special-function ones.
#ifndef AEM_F32_POLY_SINCOS
#define AEM_F32_POLY_SINCOS 0
#endif

__device__ __forceinline__ float rsqrt_approx(float v) {
#if AEM_F32_ACCURATE_MATH
    return __frsqrt_rn(v);
#else
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
#endif
}
__device__ __forceinline__ float sqrt_approx(float v) {
#if AEM_F32_ACCURATE_MATH
    return __fsqrt_rn(v);
#else
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
#endif
}
__device__ __forceinline__ float rcp_approx(float v) {
#if AEM_F32_ACCURATE_MATH
    return __frcp_rn(v);
#else
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
#endif
}
__device__ __forceinline__ float ex2_approx(float v) {
#if AEM_F32_ACCURATE_MATH
    return exp2f(v);
#else
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
#endif
}
__device__ __forceinline__ void sincos_approx(float v, float *s, float *c) {
#if AEM_F32_ACCURATE_MATH
    sincosf(v, s, c);
#else
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(v));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(v));
#endif
}
__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(u64 r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

struct C2x2 {  // two complex numbers: re = (re_a, re_b), im = (im_a, im_b)
    u64 re, im;
};

// Both phases reduced into [-pi, pi] modulo 2 pi, then sine and cosine by
// the polynomials of AEM_F32_POLY_SINCOS (paired FP32 arithmetic only).
__device__ __forceinline__ void sincos2_poly(u64 x, u64 &sn, u64 &cs) {
    const float inv2pi = 0.159154943091895336f, shift = 12582912.0f;
    const float c1 = 6.28318548202514648f, c2 = -1.74845553146951215e-7f;
    const u64 t = fma2(x, pk2(inv2pi, inv2pi), pk2(shift, shift));
    const u64 k = sub2(t, pk2(shift, shift));
    const u64 r = fma2(k, pk2(-c2, -c2), fma2(k, pk2(-c1, -c1), x));
    const u64 r2 = mul2(r, r);
    u64 p = pk2(-2.041758584425679e-08f, -2.041758584425679e-08f);
    p = fma2(p, r2, pk2(2.701278390304651e-06f, 2.701278390304651e-06f));
    p = fma2(p, r2, pk2(-0.00019810261437669396f, -0.00019810261437669396f));
    p = fma2(p, r2, pk2(0.008332478813827038f, 0.008332478813827038f));
    p = fma2(p, r2, pk2(-0.1666656732559204f, -0.1666656732559204f));
    p = fma2(p, r2, pk2(0.9999997019767761f, 0.9999997019767761f));
    sn = mul2(p, r);
    u64 q = pk2(1.729504983671859e-09f, 1.729504983671859e-09f);
    q = fma2(q, r2, pk2(-2.709448949644866e-07f, -2.709448949644866e-07f));
    q = fma2(q, r2, pk2(2.4771701646386646e-05f, 2.4771701646386646e-05f));
    q = fma2(q, r2, pk2(-0.0013887904351577163f, -0.0013887904351577163f));
    q = fma2(q, r2, pk2(0.04166651517152786f, 0.04166651517152786f));
    q = fma2(q, r2, pk2(-0.49999991059303284f, -0.49999991059303284f));
    cs = fma2(q, r2, kOne2);
}

// Both phases of a pair reduced into [-pi, pi] modulo 2 pi (AEM_F32_REDUCE_PHASE):
// the shifter 1.5 * 2^23 rounds x / (2 pi) to the nearest integer k for
// |x| < 2^22 pi; C1 = float(2 pi), C2 = float(2 pi - C1).
__device__ __forceinline__ u64 reduce_2pi2(u64 x) {
#if AEM_F32_REDUCE_PHASE
    const float inv2pi = 0.159154943091895336f, shift = 12582912.0f;
    const float c1 = 6.28318548202514648f, c2 = -1.74845553146951215e-7f;
    const u64 t = fma2(x, pk2(inv2pi, inv2pi), pk2(shift, shift));
    const u64 k = sub2(t, pk2(shift, shift));
    return fma2(k, pk2(-c2, -c2), fma2(k, pk2(-c1, -c1), x));
#else
    return x;
#endif
}

}  // namespace f32x2
}  // namespace aem
