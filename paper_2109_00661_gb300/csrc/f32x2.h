// Paired FP32 arithmetic and the hardware approximations shared by the FP32
// forward kernel (forward.cu) and its adjoint (adjoint.cu).
//
// Two values (two Hankel abscissae of one frequency in both kernels) travel
// in one 64-bit register pair and are advanced with the sm_100+ paired FP32
// instructions (add/sub/mul/fma .rn.f32x2): one issue slot per operation on
// both.  The special functions (rsqrt, rcp, ex2, sin, cos) are the hardware
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

__device__ __forceinline__ float rsqrt_approx(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float rcp_approx(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float ex2_approx(float v) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ void sincos_approx(float v, float *s, float *c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(v));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(v));
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

}  // namespace f32x2
}  // namespace aem
