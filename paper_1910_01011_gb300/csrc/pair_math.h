// pair_math.h -- packed FP32 on sm_103a: two values per float2, one
// FFMA2 / FADD2 / FMUL2 for both lanes, and the MUFU approximations the
// far-field and field kernels use (PTX .approx.ftz forms).
#pragma once

#include <cuda_runtime.h>

namespace gbem {

typedef float2 f2;

__device__ __forceinline__ f2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 neg2(f2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void sincos_approx(float x, float* s, float* c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(x));
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace gbem
