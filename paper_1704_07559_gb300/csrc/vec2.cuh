// vec2.cuh -- two lattice nodes per thread in packed FP32 arithmetic.
//
// Blackwell executes FP32 add, multiply and fused multiply-add on a pair of values as one
// instruction (__fadd2_rn, __fmul2_rn, __ffma2_rn, sm_100 and later).  The step kernel is written
// once over a scalar type R; F2 is a drop-in R holding the same quantity for two x-adjacent
// nodes, so each arithmetic instruction advances both.  Every operation rounds each lane exactly
// as the scalar float operation would (subtraction is a - b = fma(b, -1, a), exact in one rounding).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct F2 {
    float2 v;
    F2() = default;
    __host__ __device__ constexpr explicit F2(float s) : v{s, s} {}
    __host__ __device__ constexpr F2(float a, float b) : v{a, b} {}
    __host__ __device__ constexpr explicit F2(float2 u) : v(u) {}
    __device__ __forceinline__ float lo() const { return v.x; }
    __device__ __forceinline__ float hi() const { return v.y; }
};

// scalar fused multiply-add under the same name, so code written over R finds one overload set
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.0f, -1.0f))); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }

// scalar type of a (possibly packed) compute type
template <class R>
struct Scalar {
    using T = R;
};
template <>
struct Scalar<F2> {
    using T = float;
};

}  // namespace lbm
