// A pair of FP32 lanes, one per site, whose arithmetic issues as the packed
// two-lane instructions of sm_100 and later (fma.rn.f32x2, add.rn.f32x2,
// mul.rn.f32x2): one instruction performs the same operation on both sites,
// with the rounding of the scalar instruction in each lane.  The FP32
// link arithmetic (link_alg.cuh) is written for a lane type T, so T = f2
// evaluates two sites in the issue slots of one.
//
// Data-dependent control flow (the scaling loop of the exponential, the
// branch of the re-unitarisation factor) takes one path for both lanes:
// the helpers below reduce a lane predicate to "any lane" or "all lanes".
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace glasma {

struct f2 {
  float2 v;
  __device__ __forceinline__ f2() {}
  __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit f2(float2 a) : v(a) {}
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.v.x, -a.v.y); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(float a, f2 b) { return f2(__fmul2_rn(make_float2(a, a), b.v)); }
__device__ __forceinline__ f2& operator+=(f2& a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2& operator-=(f2& a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2& operator*=(f2& a, f2 b) { return a = a * b; }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }

// lane predicates
__device__ __forceinline__ bool any_gt(f2 a, float b) { return a.v.x > b || a.v.y > b; }
__device__ __forceinline__ bool all_zero(f2 a) { return a.v.x == 0.f && a.v.y == 0.f; }
__device__ __forceinline__ bool all_abs_lt(f2 a, float b) { return fabsf(a.v.x) < b && fabsf(a.v.y) < b; }
__device__ __forceinline__ bool any_gt(float a, float b) { return a > b; }
__device__ __forceinline__ bool all_zero(float a) { return a == 0.f; }
__device__ __forceinline__ bool all_abs_lt(float a, float b) { return fabsf(a) < b; }

// per-lane functions without a packed form
__device__ __forceinline__ f2 lane_sqrt(f2 a) { return f2(sqrtf(a.v.x), sqrtf(a.v.y)); }
__device__ __forceinline__ f2 lane_abs(f2 a) { return f2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ f2 lane_div(f2 a, f2 b) { return f2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ f2 lane_sincos_s(f2 a, f2* c) {
  float s0, c0, s1, c1;
  sincosf(a.v.x, &s0, &c0);
  sincosf(a.v.y, &s1, &c1);
  *c = f2(c0, c1);
  return f2(s0, s1);
}

}  // namespace glasma
