// Arithmetic on one site (float) or on two sites at once (float2). The float2 forms map
// to Blackwell's packed FP32 instructions (__fadd2_rn / __fmul2_rn / __ffma2_rn): one
// instruction performs the same IEEE round-to-nearest operation on both halves, so a
// thread that owns two lattice sites issues each step of the per-site algebra once.
#pragma once

#include <cuda_runtime.h>

namespace flbm {

__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }

// FP64 forms, for set-up code that evaluates the same generated algebra in double.
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

template <typename T>
__device__ __forceinline__ T splat(float x);
template <>
__device__ __forceinline__ float splat<float>(float x) {
  return x;
}
template <>
__device__ __forceinline__ float2 splat<float2>(float x) {
  return make_float2(x, x);
}
template <>
__device__ __forceinline__ double splat<double>(float x) {
  return (double)x;
}

// A constant given in double, rounded once to the value type (generated code).
template <typename T>
__device__ __forceinline__ T rat(double x);
template <>
__device__ __forceinline__ float rat<float>(double x) {
  return (float)x;
}
template <>
__device__ __forceinline__ float2 rat<float2>(double x) {
  return make_float2((float)x, (float)x);
}
template <>
__device__ __forceinline__ double rat<double>(double x) {
  return x;
}

// Number of sites a value of type T carries.
template <typename T>
struct Lanes;
template <>
struct Lanes<float> {
  static constexpr int n = 1;
};
template <>
struct Lanes<float2> {
  static constexpr int n = 2;
};

// Per-lane access (lane 0 = first site, lane 1 = second site).
__device__ __forceinline__ float lane(float v, int) { return v; }
__device__ __forceinline__ float lane(float2 v, int l) { return l == 0 ? v.x : v.y; }
__device__ __forceinline__ void set_lane(float &v, int, float x) { v = x; }
__device__ __forceinline__ void set_lane(float2 &v, int l, float x) {
  if (l == 0)
    v.x = x;
  else
    v.y = x;
}

// 1 / x and sqrt(x) of each lane by the hardware approximations (PTX rcp.approx.ftz and
// sqrt.approx.ftz: within about one unit in the last place for the positive normal
// densities the step sees), instead of the IEEE-rounded division and square root, whose
// refinement and special-case paths cost several instructions per lane.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_fast_lanes(float x) { return rcp_fast(x); }
__device__ __forceinline__ float2 rcp_fast_lanes(float2 x) { return make_float2(rcp_fast(x.x), rcp_fast(x.y)); }
__device__ __forceinline__ float sqrt_fast_lanes(float x) { return sqrt_fast(x); }
__device__ __forceinline__ float2 sqrt_fast_lanes(float2 x) { return make_float2(sqrt_fast(x.x), sqrt_fast(x.y)); }

}  // namespace flbm
