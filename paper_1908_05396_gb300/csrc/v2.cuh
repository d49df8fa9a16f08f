// v2.cuh -- a pair of FP32 values, one per node, computed with the packed
// FP32 instructions of sm_100+ (two lanes per add, multiply or fused
// multiply-add).  The collision template runs on it unchanged, so one thread
// collides two nodes for the arithmetic instructions of one.
#pragma once

#include <cuda_runtime.h>

namespace clbm {

// Keep the scalar overloads visible next to the V2 ones below.
using ::fmax;
using ::fmin;
using ::sqrt;

struct V2 {
  float2 v;
  __device__ __forceinline__ V2() {}
  __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ V2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ V2(double s) : v(make_float2(float(s), float(s))) {}
  __device__ __forceinline__ V2(int s) : v(make_float2(float(s), float(s))) {}
  __device__ __forceinline__ explicit V2(float2 f) : v(f) {}
};

__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ V2 operator-(V2 a) { return V2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ V2& operator+=(V2& a, V2 b) { a = a + b; return a; }
__device__ __forceinline__ V2& operator-=(V2& a, V2 b) { a = a - b; return a; }
__device__ __forceinline__ V2& operator*=(V2& a, V2 b) { a = a * b; return a; }
__device__ __forceinline__ V2 operator+(V2 a, float b) { return a + V2(b); }
__device__ __forceinline__ V2 operator+(float a, V2 b) { return V2(a) + b; }
__device__ __forceinline__ V2 operator-(V2 a, float b) { return a - V2(b); }
__device__ __forceinline__ V2 operator-(float a, V2 b) { return V2(a) - b; }
__device__ __forceinline__ V2 operator*(V2 a, float b) { return a * V2(b); }
__device__ __forceinline__ V2 operator*(float a, V2 b) { return V2(a) * b; }

__device__ __forceinline__ V2 fma(V2 a, V2 b, V2 c) { return V2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ V2 fmax(V2 a, V2 b) {
  return V2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y));
}
__device__ __forceinline__ V2 fmin(V2 a, V2 b) {
  return V2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y));
}
__device__ __forceinline__ V2 sqrt(V2 a) { return V2(sqrtf(a.v.x), sqrtf(a.v.y)); }

__device__ __forceinline__ float lane0(V2 a) { return a.v.x; }
__device__ __forceinline__ float lane1(V2 a) { return a.v.y; }

}  // namespace clbm
