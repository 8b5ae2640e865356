// lb_pair.cuh -- two FP32 lanes in one register pair, computed with the
// packed FP32x2 instructions of sm_100 and later (one issue slot for two
// node updates).
//
// Every operator is the lane-wise IEEE operation with round-to-nearest-even,
// exactly as the scalar FP32 instruction it replaces (a - b is evaluated as
// a + (-b), which rounds identically), so the per-node arithmetic of
// lb_collide.cuh instantiated with f32x2 produces, lane by lane, the same bits
// as its scalar float instantiation.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbgb {

struct f32x2 {
  float x, y;
  __host__ __device__ constexpr f32x2() : x(0.0f), y(0.0f) {}
  __host__ __device__ constexpr f32x2(float a, float b) : x(a), y(b) {}
  // broadcast (the scalar conversion of the value, in both lanes)
  __host__ __device__ constexpr explicit f32x2(float v) : x(v), y(v) {}
  __host__ __device__ constexpr explicit f32x2(double v) : x(float(v)), y(float(v)) {}
  __host__ __device__ constexpr explicit f32x2(int v) : x(float(v)), y(float(v)) {}
};

__device__ __forceinline__ float2 as_f2(f32x2 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f32x2 of_f2(float2 v) { return f32x2(v.x, v.y); }

__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) { return of_f2(__fadd2_rn(as_f2(a), as_f2(b))); }
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return f32x2(-a.x, -a.y); }
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) { return of_f2(__fadd2_rn(as_f2(a), as_f2(-b))); }
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) { return of_f2(__fmul2_rn(as_f2(a), as_f2(b))); }
__device__ __forceinline__ f32x2 fma_r(f32x2 a, f32x2 b, f32x2 c) {
  return of_f2(__ffma2_rn(as_f2(a), as_f2(b), as_f2(c)));
}

// ------------------------------------------------------------ storage pairs
// two adjacent stored values <-> one f32x2 (the address must be aligned to
// two elements)
template <class S>
__device__ __forceinline__ f32x2 load_pair(const S* p);
template <>
__device__ __forceinline__ f32x2 load_pair<float>(const float* p) {
  return of_f2(*reinterpret_cast<const float2*>(p));
}
template <>
__device__ __forceinline__ f32x2 load_pair<__half>(const __half* p) {
  return of_f2(__half22float2(*reinterpret_cast<const __half2*>(p)));
}
template <>
__device__ __forceinline__ f32x2 load_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
  return of_f2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p)));
}

template <class S>
__device__ __forceinline__ void store_pair(S* p, f32x2 v);
template <>
__device__ __forceinline__ void store_pair<float>(float* p, f32x2 v) {
  *reinterpret_cast<float2*>(p) = as_f2(v);
}
template <>
__device__ __forceinline__ void store_pair<__half>(__half* p, f32x2 v) {
  // lane-wise round-to-nearest-even, as __float2half_rn
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.x, v.y);
}
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* p, f32x2 v) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
}

}  // namespace lbgb
