// Inner-product helpers shared by the single-problem and batched GEMVs:
// 16-byte dot products of stored matrix entries (FP32, FP16, BF16) with FP32
// vectors, and the double-float product-accumulate of the hi + lo residual.
#pragma once
#include "common.cuh"

template <class TA> struct Dot16;
template <> struct Dot16<float> {
  static constexpr int E = 4;
  static __device__ __forceinline__ float run(float acc, const uint4& q, const float* xs) {
    const float4 b = *reinterpret_cast<const float4*>(xs);
    acc = fmaf(__uint_as_float(q.x), b.x, acc);
    acc = fmaf(__uint_as_float(q.y), b.y, acc);
    acc = fmaf(__uint_as_float(q.z), b.z, acc);
    acc = fmaf(__uint_as_float(q.w), b.w, acc);
    return acc;
  }
};
template <> struct Dot16<__half> {
  static constexpr int E = 8;
  static __device__ __forceinline__ float run(float acc, const uint4& q, const float* xs) {
    const float4 b0 = *reinterpret_cast<const float4*>(xs);
    const float4 b1 = *reinterpret_cast<const float4*>(xs + 4);
    float2 f;
    f = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    acc = fmaf(f.x, b0.x, acc);
    acc = fmaf(f.y, b0.y, acc);
    f = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    acc = fmaf(f.x, b0.z, acc);
    acc = fmaf(f.y, b0.w, acc);
    f = __half22float2(*reinterpret_cast<const __half2*>(&q.z));
    acc = fmaf(f.x, b1.x, acc);
    acc = fmaf(f.y, b1.y, acc);
    f = __half22float2(*reinterpret_cast<const __half2*>(&q.w));
    acc = fmaf(f.x, b1.z, acc);
    acc = fmaf(f.y, b1.w, acc);
    return acc;
  }
};
template <> struct Dot16<__nv_bfloat16> {
  static constexpr int E = 8;
  static __device__ __forceinline__ float run(float acc, const uint4& q, const float* xs) {
    const float4 b0 = *reinterpret_cast<const float4*>(xs);
    const float4 b1 = *reinterpret_cast<const float4*>(xs + 4);
    float2 f;
    f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
    acc = fmaf(f.x, b0.x, acc);
    acc = fmaf(f.y, b0.y, acc);
    f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
    acc = fmaf(f.x, b0.z, acc);
    acc = fmaf(f.y, b0.w, acc);
    f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.z));
    acc = fmaf(f.x, b1.x, acc);
    acc = fmaf(f.y, b1.y, acc);
    f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.w));
    acc = fmaf(f.x, b1.z, acc);
    acc = fmaf(f.y, b1.w, acc);
    return acc;
  }
};

// s + (ah + al)(xh + xl) in double-float (the al xl term is below the precision)
__device__ __forceinline__ dfl df_acc_prod(dfl s, float ah, float al, float xh, float xl) {
  const dfl p = df_two_prod(ah, xh);
  float e = fmaf(ah, xl, p.lo);
  e = fmaf(al, xh, e);
  const dfl t = df_two_sum(s.hi, p.hi);
  const float lo = t.lo + (s.lo + e);
  return df_fast_two_sum(t.hi, lo);
}

