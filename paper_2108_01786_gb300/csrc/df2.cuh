// Double-float arithmetic on two independent lanes at once.
//
// A double-float number is an unevaluated sum hi + lo of two FP32 values
// (about 48 significant bits; Hida, Li & Bailey's construction with
// Knuth's TwoSum and an FMA-based TwoProd).  The Blackwell FP32 datapath
// executes packed pairs: one FADD2 / FMUL2 / FFMA2 warp instruction gives two
// FP32 results per thread.  df2 carries two double-float numbers (lane x and
// lane y) in float2 registers, so every step below costs one issue slot for
// both lanes.  The combined forms (a b + c d + k with one renormalisation)
// replace chains of separate products and sums: the exact parts of the
// products and of the sum are kept by TwoProd / TwoSum, every low-order part
// goes into one error term, and a single Fast2Sum renormalises at the end;
// the result is within a few units of 2^-48 of |a b| + |c d| + |k|.
#pragma once
#include <cuda_runtime.h>

struct df2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once: b * (-1) + a
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df2 d2_neg(df2 a) { return {p_neg(a.hi), p_neg(a.lo)}; }

__device__ __forceinline__ df2 d2_two_sum(float2 a, float2 b) {
  const float2 s = p_add(a, b);
  const float2 bb = p_sub(s, a);
  const float2 e = p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb));
  return {s, e};
}
__device__ __forceinline__ df2 d2_fast_two_sum(float2 a, float2 b) {
  const float2 s = p_add(a, b);
  return {s, p_sub(b, p_sub(s, a))};
}

// a + b
__device__ __forceinline__ df2 d2_add(df2 a, df2 b) {
  const df2 s = d2_two_sum(a.hi, b.hi);
  return d2_fast_two_sum(s.hi, p_add(s.lo, p_add(a.lo, b.lo)));
}

// a * b
__device__ __forceinline__ df2 d2_mul(df2 a, df2 b) {
  const float2 p = p_mul(a.hi, b.hi);
  float2 e = p_fma(a.hi, b.hi, p_neg(p));
  e = p_fma(a.hi, b.lo, e);
  e = p_fma(a.lo, b.hi, e);
  return d2_fast_two_sum(p, e);
}

// a * b + k (k a plain FP32 constant, added exactly)
__device__ __forceinline__ df2 d2_mul_addf(df2 a, df2 b, float2 k) {
  const float2 p = p_mul(a.hi, b.hi);
  float2 e = p_fma(a.hi, b.hi, p_neg(p));
  const df2 s = d2_two_sum(p, k);
  e = p_add(e, s.lo);
  e = p_fma(a.hi, b.lo, e);
  e = p_fma(a.lo, b.hi, e);
  return d2_fast_two_sum(s.hi, e);
}

// a * b + c * d (+ khi added exactly when K) + elo (a low-order FP32 term)
template <bool K>
__device__ __forceinline__ df2 d2_dot2(df2 a, df2 b, df2 c, df2 d, float2 khi, float2 elo) {
  const float2 p1 = p_mul(a.hi, b.hi);
  const float2 e1 = p_fma(a.hi, b.hi, p_neg(p1));
  const float2 p2 = p_mul(c.hi, d.hi);
  const float2 e2 = p_fma(c.hi, d.hi, p_neg(p2));
  const df2 s = d2_two_sum(p1, p2);
  float2 e = p_add(p_add(e1, e2), p_add(s.lo, elo));
  float2 h = s.hi;
  if (K) {
    const df2 u = d2_two_sum(s.hi, khi);
    h = u.hi;
    e = p_add(e, u.lo);
  }
  e = p_fma(a.hi, b.lo, e);
  e = p_fma(a.lo, b.hi, e);
  e = p_fma(c.hi, d.lo, e);
  e = p_fma(c.lo, d.hi, e);
  return d2_fast_two_sum(h, e);
}

// 1 / b: the hardware approximation r per lane, then one Newton step with its
// second-order term, e = 1 - b r, 1/b = r (1 + e + e^2 + ...)
__device__ __forceinline__ df2 d2_rcp(df2 b) {
  float2 r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r.x) : "f"(b.hi.x));
  asm("rcp.approx.f32 %0, %1;" : "=f"(r.y) : "f"(b.hi.y));
  float2 e = p_fma(p_neg(b.hi), r, f2(1.f));
  e = p_fma(p_neg(b.lo), r, e);
  const float2 re = p_mul(r, e);
  return d2_fast_two_sum(r, p_fma(re, e, re));
}
