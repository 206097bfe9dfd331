// The periodic Cauchy kernel for a pair of nodes, G = 1/2 cot((zeta_l - zeta_m)/2),
// in double-float or FP64 (shared by the assembly and the target evaluation).
//
// Far field (|d| >= 0.1): separable form of App. E, G = i/2 + i/d with
// d = P_l Q_m - 1, P = e^{i zeta}, Q = e^{-i zeta} (plus the cross terms of
// their third words).  Near field: Delta = zeta_l - zeta_m from the FP64 nodes,
// reduced mod 2 pi in double-double, d = i Delta E(i Delta) with
// E(w) = (e^w - 1)/w by Horner's rule, G = i/2 + 1/(Delta E).
#pragma once
#include "common.cuh"

#define DFC(x) {(float)(x), (float)((x) - (double)(float)(x))}
// 1/(n+1)!, n = 0..11 : Taylor coefficients of E(w) = (e^w - 1)/w
static __constant__ float2 c_taylor_df[12] = {
    DFC(1.0), DFC(1.0 / 2.0), DFC(1.0 / 6.0), DFC(1.0 / 24.0), DFC(1.0 / 120.0),
    DFC(1.0 / 720.0), DFC(1.0 / 5040.0), DFC(1.0 / 40320.0), DFC(1.0 / 362880.0),
    DFC(1.0 / 3628800.0), DFC(1.0 / 39916800.0), DFC(1.0 / 479001600.0)};
static __constant__ double c_taylor64[12] = {
    1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0,
    1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0, 1.0 / 479001600.0};

template <class R> __device__ __forceinline__ R taylor_coef(int n);
template <> __device__ __forceinline__ dfl taylor_coef<dfl>(int n) {
  const float2 c = c_taylor_df[n];
  return {c.x, c.y};
}
template <> __device__ __forceinline__ double taylor_coef<double>(int n) { return c_taylor64[n]; }

#define TWO_PI_HI 6.283185307179586
#define TWO_PI_LO 2.4492935982947064e-16
#define INV_TWO_PI 0.15915494309189535

// Delta = zeta_l - zeta_m reduced to the nearest periodic image (the kernel has
// period 2 pi in Re Delta), in FP64 with a double-double 2 pi.
__device__ __forceinline__ double2 node_delta(double2 zl, double2 zm) {
  double dx = zl.x - zm.x;
  const double dy = zl.y - zm.y;
  const double n = rint(dx * INV_TWO_PI);
  dx = fma(-n, TWO_PI_HI, dx);
  dx = fma(-n, TWO_PI_LO, dx);
  return make_double2(dx, dy);
}

// R = Delta * E(i Delta): then i/d = 1/R with d = e^{i Delta} - 1.
template <class R>
__device__ __forceinline__ cx<R> near_R(double2 dlt) {
  const cx<R> D = {r_from_double<R>(dlt.x), r_from_double<R>(dlt.y)};
  const cx<R> w = {r_neg(D.im), D.re};
  const float m2 = (float)(dlt.x * dlt.x + dlt.y * dlt.y);
  const int K = m2 < 1.6e-5f ? 5 : (m2 < 4e-4f ? 7 : (m2 < 3.6e-3f ? 9 : 11));
  cx<R> E = {taylor_coef<R>(K), r_from_double<R>(0.0)};
  for (int n = K - 1; n >= 0; --n) {
    E = c_mul(E, w);
    E.re = r_add(E.re, taylor_coef<R>(n));
  }
  return c_mul(D, E);
}

// w = P Q plus the cross terms of the third words (double-float only)
__device__ __forceinline__ void pq_product(const cx<double>& P, const cx<double>& Q, float2, float2,
                                           double& wr, double& wi) {
  wr = P.re * Q.re - P.im * Q.im;
  wi = P.re * Q.im + P.im * Q.re;
}
__device__ __forceinline__ void pq_product(const cx<dfl>& P, const cx<dfl>& Q, float2 Pc, float2 Qc,
                                           dfl& wr, dfl& wi) {
  wr = P.re * Q.re - P.im * Q.im;
  wi = P.re * Q.im + P.im * Q.re;
  float cr = P.re.hi * Qc.x;
  cr = fmaf(-P.im.hi, Qc.y, cr);
  cr = fmaf(Pc.x, Q.re.hi, cr);
  cr = fmaf(-Pc.y, Q.im.hi, cr);
  float ci = P.re.hi * Qc.y;
  ci = fmaf(P.im.hi, Qc.x, ci);
  ci = fmaf(Pc.x, Q.im.hi, ci);
  ci = fmaf(Pc.y, Q.re.hi, ci);
  wr = df_addf(wr, cr);
  wi = df_addf(wi, ci);
}

// G = 1/2 cot((zeta_l - zeta_m)/2) for l != m: far field i/2 + i/d, near field i/2 + 1/R.
template <class R>
__device__ __forceinline__ cx<R> half_cot_pair(const cx<R>& P, const cx<R>& Q, float2 Pc, float2 Qc,
                                               double2 zl, double2 zm, float near2) {
  R wr, wi;
  pq_product(P, Q, Pc, Qc, wr, wi);
  const R dr = r_addf(wr, -1.0f);
  const R n2 = r_add(r_sqr(dr), r_sqr(wi));
  cx<R> G;
  if (r_hi(n2) < near2) {
    const cx<R> Rv = near_R<R>(node_delta(zl, zm));
    const R inv = r_rcp(r_add(r_sqr(Rv.re), r_sqr(Rv.im)));
    G.re = r_mul(Rv.re, inv);
    G.im = r_addf(r_neg(r_mul(Rv.im, inv)), 0.5f);
  } else {
    const R inv = r_rcp(n2);
    G.re = r_mul(wi, inv);
    G.im = r_addf(r_mul(dr, inv), 0.5f);
  }
  return G;
}

template <class R>
__device__ __forceinline__ R cre(const cx<R>& Z, const cx<R>& G) {  // Re{Z G}
  return r_sub(r_mul(Z.re, G.re), r_mul(Z.im, G.im));
}
template <class R>
__device__ __forceinline__ R cim(const cx<R>& Z, const cx<R>& G) {  // Im{Z G}
  return r_add(r_mul(Z.re, G.im), r_mul(Z.im, G.re));
}

