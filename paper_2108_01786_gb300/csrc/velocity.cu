// Normal velocity of the free surface, Sec. 3.4:
//   s_alpha U = [eq. d:phi:mv] + sum_{j>=1} (1/M_j) sum_l K_j0(beta_l, alpha) omega_j'(beta_l)
//             - 1/2 H omega_0' - (1/M_0) sum_l G_00(beta_l, alpha) omega_0'(beta_l)
// with K_j0(beta, alpha) = Im{zeta_0'(alpha) C},  G_00(beta, alpha) = Re{zeta_0'(alpha) C}
// - 1/2 cot((alpha - beta)/2) and C = 1/2 cot((zeta_0(alpha) - zeta_j(beta))/2),
// diagonal limit G_00(alpha, alpha) = Re{zeta''/(2 zeta')}.
//
// Since zeta_0'(alpha) does not depend on the source, only the complex sums
//   s1 = sum_{l not on Gamma_0} C_ml c_l,   s0 = sum_{l on Gamma_0, l != m} C_ml c_l,
//   t0 = sum_{l on Gamma_0, l != m} 1/2 cot(pi (m - l)/M_0) c_l,   c_l = omega_l' / M_l,
// are formed per target, with C_ml = -(i/2 + i/d_ml), d_ml = P_l Q_m - 1 (far) or
// from the FP64 node difference (near), exactly as in the assembly.
// omega' and H omega_0' are circulant products with the spectral kernels of
// each boundary (symbols ik and |k|, Nyquist mode zero), in double-float.
#include <cstring>

#include <cmath>
#include "common.cuh"
#include "nvtx.cuh"
#include "dft.cuh"


#define TWO_PI_HI_V 6.283185307179586
#define TWO_PI_LO_V 2.4492935982947064e-16
#define INV_TWO_PI_V 0.15915494309189535

__constant__ float2 c_taylor_v[12] = {
#define DFCV(x) {(float)(x), (float)((x) - (double)(float)(x))}
    DFCV(1.0), DFCV(1.0 / 2.0), DFCV(1.0 / 6.0), DFCV(1.0 / 24.0), DFCV(1.0 / 120.0),
    DFCV(1.0 / 720.0), DFCV(1.0 / 5040.0), DFCV(1.0 / 40320.0), DFCV(1.0 / 362880.0),
    DFCV(1.0 / 3628800.0), DFCV(1.0 / 39916800.0), DFCV(1.0 / 479001600.0)};

// Delta = zeta_l - zeta_m reduced to the nearest periodic image, then
// R = Delta E(i Delta), E(w) = (e^w - 1)/w, so that i/d = 1/R for d = e^{i Delta} - 1.
__device__ __forceinline__ cx<dfl> near_R_v(double2 zl, double2 zm) {
  double dx = zl.x - zm.x;
  const double dy = zl.y - zm.y;
  const double n = rint(dx * INV_TWO_PI_V);
  dx = fma(-n, TWO_PI_HI_V, dx);
  dx = fma(-n, TWO_PI_LO_V, dx);
  const cx<dfl> D = {df_from_double(dx), df_from_double(dy)};
  const cx<dfl> w = {-D.im, D.re};
  const float m2 = (float)(dx * dx + dy * dy);
  const int K = m2 < 1.6e-5f ? 5 : (m2 < 4e-4f ? 7 : (m2 < 3.6e-3f ? 9 : 11));
  cx<dfl> E = {{c_taylor_v[K].x, c_taylor_v[K].y}, {0.f, 0.f}};
  for (int k = K - 1; k >= 0; --k) {
    E = c_mul(E, w);
    E.re = E.re + dfl{c_taylor_v[k].x, c_taylor_v[k].y};
  }
  return c_mul(D, E);
}

// ---------------------------------------------------------------------------
// Spectral derivative and Hilbert transform by a four-step DFT in FP64.
// For a boundary of M = M1 M2 points, X[k1 + M1 k2] = sum_{n2} W^{M1 n2 k2}
// [W^{n2 k1} sum_{n1} x[M2 n1 + n2] W^{M2 n1 k1}],  W = e^{-2 pi i / M}
// (two passes of direct sums of length M1 and M2).  omega' = IDFT(i k X) and
// H omega_0' = IDFT(|k| X) (signed wavenumber k, Nyquist mode zero), the
// inverse taken as conj(DFT(conj(.)))/M.  A direct circulant convolution with
// the derivative kernel (entries up to M/2pi of alternating sign) loses too
// many digits; the DFT keeps FP64 accuracy in every mode.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dft_find(const DftJobs& J, int t) {
  int lo = 0;
  while (lo + 1 < J.n && t >= J.j[lo + 1].start) ++lo;
  return lo;
}

__device__ __forceinline__ double signed_k(int i, int M) {
  if (2 * i == M) return 0.0;           // Nyquist mode set to zero (even M)
  return (double)(2 * i < M ? i : i - M);
}

__device__ __forceinline__ double2 dft_input(const DftJob& jb, const double* __restrict__ xr,
                                             const double2* __restrict__ xc, int i) {
  if (jb.mode == 0) return make_double2(xr[jb.off_in + i], 0.0);
  const double2 X = xc[jb.off_in + i];
  if (jb.mode == 3) return X;                                    // complex input as is
  if (jb.mode == 6) {                                            // conj(rho(k) X), eq. filter
    const int ka = (2 * i <= jb.M) ? i : jb.M - i;               // |k|, Nyquist at M/2
    const double r = (double)ka / (0.5 * (double)jb.M);
    const double rho = exp(-36.0 * pow(r, 36.0));
    return make_double2(rho * X.x, -rho * X.y);
  }
  const double k = signed_k(i, jb.M);
  if (jb.mode == 5) return make_double2(-k * k * X.x, k * k * X.y);   // conj(-k^2 X)
  if (jb.mode == 7) {                                            // conj(X/(ik)), 0 at k = 0
    if (k == 0.0) return make_double2(0.0, 0.0);
    return make_double2(X.y / k, X.x / k);
  }
  if (jb.mode == 4) {                                            // conj(-i sgn(k) X)
    const double sg = (k > 0.0) ? 1.0 : (k < 0.0 ? -1.0 : 0.0);
    return make_double2(sg * X.y, sg * X.x);
  }
  if (jb.mode == 1) return make_double2(-k * X.y, -k * X.x);   // conj(i k X)
  const double ak = fabs(k);
  return make_double2(ak * X.x, -ak * X.y);                      // conj(|k| X)
}

// Each output is summed by DFT_SPLIT consecutive lanes (strided terms, a fixed
// shuffle tree), so a transform of M points keeps DFT_SPLIT M threads busy.
__device__ __forceinline__ unsigned dft_group_mask() {
  const unsigned lane = threadIdx.x & 31;
  return ((1u << DFT_SPLIT) - 1u) << (lane & ~(unsigned)(DFT_SPLIT - 1));
}

__device__ __forceinline__ void dft_group_sum(double& sr, double& si) {
  const unsigned mask = dft_group_mask();
#pragma unroll
  for (int o = DFT_SPLIT / 2; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(mask, sr, o);
    si += __shfl_xor_sync(mask, si, o);
  }
}

// pass A: Y[n2 M1 + k1] = W^{n2 k1} sum_{n1} x[M2 n1 + n2] W^{M2 n1 k1}
__global__ void k_dft_a(DftJobs J, const double* __restrict__ xr, const double2* __restrict__ xc,
                        const double2* __restrict__ tw, double2* __restrict__ Y,
                        long long in_stride, long long out_stride) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = (int)(gt / DFT_SPLIT), sub = (int)(gt % DFT_SPLIT);
  if (t >= J.total) return;   // whole groups leave together
  if (xr) xr += blockIdx.y * in_stride;
  if (xc) xc += blockIdx.y * in_stride;
  Y += blockIdx.y * out_stride;
  const DftJob jb = J.j[dft_find(J, t)];
  const int q = t - jb.start;
  const int n2 = q / jb.M1, k1 = q - n2 * jb.M1;
  const int M = jb.M;
  const long long step = ((long long)jb.M2 * k1) % M;
  int idx = (int)((step * sub) % M);
  const int inc = (int)((step * DFT_SPLIT) % M);
  double sr = 0.0, si = 0.0;
  for (int n1 = sub; n1 < jb.M1; n1 += DFT_SPLIT) {
    const double2 x = dft_input(jb, xr, xc, jb.M2 * n1 + n2);
    const double2 w = tw[jb.off_tw + idx];
    sr = fma(x.x, w.x, fma(-x.y, w.y, sr));
    si = fma(x.x, w.y, fma(x.y, w.x, si));
    idx += inc;
    if (idx >= M) idx -= M;
  }
  dft_group_sum(sr, si);
  if (sub == 0) {
    const double2 w = tw[jb.off_tw + (int)(((long long)n2 * k1) % M)];
    Y[jb.off_out + q] = make_double2(sr * w.x - si * w.y, sr * w.y + si * w.x);
  }
}

// pass B: X[k1 + M1 k2] = sum_{n2} Y[n2 M1 + k1] W^{M1 n2 k2}
__global__ void k_dft_b(DftJobs J, const double2* __restrict__ Y, const double2* __restrict__ tw,
                        double2* __restrict__ X, long long stride) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = (int)(gt / DFT_SPLIT), sub = (int)(gt % DFT_SPLIT);
  if (t >= J.total) return;
  Y += blockIdx.y * stride;
  X += blockIdx.y * stride;
  const DftJob jb = J.j[dft_find(J, t)];
  const int q = t - jb.start;
  const int k2 = q / jb.M1, k1 = q - k2 * jb.M1;
  const int M = jb.M;
  const long long step = ((long long)jb.M1 * k2) % M;
  int idx = (int)((step * sub) % M);
  const int inc = (int)((step * DFT_SPLIT) % M);
  double sr = 0.0, si = 0.0;
  for (int n2 = sub; n2 < jb.M2; n2 += DFT_SPLIT) {
    const double2 y = Y[jb.off_out + n2 * jb.M1 + k1];
    const double2 w = tw[jb.off_tw + idx];
    sr = fma(y.x, w.x, fma(-y.y, w.y, sr));
    si = fma(y.x, w.y, fma(y.y, w.x, si));
    idx += inc;
    if (idx >= M) idx -= M;
  }
  dft_group_sum(sr, si);
  if (sub == 0) X[jb.off_out + q] = make_double2(sr, si);
}

// spectra -> omega'/M_l (df, all nodes), omega' and H omega_0' (real part / M)
__global__ void k_dft_extract(Blocks B, const double2* __restrict__ X2, float2* __restrict__ cw,
                              float2* __restrict__ hw0, float* __restrict__ xh,
                              float* __restrict__ xl, double* __restrict__ wp64, long long ld) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // vector blockIdx.y of a batch (cw and wp64 are not batched)
  X2 += blockIdx.y * (long long)(B.N + B.M[0]);
  hw0 += blockIdx.y * (long long)B.M[0];
  if (xh) {
    xh += blockIdx.y * ld;
    xl += blockIdx.y * ld;
  }
  if (xh && t >= B.N + B.M[0] && t < ld + B.M[0]) {  // zero padding of xh, xl
    const int p = t - B.M[0];
    xh[p] = 0.f;
    xl[p] = 0.f;
    return;
  }
  if (t >= B.N + B.M[0]) return;
  if (t < B.N) {
    int k = 0;
    while (k + 1 < B.nb && t >= B.off[k + 1]) ++k;
    const double M = (double)B.M[k];
    const double d = X2[t].x / M;            // omega'
    const dfl c = df_from_double(d / M);     // omega' / M_k
    if (cw) cw[t] = make_float2(c.hi, c.lo);
    if (xh) {
      xh[t] = c.hi;
      xl[t] = c.lo;
    }
    if (wp64) wp64[t] = d;
  } else {
    const int m = t - B.N;
    const double h = X2[t].x / (double)B.M[0];
    const dfl hh = df_from_double(h);
    hw0[m] = make_float2(hh.hi, hh.lo);
  }
}

#define VEL_CH 1024
#define VEL_FIELDS 8   // S1.re S1.im cs1 S0.re S0.im cs0 t0 (pad)

__global__ void __launch_bounds__(256) k_velocity_partial(
    int N, int M0, const float4* __restrict__ nP, const float4* __restrict__ nQ,
    const float4* __restrict__ nPQc, const double2* __restrict__ z64, const int* __restrict__ blk, const float2* __restrict__ cw,
    const float2* __restrict__ Ttab, float near2, float2* __restrict__ part) {
  __shared__ float4 sP[VEL_CH];
  __shared__ float2 sPc[VEL_CH];
  __shared__ double2 sZ[VEL_CH];
  __shared__ float2 sC[VEL_CH];
  __shared__ int sB[VEL_CH];
  const int s0 = blockIdx.y * VEL_CH;
  const int ns = min(VEL_CH, N - s0);
  for (int t = threadIdx.x; t < ns; t += blockDim.x) {
    sP[t] = nP[s0 + t];
    const float4 pq = nPQc[s0 + t];
    sPc[t] = make_float2(pq.x, pq.y);
    sZ[t] = z64[s0 + t];
    sC[t] = cw[s0 + t];
    sB[t] = blk[s0 + t];
  }
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M0) return;
  const float4 qv = nQ[m];
  const dfl qr = {qv.x, qv.y}, qi = {qv.z, qv.w};
  const float4 qc4 = nPQc[m];
  const float qcr = qc4.z, qci = qc4.w;
  const double2 zm = z64[m];
  dfl S1r = {0, 0}, S1i = {0, 0}, cs1 = {0, 0}, S0r = {0, 0}, S0i = {0, 0}, cs0 = {0, 0}, t0 = {0, 0};
  for (int t = 0; t < ns; ++t) {
    const int l = s0 + t;
    if (l == m) continue;
    const float4 pv = sP[t];
    const dfl pr = {pv.x, pv.y}, pi = {pv.z, pv.w};
    const float2 cv = sC[t];
    const dfl c = {cv.x, cv.y};
    const float2 pc = sPc[t];
    float cr = pr.hi * qcr;
    cr = fmaf(-pi.hi, qci, cr);
    cr = fmaf(pc.x, qr.hi, cr);
    cr = fmaf(-pc.y, qi.hi, cr);
    float ci = pr.hi * qci;
    ci = fmaf(pi.hi, qcr, ci);
    ci = fmaf(pc.x, qi.hi, ci);
    ci = fmaf(pc.y, qr.hi, ci);
    const dfl wr = df_addf(pr * qr - pi * qi, cr);
    const dfl wi = df_addf(pr * qi + pi * qr, ci);
    const dfl dr = df_addf(wr, -1.0f);
    const dfl n2 = df_sqr(dr) + df_sqr(wi);
    dfl ar, ai;  // (1/d) c
    if (n2.hi < near2) {
      const cx<dfl> Rv = near_R_v(sZ[t], zm);
      const dfl q = c * df_rcp(df_sqr(Rv.re) + df_sqr(Rv.im));
      ar = -(Rv.im * q);
      ai = -(Rv.re * q);
    } else {
      const dfl q = c * df_rcp(n2);
      ar = dr * q;
      ai = -(wi * q);
    }
    if (sB[t] == 0) {
      S0r = S0r + ar;
      S0i = S0i + ai;
      cs0 = cs0 + c;
      int idx = m - l;
      if (idx < 0) idx += M0;
      const float2 tv = Ttab[idx];
      t0 = t0 + dfl{tv.x, tv.y} * c;
    } else {
      S1r = S1r + ar;
      S1i = S1i + ai;
      cs1 = cs1 + c;
    }
  }
  float2* p = part + (size_t)blockIdx.y * VEL_FIELDS * M0;
  p[0 * M0 + m] = make_float2(S1r.hi, S1r.lo);
  p[1 * M0 + m] = make_float2(S1i.hi, S1i.lo);
  p[2 * M0 + m] = make_float2(cs1.hi, cs1.lo);
  p[3 * M0 + m] = make_float2(S0r.hi, S0r.lo);
  p[4 * M0 + m] = make_float2(S0i.hi, S0i.lo);
  p[5 * M0 + m] = make_float2(cs0.hi, cs0.lo);
  p[6 * M0 + m] = make_float2(t0.hi, t0.lo);
}

__global__ void k_velocity_finish(int M0, int nchunk, FlowParams F, const float2* __restrict__ part,
                                  const double2* __restrict__ z64, const double2* __restrict__ dz64,
                                  const double* __restrict__ gdiag64, const float2* __restrict__ cw,
                                  const float2* __restrict__ hw0, double* __restrict__ U) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M0) return;
  dfl acc[7];
  for (int f = 0; f < 7; ++f) acc[f] = {0.f, 0.f};
  for (int ch = 0; ch < nchunk; ++ch) {
    const float2* p = part + (size_t)ch * VEL_FIELDS * M0;
    for (int f = 0; f < 7; ++f) {
      const float2 v = p[f * M0 + m];
      acc[f] = acc[f] + dfl{v.x, v.y};
    }
  }
  const double S1r = df_to_double(acc[0]), S1i = df_to_double(acc[1]), cs1 = df_to_double(acc[2]);
  const double S0r = df_to_double(acc[3]), S0i = df_to_double(acc[4]), cs0 = df_to_double(acc[5]);
  const double t0 = df_to_double(acc[6]);
  // s = -(i/2) sum c - i S
  const double s1r = S1i, s1i = -S1r - 0.5 * cs1;
  const double s0r = S0i, s0i = -S0r - 0.5 * cs0;
  const double2 zp = dz64[m];
  const double Kterm = zp.x * s1i + zp.y * s1r;    // Im{zeta_0' s1}
  const double Gterm = zp.x * s0r - zp.y * s0i;    // Re{zeta_0' s0}
  const double cm = df_to_double(dfl{cw[m].x, cw[m].y});
  const double h = df_to_double(dfl{hw0[m].x, hw0[m].y});
  // eq. d:phi:mv
  double asum = 0.0;
  for (int j = 2; j < F.nb; ++j) asum += F.a[j - 2];
  double mv = -(F.V1 + 0.5 * asum) * zp.y;
  const double2 zm = z64[m];
  for (int j = 2; j < F.nb; ++j) {
    const double ux = zm.x - F.zc[j - 2].x, uy = zm.y - F.zc[j - 2].y;
    double s, c;
    sincos(ux, &s, &c);
    const double e = exp(-uy);
    const double qr = e * c - 1.0, qi = e * s;      // e^{iu} - 1
    const double n2 = qr * qr + qi * qi;
    const double hr = qi / n2, hi = 0.5 + qr / n2;  // 1/2 cot(u/2) = i/2 + i/q
    mv += F.a[j - 2] * (hr * zp.x - hi * zp.y);
  }
  const double total = mv + Kterm - Gterm + t0 - gdiag64[m] * cm - 0.5 * h;
  U[m] = total / hypot(zp.x, zp.y);
}

// s_alpha U = [eq. d:phi:mv] + sum_c V_mc omega_c'/M_c - 1/2 H omega_0'
// (rows m0 .. m1 - 1 of the surface: all of it unless the context is row-partitioned)
__global__ void k_velocity_finish_v(int m0, int m1, long long ld, int npanel, FlowParams F,
                                    const double* __restrict__ ypart,
                                    const double2* __restrict__ z64,
                                    const double2* __restrict__ dz64,
                                    const float2* __restrict__ hw0, double* __restrict__ U) {
  const int m = m0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= m1) return;
  double y = 0.0;
  for (int p = 0; p < npanel; ++p) y += ypart[(size_t)p * ld + m];
  const double h = df_to_double(dfl{hw0[m].x, hw0[m].y});
  const double2 zp = dz64[m];
  double asum = 0.0;
  for (int j = 2; j < F.nb; ++j) asum += F.a[j - 2];
  double mv = -(F.V1 + 0.5 * asum) * zp.y;
  const double2 zm = z64[m];
  for (int j = 2; j < F.nb; ++j) {
    const double ux = zm.x - F.zc[j - 2].x, uy = zm.y - F.zc[j - 2].y;
    double s, c;
    sincos(ux, &s, &c);
    const double e = exp(-uy);
    const double qr = e * c - 1.0, qi = e * s;      // e^{iu} - 1
    const double n2 = qr * qr + qi * qi;
    const double hr = qi / n2, hi = 0.5 + qr / n2;  // 1/2 cot(u/2) = i/2 + i/q
    mv += F.a[j - 2] * (hr * zp.x - hi * zp.y);
  }
  U[m] = (mv + y - 0.5 * h) / hypot(zp.x, zp.y);
}

__global__ void k_psi(Blocks B, const double* __restrict__ omega, double* __restrict__ psi) {
  __shared__ double red[32];
  const int k = blockIdx.x + 2;
  if (k >= B.nb) return;
  const int o = B.off[k], M = B.M[k];
  double s = 0.0;
  for (int l = threadIdx.x; l < M; l += blockDim.x) s += omega[o + l];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) psi[k - 2] = t / (double)M;
  }
}

bie_status vgemv_run(bie_ctx* c, const float* xh, const float* xl, const double* x64,
                     double** ypart_out, int* npanel_out);

// omega'/M_k as double-float hi/lo arrays (zero padded to ld) and H omega_0',
// by the FP64 four-step DFT: the inputs of the U-matrix product
bie_status velocity_weights(bie_ctx* c, int nvec, const double* omega, float* xh, float* xl,
                            float2* hw0) {
  const Blocks B = make_blocks(c);
  const int N = c->N, M0 = c->M[0];
  double2 *dY, *dX2;
  BIE_GET(c, double2, "mdft_Y", (size_t)nvec * (N + M0), dY);
  BIE_GET(c, double2, "mdft_X2", (size_t)nvec * (N + M0), dX2);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "velocity: twiddles");
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  int s1 = 0, s2 = 0;
  for (int k = 0; k < c->nb; ++k) {
    const int M = c->M[k], M1 = c->fft_m1[k], o = c->off[k];
    J1.j[J1.n++] = DftJob{M, M1, M / M1, o, o, o, 0, s1};
    s1 += M;
    J2.j[J2.n++] = DftJob{M, M1, M / M1, o, o, o, 1, s2};
    s2 += M;
  }
  J2.j[J2.n++] = DftJob{M0, c->fft_m1[0], M0 / c->fft_m1[0], 0, N, 0, 2, s2};
  s2 += M0;
  J1.total = s1;
  J2.total = s2;
  const long long sY = N + M0;
  k_dft_a<<<dft_grid(dim3((s1 + 255) / 256, nvec)), 256, 0, c->stream>>>(J1, omega, nullptr, tw, dY, N, sY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  // every vector's work arrays have stride N + M0; the spectra of the first
  // pair of passes go to X2, which the second pair reads and then overwrites
  k_dft_b<<<dft_grid(dim3((s1 + 255) / 256, nvec)), 256, 0, c->stream>>>(J1, dY, tw, dX2, sY);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid(dim3((s2 + 255) / 256, nvec)), 256, 0, c->stream>>>(J2, nullptr, dX2, tw, dY, sY, sY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(dim3((s2 + 255) / 256, nvec)), 256, 0, c->stream>>>(J2, dY, tw, dX2, sY);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  const long long next = c->ld + M0;
  k_dft_extract<<<dim3((unsigned)((next + 255) / 256), nvec), 256, 0, c->stream>>>(
      B, dX2, nullptr, hw0, xh, xl, nullptr, c->ld);
  BIE_LAUNCH_CHECK(c, "k_dft_extract");
  return BIE_OK;
}

// U from given derivative weights cw = omega'/M (all nodes) and hw0 = H omega_0'
// (surface), by the matrix-free kernels
bie_status velocity_from_weights(bie_ctx* c, const float2* cw, const float2* hw0, double* U) {
  const FlowParams F = make_flow(c);
  const int N = c->N, M0 = c->M[0];
  const int nchunk = (N + VEL_CH - 1) / VEL_CH;
  float2* part;
  BIE_GET(c, float2, "vel_part", (size_t)nchunk * VEL_FIELDS * M0, part);
  bool oom = false;
  const float2* Ttab = (const float2*)ctx_buf(c, "Ttab", sizeof(float2) * M0, &oom);
  const float4* nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  const float4* nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  const float4* nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  const double2* z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double* gdiag64 = (const double*)ctx_buf(c, "gdiag64", sizeof(double) * M0, &oom);
  const int* blk = (const int*)ctx_buf(c, "blk", sizeof(int) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "velocity: buffers");
  k_velocity_partial<<<dim3((M0 + 255) / 256, nchunk), 256, 0, c->stream>>>(
      N, M0, nP, nQ, nPQc, z64, blk, cw, Ttab, 0.01f, part);
  BIE_LAUNCH_CHECK(c, "k_velocity_partial");
  k_velocity_finish<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, nchunk, F, part, z64, dz64, gdiag64,
                                                             cw, hw0, U);
  BIE_LAUNCH_CHECK(c, "k_velocity_finish");
  return BIE_OK;
}

bie_status velocity_run(bie_ctx* c, const double* omega, double* U, double* psi) {
  BIE_NVTX("normal_velocity");
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  const int N = c->N, M0 = c->M[0];
  const int nchunk = (N + VEL_CH - 1) / VEL_CH;
  float2 *cw, *hw0, *part;
  double2 *dY, *dX1, *dX2;
  BIE_GET(c, float2, "vel_cw", N, cw);
  BIE_GET(c, float2, "vel_hw0", M0, hw0);
  BIE_GET(c, float2, "vel_part", (size_t)nchunk * VEL_FIELDS * M0, part);
  BIE_GET(c, double2, "dft_Y", N + M0, dY);
  BIE_GET(c, double2, "dft_X1", N, dX1);
  BIE_GET(c, double2, "dft_X2", N + M0, dX2);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  const float2* Ttab = (const float2*)ctx_buf(c, "Ttab", sizeof(float2) * M0, &oom);
  const float4* nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  const float4* nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  const float4* nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  const double2* z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double* gdiag64 = (const double*)ctx_buf(c, "gdiag64", sizeof(double) * M0, &oom);
  const int* blk = (const int*)ctx_buf(c, "blk", sizeof(int) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "velocity: buffers");
  const int pr = prof_begin(c, 3, -1);
  // forward DFT of every boundary's omega
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  int s1 = 0, s2 = 0;
  for (int k = 0; k < c->nb; ++k) {
    const int M = c->M[k], M1 = c->fft_m1[k], o = c->off[k];
    J1.j[J1.n++] = DftJob{M, M1, M / M1, o, o, o, 0, s1};
    s1 += M;
    J2.j[J2.n++] = DftJob{M, M1, M / M1, o, o, o, 1, s2};
    s2 += M;
  }
  J2.j[J2.n++] = DftJob{M0, c->fft_m1[0], M0 / c->fft_m1[0], 0, N, 0, 2, s2};
  s2 += M0;
  J1.total = s1;
  J2.total = s2;
  k_dft_a<<<dft_grid((s1 + 255) / 256), 256, 0, c->stream>>>(J1, omega, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid((s1 + 255) / 256), 256, 0, c->stream>>>(J1, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  // inverse of (i k X) per boundary and of (|k| X_0), as conj(DFT(conj(.)))
  k_dft_a<<<dft_grid((s2 + 255) / 256), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid((s2 + 255) / 256), 256, 0, c->stream>>>(J2, dY, tw, dX2);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  const bool useV = c->assembled;
  float *vxh = nullptr, *vxl = nullptr;
  double* vwp = nullptr;
  if (useV) {
    if (c->precision == BIE_FP64) {
      BIE_GET(c, double, "vel_wp64", c->ld, vwp);
    } else {
      BIE_GET(c, float, "vel_xh", c->ld, vxh);
      BIE_GET(c, float, "vel_xl", c->ld, vxl);
    }
  }
  const long long next = useV ? c->ld + M0 : (long long)N + M0;
  k_dft_extract<<<(unsigned)((next + 255) / 256), 256, 0, c->stream>>>(B, dX2, cw, hw0, vxh, vxl, vwp,
                                                                     c->ld);
  BIE_LAUNCH_CHECK(c, "k_dft_extract");
  if (useV) {
    double* ypart = nullptr;
    int npanel = 0;
    bie_status s = vgemv_run(c, vxh, vxl, vwp, &ypart, &npanel);
    if (s != BIE_OK) return s;
    const int nv = local_vrows(c);
    if (nv > 0) {
      k_velocity_finish_v<<<(nv + 255) / 256, 256, 0, c->stream>>>(c->row0, c->row0 + nv, c->ld, npanel,
                                                                 F, ypart, z64, dz64, hw0, U);
      BIE_LAUNCH_CHECK(c, "k_velocity_finish_v");
    }
    s = part_allgather(c, U, 8, M0);   // the other parts' surface rows
    if (s != BIE_OK) return s;
    prof_end(c, pr);
    if (psi && c->nb > 2) {
      k_psi<<<c->nb - 2, 256, 0, c->stream>>>(B, omega, psi);
      BIE_LAUNCH_CHECK(c, "k_psi");
    }
    return BIE_OK;
  }
  k_velocity_partial<<<dim3((M0 + 255) / 256, nchunk), 256, 0, c->stream>>>(
      N, M0, nP, nQ, nPQc, z64, blk, cw, Ttab, 0.01f, part);
  BIE_LAUNCH_CHECK(c, "k_velocity_partial");
  k_velocity_finish<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, nchunk, F, part, z64, dz64, gdiag64,
                                                             cw, hw0, U);
  prof_end(c, pr);
  BIE_LAUNCH_CHECK(c, "k_velocity_finish");
  if (psi && c->nb > 2) {
    k_psi<<<c->nb - 2, 256, 0, c->stream>>>(B, omega, psi);
    BIE_LAUNCH_CHECK(c, "k_psi");
  }
  return BIE_OK;
}

// ---------------------------------------------------------------------------
// Normal velocity without any device allocation.
//
// For callers that cannot allocate device memory themselves or let a library
// do it: code running under an allocator that forbids cudaMalloc after start-up
// (a pool that owns all of HBM, a real-time loop where an allocation may
// stall), or a host program embedding this library next to another runtime
// that owns the device heap.  bie_normal_velocity() needs a context, and
// contexts allocate their workspace on first use; this entry point instead
// works in one file-scope device array of fixed size, shared by all calls in
// the process, and allocates nothing.
//
// Limits: N = sum M_k <= BIE_STATIC_MAXN (include/bie.h).
// The scratch array keeps the last call's contents; every word a call reads is
// written earlier in the same call, so nothing needs clearing.  Calls that
// overlap on the GPU (two streams, or two host threads) share the array and
// race: serialise them.  The array's device address belongs to the CUDA
// context current at the call, so it is looked up again (cudaGetSymbolAddress)
// on every call whose stream is not being captured: a reset device or a
// caller-made driver context gets its own address.  A captured call uses the
// address of the last uncaptured call on that device, so make one call on the
// device before capturing.  The stream must belong to the current device.
// ---------------------------------------------------------------------------
#include <mutex>

#define BIE_STATIC_NCHUNK ((BIE_STATIC_MAXN + VEL_CH - 1) / VEL_CH)

__global__ void k_node_prep(Blocks B, const double2* __restrict__ z, const double2* __restrict__ dz,
                            const double2* __restrict__ d2z, int* __restrict__ blk,
                            float* __restrict__ wgt, double* __restrict__ wgt64,
                            float* __restrict__ sgn, float4* __restrict__ nP,
                            float4* __restrict__ nQ, float4* __restrict__ nPQc,
                            float4* __restrict__ nZp, float2* __restrict__ nDiag,
                            double2* __restrict__ P64, double2* __restrict__ Q64,
                            double* __restrict__ diag64, double* __restrict__ gdiag64, long long ld);
__global__ void k_spectral_tables(Blocks B, double2* __restrict__ tw, float2* __restrict__ Ttab,
                                  double* __restrict__ T64, float2* __restrict__ Tall);

// byte layout of the scratch array (each piece 256-byte aligned)
struct StaticLayout {
  size_t blk, wgt, wgt64, sgn, nP, nQ, nPQc, nZp, nDiag, P64, Q64, diag64, gdiag64, tw, Ttab, dY,
      dX1, dX2, cw, hw0, part, total;
};
static constexpr size_t sa(size_t x) { return (x + 255) / 256 * 256; }
static constexpr size_t kSN = BIE_STATIC_MAXN;
static constexpr size_t kSLD = (BIE_STATIC_MAXN + BIE_LD_ALIGN - 1) / BIE_LD_ALIGN * BIE_LD_ALIGN;
static constexpr size_t kStaticBytes =
    sa(4 * kSLD) + sa(4 * kSLD) + sa(8 * kSLD) + sa(4 * kSLD) + 4 * sa(16 * kSN) +
    sa(8 * kSN) + 2 * sa(16 * kSN) + sa(8 * kSN) + sa(8 * kSN) + sa(16 * kSN) + sa(8 * kSN) +
    sa(16 * 2 * kSN) + sa(16 * kSN) + sa(16 * 2 * kSN) + sa(8 * kSN) + sa(8 * kSN) +
    sa(8 * (size_t)BIE_STATIC_NCHUNK * VEL_FIELDS * kSN);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

static StaticLayout static_layout() {
  StaticLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += sa(bytes);
    return at;
  };
  L.blk = take(4 * kSLD);
  L.wgt = take(4 * kSLD);
  L.wgt64 = take(8 * kSLD);
  L.sgn = take(4 * kSLD);
  L.nP = take(16 * kSN);
  L.nQ = take(16 * kSN);
  L.nPQc = take(16 * kSN);
  L.nZp = take(16 * kSN);
  L.nDiag = take(8 * kSN);
  L.P64 = take(16 * kSN);
  L.Q64 = take(16 * kSN);
  L.diag64 = take(8 * kSN);
  L.gdiag64 = take(8 * kSN);
  L.tw = take(16 * kSN);
  L.Ttab = take(8 * kSN);
  L.dY = take(16 * 2 * kSN);
  L.dX1 = take(16 * kSN);
  L.dX2 = take(16 * 2 * kSN);
  L.cw = take(8 * kSN);
  L.hw0 = take(8 * kSN);
  L.part = take(8 * (size_t)BIE_STATIC_NCHUNK * VEL_FIELDS * kSN);
  L.total = o;
  return L;
}

static std::mutex g_static_mu;
static void* g_static_dev[256];   // address from the last uncaptured call, per device

extern "C" bie_status bie_normal_velocity_static(int nb, const int* M_host, const double* zeta_dev,
                                                 const double* dzeta_dev, const double* d2zeta_dev,
                                                 const double* zc_host, double V1,
                                                 const double* a_host, const double* omega_dev,
                                                 double* U_dev, double* psi_dev, void* cuda_stream) {
  if (nb < 2 || nb > BIE_MAXB || !M_host || !zeta_dev || !dzeta_dev || !d2zeta_dev ||
      !omega_dev || !U_dev || (nb > 2 && (!zc_host || !a_host)))
    return BIE_ERR_ARG;
  long long N = 0;
  for (int k = 0; k < nb; ++k) {
    if (M_host[k] < 8) return BIE_ERR_ARG;
    N += M_host[k];
  }
  if (N > BIE_STATIC_MAXN) return BIE_ERR_ARG;  // beyond the fixed scratch size
  const StaticLayout L = static_layout();
  if (L.total > kStaticBytes) return BIE_ERR_STATE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (st) {
    int sdev = -1;
    if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return BIE_ERR_ARG;
    }
    if (sdev != dev) return BIE_ERR_ARG;   // the stream belongs to another device
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return BIE_ERR_CUDA;
      }
      g_static_dev[dev] = p;
    } else if (!g_static_dev[dev]) {
      return BIE_ERR_STATE;   // captured before any uncaptured call on this device
    }
    base = (unsigned char*)g_static_dev[dev];
  }
  Blocks B;
  memset(&B, 0, sizeof(B));
  B.nb = nb;
  B.N = (int)N;
  B.off[0] = 0;
  for (int k = 0; k < BIE_MAXB; ++k) {
    B.M[k] = k < nb ? M_host[k] : 0;
    B.off[k + 1] = B.off[k] + B.M[k];
  }
  FlowParams F;
  memset(&F, 0, sizeof(F));
  F.nb = nb;
  F.V1 = V1;
  for (int j = 2; j < nb; ++j) {
    F.a[j - 2] = a_host[j - 2];
    F.zc[j - 2] = make_double2(zc_host[2 * (j - 2)], zc_host[2 * (j - 2) + 1]);
  }
  const int M0 = B.M[0];
  const long long ld = round_up(N, BIE_LD_ALIGN);
  const double2* z = (const double2*)zeta_dev;
  const double2* dz = (const double2*)dzeta_dev;
  int* blk = (int*)(base + L.blk);
  float4* nP = (float4*)(base + L.nP);
  float4* nQ = (float4*)(base + L.nQ);
  float4* nPQc = (float4*)(base + L.nPQc);
  double* gdiag64 = (double*)(base + L.gdiag64);
  double2* tw = (double2*)(base + L.tw);
  float2* Ttab = (float2*)(base + L.Ttab);
  double2* dY = (double2*)(base + L.dY);
  double2* dX1 = (double2*)(base + L.dX1);
  double2* dX2 = (double2*)(base + L.dX2);
  float2* cw = (float2*)(base + L.cw);
  float2* hw0 = (float2*)(base + L.hw0);
  float2* part = (float2*)(base + L.part);
  k_node_prep<<<(unsigned)((ld + 255) / 256), 256, 0, st>>>(
      B, z, dz, (const double2*)d2zeta_dev, blk, (float*)(base + L.wgt), (double*)(base + L.wgt64),
      (float*)(base + L.sgn), nP, nQ, nPQc, (float4*)(base + L.nZp), (float2*)(base + L.nDiag),
      (double2*)(base + L.P64), (double2*)(base + L.Q64), (double*)(base + L.diag64), gdiag64, ld);
  k_spectral_tables<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(B, tw, Ttab, nullptr, nullptr);
  int m1[BIE_MAXB];
  for (int k = 0; k < nb; ++k) {
    int best = 1;
    for (int d = 1; (long long)d * d <= B.M[k]; ++d)
      if (B.M[k] % d == 0) best = d;
    m1[k] = best;
  }
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  int s1 = 0, s2 = 0;
  for (int k = 0; k < nb; ++k) {
    const int M = B.M[k], o = B.off[k];
    J1.j[J1.n++] = DftJob{M, m1[k], M / m1[k], o, o, o, 0, s1};
    s1 += M;
    J2.j[J2.n++] = DftJob{M, m1[k], M / m1[k], o, o, o, 1, s2};
    s2 += M;
  }
  J2.j[J2.n++] = DftJob{M0, m1[0], M0 / m1[0], 0, (int)N, 0, 2, s2};
  s2 += M0;
  J1.total = s1;
  J2.total = s2;
  k_dft_a<<<dft_grid((s1 + 255) / 256), 256, 0, st>>>(J1, omega_dev, nullptr, tw, dY);
  k_dft_b<<<dft_grid((s1 + 255) / 256), 256, 0, st>>>(J1, dY, tw, dX1);
  k_dft_a<<<dft_grid((s2 + 255) / 256), 256, 0, st>>>(J2, nullptr, dX1, tw, dY);
  k_dft_b<<<dft_grid((s2 + 255) / 256), 256, 0, st>>>(J2, dY, tw, dX2);
  k_dft_extract<<<(unsigned)((N + M0 + 255) / 256), 256, 0, st>>>(B, dX2, cw, hw0, nullptr, nullptr,
                                                                  nullptr, ld);
  const int nchunk = (int)((N + VEL_CH - 1) / VEL_CH);
  k_velocity_partial<<<dim3((M0 + 255) / 256, nchunk), 256, 0, st>>>(
      (int)N, M0, nP, nQ, nPQc, z, blk, cw, Ttab, 0.01f, part);
  k_velocity_finish<<<(M0 + 255) / 256, 256, 0, st>>>(M0, nchunk, F, part, z, dz, gdiag64, cw, hw0,
                                                      U_dev);
  if (psi_dev && nb > 2) k_psi<<<nb - 2, 256, 0, st>>>(B, omega_dev, psi_dev);
  if (cudaGetLastError() != cudaSuccess) return BIE_ERR_CUDA;
  return BIE_OK;
}

// ---------------------------------------------------------------------------
// auxiliary Dirichlet data for Phi_t - C(t) (Sec. 4, eq. pressure:d:prob)
// ---------------------------------------------------------------------------
// b_0 = tau kappa - (phi_alpha^2 / s_alpha^2 + U^2)/2 - g eta on the surface,
// b_k = 0 elsewhere; phi_alpha = phi~_alpha + Re{Phi_mv'(zeta) zeta'} with
// Phi_mv' = V1 + sum_j a_j (1/2 - i/2 cot((z - z_j)/2)) (eq. d:phi:cyl).
__global__ void k_pressure_rhs(int N, int M0, FlowParams F, const double2* __restrict__ X2,
                               const double2* __restrict__ z64, const double2* __restrict__ dz64,
                               const double2* __restrict__ d2z64, const double* __restrict__ U,
                               double tau, double g, double* __restrict__ b) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  if (m >= M0) {
    b[m] = 0.0;
    return;
  }
  const double2 z = z64[m], zp = dz64[m], zpp = d2z64[m];
  double re = F.V1;   // Re Phi_mv'
  double im = 0.0;    // Im Phi_mv'
  for (int j = 2; j < F.nb; ++j) {
    const double ux = z.x - F.zc[j - 2].x, uy = z.y - F.zc[j - 2].y;
    double sn, cs;
    sincos(ux, &sn, &cs);
    const double e = exp(-uy);
    const double qr = e * cs - 1.0, qi = e * sn;      // e^{iu} - 1
    const double n2 = qr * qr + qi * qi;
    const double hr = qi / n2, hi = 0.5 + qr / n2;    // 1/2 cot(u/2) = hr + i hi
    re += F.a[j - 2] * (0.5 + hi);
    im -= F.a[j - 2] * hr;
  }
  const double phia = X2[m].x / (double)M0 + (re * zp.x - im * zp.y);
  const double s2 = zp.x * zp.x + zp.y * zp.y;
  const double s = sqrt(s2);
  const double kappa = (zpp.y * zp.x - zpp.x * zp.y) / (s2 * s);
  const double u = U[m];
  b[m] = tau * kappa - 0.5 * (phia * phia / s2 + u * u) - g * z.y;
}

extern "C" bie_status bie_pressure_rhs(bie_ctx* c, const double* phit, const double* U, double tau,
                                       double g, double* b) {
  BIE_NVTX("bie_pressure_rhs");
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom || !c->have_flow)
    return ctx_fail(c, BIE_ERR_STATE, "bie_pressure_rhs: set geometry and flow first");
  if (!phit || !U || !b) return ctx_fail(c, BIE_ERR_ARG, "bie_pressure_rhs: null pointer");
  if (!std::isfinite(tau) || !std::isfinite(g))
    return ctx_fail(c, BIE_ERR_ARG, "bie_pressure_rhs: tau and g must be finite");
  cudaSetDevice(c->device);
  const int N = c->N, M0 = c->M[0];
  double2 *dY, *dX1, *dX2;
  BIE_GET(c, double2, "prs_Y", M0, dY);
  BIE_GET(c, double2, "prs_X1", M0, dX1);
  BIE_GET(c, double2, "prs_X2", M0, dX2);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  const double2* z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double2* d2z64 = (const double2*)ctx_buf(c, "d2zeta", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_pressure_rhs: buffers");
  // phi~_alpha by the four-step DFT of the surface block (modes 0 then 1)
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  const int M1 = c->fft_m1[0];
  J1.j[J1.n++] = DftJob{M0, M1, M0 / M1, 0, 0, 0, 0, 0};
  J2.j[J2.n++] = DftJob{M0, M1, M0 / M1, 0, 0, 0, 1, 0};
  J1.total = J2.total = M0;
  const unsigned gb = (unsigned)((M0 + 255) / 256);
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J1, phit, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J1, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J2, dY, tw, dX2);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_pressure_rhs<<<(N + 255) / 256, 256, 0, c->stream>>>(N, M0, make_flow(c), dX2, z64, dz64, d2z64,
                                                         U, tau, g, b);
  BIE_LAUNCH_CHECK(c, "k_pressure_rhs");
  return BIE_OK;
}

// psi|_j = <1_j, omega> for the obstacles j >= 2 (eq. psi:k): psi[j - 2]
bie_status psi_run(bie_ctx* c, const double* omega, double* psi) {
  if (c->nb <= 2) return BIE_OK;
  const Blocks B = make_blocks(c);
  k_psi<<<c->nb - 2, 256, 0, c->stream>>>(B, omega, psi);
  BIE_LAUNCH_CHECK(c, "k_psi");
  return BIE_OK;
}
