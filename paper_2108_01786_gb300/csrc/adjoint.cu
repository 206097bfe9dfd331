// Backward pass: the gradient of a functional J(U) of the normal velocity with
// respect to the node data, the obstacle centres and phi~ (the adjoint of the
// solve of eq. lin:sys followed by the U formula of Sec. 3.4).
//
// Forward map.  A(g) omega = b(g, phi~) (Table 1, eq. Awb), then
//   s_alpha U = N,  N = [eq. d:phi:mv] + sum_c V_mc omega_c'/M_c - 1/2 H omega_0'
// with V the surface U-matrix stored by the assembly and omega' = D omega the
// spectral derivative of each boundary's density.
//
// Backward, given gU = dJ/dU:
//   Nbar = gU / s_alpha,
//   omegabar = -D (W V^T Nbar) - 1/2 |D| Nbar   (D^T = -D, H^T = -H, D H = |D|),
//   A^T lambda = omegabar                        (the adjoint system),
//   dJ = lambda . (db - dA omega) + Nbar . dN|_omega + sbar . d s_alpha.
// With A = S W + Sigma (S the stored values, W = diag(1/M_j), Sigma = +-1/2),
// A^T = W (S^T W + Sigma) W^{-1}: the solver's operator on the transposed
// storage, applied to mu = lambda / w with right-hand side omegabar / w.
//
// The geometry terms are contracted pair by pair without forming dA: every
// entry is a component of a holomorphic h = zeta_l' G(zeta_l - zeta_m),
// G(x) = 1/2 cot(x/2), G'(x) = -(G^2 + 1/4).  For a real coefficient c times
// Im h (Re h) the cotangent of an input u is c i conj(dh/du) (c conj(dh/du)),
// in the convention g = dJ/dRe u + i dJ/dIm u.  For an unordered node pair the
// A terms of (m,l) and (l,m) and the V terms of surface rows share one G, and
// the cotangents of zeta_m and zeta_l are opposite:
//   a_l = kappa_A(m,l) - kappa_V(l,m),   a_m = kappa_V(m,l) - kappa_A(l,m),
//   gzeta'_l += conj(G) a_l,  gzeta'_m += conj(G) a_m,
//   tau = conj(G') (a_l conj(zeta_l') + a_m conj(zeta_m')),  gzeta_l += tau, gzeta_m -= tau,
// where kappa carries the coefficient (-lambda_m omega_l/M_l for A_ml,
// Nbar_m omega_l'/M_l for V_ml) times the component's phase (i for Im, 1 for
// Re, -1 for -Re, -i for -Im).
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "nvtx.cuh"
#include "dft.cuh"
#include "pair_kernel.cuh"

#define ADJ_TILE 32
#define VT_ROWS 32

// ---------------------------------------------------------------------------
// Nbar, the transposed U-matrix product and the adjoint right-hand side
// ---------------------------------------------------------------------------
__global__ void k_adj_nbar(int M0, const double* __restrict__ gU, const double2* __restrict__ dz,
                           double* __restrict__ nbar) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M0) return;
  const double2 zp = dz[m];
  nbar[m] = gU[m] / hypot(zp.x, zp.y);
}

// part[ch][c] = sum over surface rows r of chunk ch of V[r][c] Nbar_r
template <int F64>
// (stored surface rows q0 .. q1 - 1, row r at (r - q0) ld: all M_0 rows unless
// the context is row-partitioned)
__global__ void k_adj_vt(int N, int q0, int q1, long long ld, const double* __restrict__ Vf64,
                         const float* __restrict__ Vhi, const float* __restrict__ Vlo,
                         const double* __restrict__ nbar, double* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int r0 = q0 + blockIdx.y * VT_ROWS;
  const int r1 = min(r0 + VT_ROWS, q1);
  double s = 0.0;
  for (int r = r0; r < r1; ++r) {
    const size_t idx = (size_t)(r - q0) * ld + c;
    const double v = F64 ? Vf64[idx] : (double)Vhi[idx] + (double)Vlo[idx];
    s = fma(v, nbar[r], s);
  }
  part[(size_t)blockIdx.y * ld + c] = s;
}

// sum of the nch row-chunk partials of V^T Nbar into the first row (a
// partitioned context then adds the parts' sums)
__global__ void k_adj_vt_sum(int N, long long ld, int nch, double* __restrict__ part) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += part[(size_t)ch * ld + c];
  part[c] = s;
}

// DFT inputs: [0, N) (W V^T Nbar), [N, N + M0) Nbar, [N + M0, 2N + M0) omega
__global__ void k_adj_dft_in(int N, int M0, long long ld, int nch, const double* __restrict__ part,
                             const double* __restrict__ wgt64, const double* __restrict__ nbar,
                             const double* __restrict__ omega, double* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * N + M0) return;
  if (t < N) {
    double s = 0.0;
    for (int ch = 0; ch < nch; ++ch) s += part[(size_t)ch * ld + t];
    x[t] = s * wgt64[t];
  } else if (t < N + M0) {
    x[t] = nbar[t - N];
  } else {
    x[t] = omega[t - N - M0];
  }
}

// omegabar = -D(W V^T Nbar) - 1/2 |D| Nbar (surface); the solver's right-hand
// side is omegabar / w = M_k omegabar.  Also omega' (FP64) for the pair terms.
__global__ void k_adj_rhs(Blocks B, const double2* __restrict__ X2, const double* __restrict__ omega,
                          const double* __restrict__ nbar, double* __restrict__ rhs,
                          double4_16a* __restrict__ coef) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= B.N) return;
  int k = 0;
  while (k + 1 < B.nb && n >= B.off[k + 1]) ++k;
  const double M = (double)B.M[k];
  const int M0 = B.M[0];
  double wb = -X2[n].x / M;
  if (n < M0) wb -= 0.5 * X2[B.N + n].x / (double)M0;
  rhs[n] = M * wb;
  const double wp = X2[B.N + M0 + n].x / M;
  coef[n] = make_double4_16a(0.0, omega[n] / M, wp / M, n < M0 ? nbar[n] : 0.0);
}

// lambda = w mu; the coefficients (lambda, omega w, omega' w, Nbar) also as
// double-float pairs for the df pair kernel; dJ/dphi~ = lambda on the surface.
__global__ void k_adj_lambda(int N, int M0, const double* __restrict__ mu,
                             const double* __restrict__ wgt64, double4_16a* __restrict__ coef,
                             float4* __restrict__ coefdf, double* __restrict__ lam_out,
                             double* __restrict__ gphit) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double lam = mu[n] * wgt64[n];
  double4_16a c = coef[n];
  c.x = lam;
  coef[n] = c;
  const dfl u = df_from_double(c.x), v = df_from_double(c.y);
  const dfl p = df_from_double(c.z), q = df_from_double(c.w);
  coefdf[2 * n] = make_float4(u.hi, u.lo, v.hi, v.lo);
  coefdf[2 * n + 1] = make_float4(p.hi, p.lo, q.hi, q.lo);
  if (lam_out) lam_out[n] = lam;
  if (gphit && n < M0) gphit[n] = lam;
}

// ---------------------------------------------------------------------------
// pair contraction
// ---------------------------------------------------------------------------
struct AdjArgs {
  int N;
  int ntile;
  const int* blk;
  const double2* z64;
  const float4* nP;
  const float4* nQ;
  const float4* nZp;
  const float4* nPQc;
  const double2* P64;
  const double2* Q64;
  const double2* Zp64;
  const double4_16a* coef;
  const float4* coefdf;
  double* part;     // [4][ntile][N]: gzeta.re, gzeta.im, gzeta'.re, gzeta'.im
  float near2;
};

template <class R> struct AdjCoef {
  R u, v, p, q;   // lambda, omega w, omega' w, Nbar
};

template <class R> struct AdjLoad;
template <> struct AdjLoad<dfl> {
  static __device__ __forceinline__ cx<dfl> P(const AdjArgs& a, int l) {
    const float4 v = a.nP[l];
    return {{v.x, v.y}, {v.z, v.w}};
  }
  static __device__ __forceinline__ cx<dfl> Q(const AdjArgs& a, int l) {
    const float4 v = a.nQ[l];
    return {{v.x, v.y}, {v.z, v.w}};
  }
  static __device__ __forceinline__ cx<dfl> Zp(const AdjArgs& a, int l) {
    const float4 v = a.nZp[l];
    return {{v.x, v.y}, {v.z, v.w}};
  }
  static __device__ __forceinline__ AdjCoef<dfl> C(const AdjArgs& a, int l) {
    const float4 x = a.coefdf[2 * l], y = a.coefdf[2 * l + 1];
    return {{x.x, x.y}, {x.z, x.w}, {y.x, y.y}, {y.z, y.w}};
  }
};
template <> struct AdjLoad<double> {
  static __device__ __forceinline__ cx<double> P(const AdjArgs& a, int l) {
    const double2 v = a.P64[l];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ cx<double> Q(const AdjArgs& a, int l) {
    const double2 v = a.Q64[l];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ cx<double> Zp(const AdjArgs& a, int l) {
    const double2 v = a.Zp64[l];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ AdjCoef<double> C(const AdjArgs& a, int l) {
    const double4_16a c = a.coef[l];
    return {c.x, c.y, c.z, c.w};
  }
};

template <class R>
__device__ __forceinline__ cx<R> c_add(cx<R> a, cx<R> b) {
  return {r_add(a.re, b.re), r_add(a.im, b.im)};
}
template <class R>
__device__ __forceinline__ cx<R> c_conj(cx<R> a) {
  return {a.re, r_neg(a.im)};
}
template <class R>
__device__ __forceinline__ R r_zero();
template <> __device__ __forceinline__ double r_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ dfl r_zero<dfl>() { return {0.f, 0.f}; }

__device__ __forceinline__ void adj_tile_of(int t, int T, int& I, int& J) {
  // upper-triangular tiles (I <= J), row-major: row I holds T - I tiles
  int i = (int)floorf((2.0f * T + 1.0f - sqrtf((2.0f * T + 1.0f) * (2.0f * T + 1.0f) - 8.0f * t)) * 0.5f);
  if (i < 0) i = 0;
  while (i > 0 && i * T - i * (i - 1) / 2 > t) --i;
  while ((i + 1) * T - (i + 1) * i / 2 <= t) ++i;
  I = i;
  J = i + (t - (i * T - i * (i - 1) / 2));
}

// One CTA per tile pair {(I,J),(J,I)}, I <= J, 32 x 32 nodes; thread (tx, ty)
// owns column l = l0 + tx and rows ty, ty+8, ty+16, ty+24 of tile I.  Each
// node's cotangent receives one partial per other tile index, written once:
// as a column node of pair (I, J) into slot I, as a row node into slot J (on
// the diagonal tile both into slot I), so the reduction is deterministic.
template <class R>
__global__ void __launch_bounds__(256) k_adj_pairs(AdjArgs a) {
  __shared__ cx<R> sQ[ADJ_TILE];
  __shared__ cx<R> sZr[ADJ_TILE];
  __shared__ float2 sQc[ADJ_TILE];
  __shared__ double2 sZm[ADJ_TILE];
  __shared__ AdjCoef<R> sC[ADJ_TILE];
  __shared__ int sB[ADJ_TILE];
  // partials stay in R until the final write: on this GPU FP64 runs at 1/62
  // of the FP32 rate, so per-row conversions would bind the kernel
  __shared__ R sCol[8][4][ADJ_TILE];
  __shared__ R sRow[4][ADJ_TILE];
  int I, J;
  adj_tile_of(blockIdx.x, a.ntile, I, J);
  const int m0 = I * ADJ_TILE, l0 = J * ADJ_TILE;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x < ADJ_TILE) {
    const int m = m0 + threadIdx.x;
    if (m < a.N) {
      sQ[threadIdx.x] = AdjLoad<R>::Q(a, m);
      sZr[threadIdx.x] = AdjLoad<R>::Zp(a, m);
      const float4 pq = a.nPQc[m];
      sQc[threadIdx.x] = make_float2(pq.z, pq.w);
      sZm[threadIdx.x] = a.z64[m];
      sC[threadIdx.x] = AdjLoad<R>::C(a, m);
      sB[threadIdx.x] = a.blk[m];
    }
  }
  __syncthreads();
  const int l = l0 + tx;
  const bool lok = l < a.N;
  cx<R> P, Zl;
  AdjCoef<R> cl;
  float2 Pc = make_float2(0.f, 0.f);
  double2 zl = make_double2(0.0, 0.0);
  int bl = -1;
  if (lok) {
    P = AdjLoad<R>::P(a, l);
    Zl = AdjLoad<R>::Zp(a, l);
    cl = AdjLoad<R>::C(a, l);
    const float4 pq = a.nPQc[l];
    Pc = make_float2(pq.x, pq.y);
    zl = a.z64[l];
    bl = a.blk[l];
  }
  const bool diagTile = (I == J);
  const R zero = r_zero<R>();
  cx<R> gzl = {zero, zero}, gpl = {zero, zero};
#pragma unroll 1
  for (int k = 0; k < ADJ_TILE / 8; ++k) {
    const int rm = ty + 8 * k;
    const int m = m0 + rm;
    cx<R> gzm = {zero, zero}, gpm = {zero, zero};
    if (lok && m < a.N && !(diagTile && rm >= tx)) {
      const cx<R> G = half_cot_pair<R>(P, sQ[rm], Pc, sQc[rm], zl, sZm[rm], a.near2);
      // G' = -(G^2 + 1/4)
      const cx<R> Gp = {r_neg(r_addf(r_sub(r_sqr(G.re), r_sqr(G.im)), 0.25f)),
                        r_neg(r_mul(r_add(G.re, G.re), G.im))};
      const AdjCoef<R> cm = sC[rm];
      const R A1 = r_mul(cm.u, cl.v);   // lambda_m omega_l w_l   (entry (m, l))
      const R A2 = r_mul(cl.u, cm.v);   // lambda_l omega_m w_m   (entry (l, m))
      const R B1 = r_mul(cm.q, cl.p);   // Nbar_m omega_l' w_l    (V_ml, m on the surface)
      const R B2 = r_mul(cl.q, cm.p);   // Nbar_l omega_m' w_m    (V_lm, l on the surface)
      const bool sm = (sB[rm] == 0), sl = (bl == 0);
      cx<R> al, am;
      if (sm == sl) {          // Im on both entries; V entries Re (both on the surface)
        al = {r_neg(B2), r_neg(A1)};
        am = {B1, A2};
      } else if (sm) {         // (m,l): Re, (l,m): -Re; V_ml: -Im
        al = {r_neg(A1), zero};
        am = {r_neg(A2), r_neg(B1)};
      } else {                 // (m,l): -Re, (l,m): Re; V_lm: -Im
        al = {A1, B2};
        am = {A2, zero};
      }
      const cx<R> Gc = c_conj(G);
      gpl = c_add(gpl, c_mul(Gc, al));
      gpm = c_mul(Gc, am);
      const cx<R> s = c_add(c_mul(al, c_conj(Zl)), c_mul(am, c_conj(sZr[rm])));
      const cx<R> tau = c_mul(c_conj(Gp), s);
      gzl = c_add(gzl, tau);
      gzm = {r_neg(tau.re), r_neg(tau.im)};
    }
    // row m: sum over the warp's 32 columns
    gzm.re = warp_sum(gzm.re);
    gzm.im = warp_sum(gzm.im);
    gpm.re = warp_sum(gpm.re);
    gpm.im = warp_sum(gpm.im);
    if (tx == 0) {
      sRow[0][rm] = gzm.re;
      sRow[1][rm] = gzm.im;
      sRow[2][rm] = gpm.re;
      sRow[3][rm] = gpm.im;
    }
  }
  sCol[ty][0][tx] = gzl.re;
  sCol[ty][1][tx] = gzl.im;
  sCol[ty][2][tx] = gpl.re;
  sCol[ty][3][tx] = gpl.im;
  __syncthreads();
  if (threadIdx.x < 4 * ADJ_TILE) {
    const int f = threadIdx.x >> 5, i = threadIdx.x & 31;
    R cs = sCol[0][f][i];
#pragma unroll
    for (int t = 1; t < 8; ++t) cs = r_add(cs, sCol[t][f][i]);
    const size_t base = (size_t)f * a.ntile;
    if (diagTile) {
      const int n = m0 + i;
      if (n < a.N) a.part[(base + I) * a.N + n] = r_to_double(r_add(cs, sRow[f][i]));
    } else {
      const int nl = l0 + i, nm = m0 + i;
      if (nl < a.N) a.part[(base + I) * a.N + nl] = r_to_double(cs);
      if (nm < a.N) a.part[(base + J) * a.N + nm] = r_to_double(sRow[f][i]);
    }
  }
}

// ---------------------------------------------------------------------------
// per-node terms: diagonal limits, eq. d:phi:mv, s_alpha, the right-hand side
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

// 1/2 cot(u/2) = i/2 + i/(e^{iu} - 1)
__device__ __forceinline__ double2 half_cot64(double ux, double uy) {
  double s, c;
  sincos(ux, &s, &c);
  const double e = exp(-uy);
  const double qr = e * c - 1.0, qi = e * s;
  const double n2 = qr * qr + qi * qi;
  return make_double2(qi / n2, 0.5 + qr / n2);
}

__global__ void k_adj_node(Blocks B, FlowParams F, const double2* __restrict__ z64,
                           const double2* __restrict__ dz64, const double2* __restrict__ d2z64,
                           const double4_16a* __restrict__ coef, const double* __restrict__ gU,
                           const double* __restrict__ U, double2* __restrict__ gnode,
                           double2* __restrict__ gzc_part) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = B.N, M0 = B.M[0];
  if (n >= N) return;
  const double4_16a c = coef[n];   // lambda, omega w, omega' w, Nbar
  const double2 zn = z64[n], zp = dz64[n], zpp = d2z64[n];
  // diagonal entries: A_nn = w Im h, V_nn = -Re h, h = zeta''/(2 zeta');
  // dh/dzeta'' = 1/(2 zeta'), dh/dzeta' = -zeta''/(2 zeta'^2)
  const double den = zp.x * zp.x + zp.y * zp.y;
  const double2 inv = make_double2(zp.x / den, -zp.y / den);
  const double2 h1 = cscale(0.5, inv);
  const double2 h2 = cscale(-0.5, cmul(zpp, cmul(inv, inv)));
  const double2 kap = make_double2(-c.w * c.z, -c.x * c.y);
  double2 gzpp = cmul(kap, cconj(h1));
  double2 gzp = cmul(kap, cconj(h2));
  double2 gz = make_double2(0.0, 0.0);
  const int nobs = F.nb - 2;
  if (n < M0) {
    // s_alpha = |zeta'|: sbar = -gU U / s_alpha, d s_alpha / d zeta' -> zeta'/|zeta'|
    const double s = sqrt(den);
    const double sbar = -gU[n] * U[n] / s;
    gzp = cadd(gzp, cscale(sbar / s, zp));
    // eq. d:phi:mv: -(V1 + 1/2 sum a) Im zeta' + sum_j a_j Re{G(zeta - z_j) zeta'}
    const double nb = c.w;
    double asum = 0.0;
    for (int j = 0; j < nobs; ++j) asum += F.a[j];
    gzp.y += -nb * (F.V1 + 0.5 * asum);
    for (int j = 0; j < nobs; ++j) {
      const double2 G = half_cot64(zn.x - F.zc[j].x, zn.y - F.zc[j].y);
      const double2 Gp = make_double2(-(G.x * G.x - G.y * G.y + 0.25), -2.0 * G.x * G.y);
      const double w = nb * F.a[j];
      gzp = cadd(gzp, cscale(w, cconj(G)));
      const double2 t = cscale(w, cconj(cmul(Gp, zp)));
      gz = cadd(gz, t);
      gzc_part[(size_t)j * N + n] = make_double2(-t.x, -t.y);
    }
  } else {
    // b_n = -psi_mv(zeta_n), psi_mv = Im Phi_mv, Phi_mv' = V1 + sum_j a_j (1/2 - i G(z - z_j))
    const double lam = c.x;
    double2 dphi = make_double2(F.V1, 0.0);
    for (int j = 0; j < nobs; ++j) {
      const double2 G = half_cot64(zn.x - F.zc[j].x, zn.y - F.zc[j].y);
      const double2 dc = make_double2(F.a[j] * (0.5 + G.y), -F.a[j] * G.x);   // a_j (1/2 - i G)
      dphi = cadd(dphi, dc);
      // cotangent of z_j: +lambda i conj(a_j Phi_cyl')
      const double2 cj = cconj(dc);
      gzc_part[(size_t)j * N + n] = make_double2(-lam * cj.y, lam * cj.x);
    }
    const double2 cd = cconj(dphi);
    gz = cadd(gz, make_double2(lam * cd.y, -lam * cd.x));   // -lambda i conj(Phi_mv')
  }
  gnode[n] = gz;
  gnode[N + n] = gzp;
  gnode[2 * (size_t)N + n] = gzpp;
}

__global__ void k_adj_reduce(int N, int ntile, const double* __restrict__ part,
                             const double2* __restrict__ gnode, double2* __restrict__ gz,
                             double2* __restrict__ gzp, double2* __restrict__ gzpp) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int f = 0; f < 4; ++f) {
    const double* p = part + (size_t)f * ntile * N + n;
    double acc = 0.0;
    for (int t = 0; t < ntile; ++t) acc += p[(size_t)t * N];
    s[f] = acc;
  }
  const double2 a = gnode[n], b = gnode[N + n];
  gz[n] = make_double2(a.x + s[0], a.y + s[1]);
  gzp[n] = make_double2(b.x + s[2], b.y + s[3]);
  gzpp[n] = gnode[2 * (size_t)N + n];
}

__device__ __forceinline__ double block_sum256(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = threadIdx.x < 8 ? red[threadIdx.x] : 0.0;
  if (threadIdx.x < 32) t = warp_sum(t);
  return t;   // valid in thread 0
}

// one CTA (256 threads) per obstacle: g_zc[j] = sum_n gzc_part[j][n]
__global__ void __launch_bounds__(256) k_adj_zc(int N, const double2* __restrict__ part,
                                                double2* __restrict__ gzc) {
  __shared__ double red[8];
  const int j = blockIdx.x;
  double sx = 0.0, sy = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const double2 v = part[(size_t)j * N + n];
    sx += v.x;
    sy += v.y;
  }
  sx = block_sum256(sx, red);
  sy = block_sum256(sy, red);
  if (threadIdx.x == 0) gzc[j] = make_double2(sx, sy);
}

// ---------------------------------------------------------------------------
// chains: spectral derivatives of the nodes, ellipse parameters
// ---------------------------------------------------------------------------
// t = a - D x  (D x = conj(X2)/M per boundary, X2 = DFT(conj(i k DFT(x))))
__global__ void k_adj_axpy_d(Blocks B, const double2* __restrict__ a, const double2* __restrict__ X2,
                             double2* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= B.N) return;
  int k = 0;
  while (k + 1 < B.nb && n >= B.off[k + 1]) ++k;
  const double M = (double)B.M[k];
  const double2 x = X2[n];
  out[n] = make_double2(a[n].x - x.x / M, a[n].y + x.y / M);
}

struct EllParams {
  double p[BIE_MAXB][5];   // x, y, q, b, theta of obstacle j (block j + 2)
};

// zeta = z_j + e^{i theta}(q cos t - i b sin t): dJ/dp = sum_n <g, dzeta/dp> +
// <g', dzeta'/dp> + <g'', dzeta''/dp>, <a, b> = Re(conj(a) b); the centre also
// enters Phi_mv (g_zc).
__global__ void __launch_bounds__(256) k_adj_shape(Blocks B, EllParams E,
                                                   const double2* __restrict__ gz,
                                                   const double2* __restrict__ gzp,
                                                   const double2* __restrict__ gzpp,
                                                   const double2* __restrict__ gzc,
                                                   double* __restrict__ gshape) {
  __shared__ double red[8];
  const int j = blockIdx.x, k = j + 2;
  const int o = B.off[k], M = B.M[k];
  const double q = E.p[j][2], b = E.p[j][3], th = E.p[j][4];
  double rs, rc;
  sincos(th, &rs, &rc);
  const double2 r = make_double2(rc, rs);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double sa, ca;
    sincospi(2.0 * (double)i / (double)M, &sa, &ca);
    const double2 g = gz[o + i], gp = gzp[o + i], gpp = gzpp[o + i];
    auto dot = [](double2 u, double2 v) { return u.x * v.x + u.y * v.y; };
    const double2 z_q = cscale(ca, r), zp_q = cscale(-sa, r), zpp_q = cscale(-ca, r);
    const double2 z_b = cmul(r, make_double2(0.0, -sa)), zp_b = cmul(r, make_double2(0.0, -ca));
    const double2 zpp_b = cmul(r, make_double2(0.0, sa));
    const double2 rz = cmul(r, make_double2(q * ca, -b * sa));
    const double2 rzp = cmul(r, make_double2(-q * sa, -b * ca));
    const double2 rzpp = cmul(r, make_double2(-q * ca, b * sa));
    const double2 z_t = make_double2(-rz.y, rz.x), zp_t = make_double2(-rzp.y, rzp.x);
    const double2 zpp_t = make_double2(-rzpp.y, rzpp.x);
    acc[0] += g.x;
    acc[1] += g.y;
    acc[2] += dot(g, z_q) + dot(gp, zp_q) + dot(gpp, zpp_q);
    acc[3] += dot(g, z_b) + dot(gp, zp_b) + dot(gpp, zpp_b);
    acc[4] += dot(g, z_t) + dot(gp, zp_t) + dot(gpp, zpp_t);
  }
  for (int f = 0; f < 5; ++f) {
    const double s = block_sum256(acc[f], red);
    if (threadIdx.x == 0) {
      double v = s;
      if (f == 0) v += gzc[j].x;
      if (f == 1) v += gzc[j].y;
      gshape[5 * j + f] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static bie_status dft_pass(bie_ctx* c, const DftJobs& J, const double* xr, const double2* xc,
                           const double2* tw, double2* Y, double2* X) {
  const unsigned g = (unsigned)((J.total + 255) / 256);
  k_dft_a<<<dft_grid(g), 256, 0, c->stream>>>(J, xr, xc, tw, Y);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(g), 256, 0, c->stream>>>(J, Y, tw, X);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  return BIE_OK;
}

// D applied to a complex vector on every boundary: X2 = DFT(conj(i k DFT(x)))
static bie_status spectral_d(bie_ctx* c, const double2* x, const double2* tw, double2* Y,
                             double2* X1, double2* X2) {
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  int s = 0;
  for (int k = 0; k < c->nb; ++k) {
    const int M = c->M[k], M1 = c->fft_m1[k], o = c->off[k];
    J1.j[J1.n++] = DftJob{M, M1, M / M1, o, o, o, 3, s};
    J2.j[J2.n++] = DftJob{M, M1, M / M1, o, o, o, 1, s};
    s += M;
  }
  J1.total = J2.total = s;
  bie_status st = dft_pass(c, J1, nullptr, x, tw, Y, X1);
  if (st != BIE_OK) return st;
  return dft_pass(c, J2, nullptr, X1, tw, Y, X2);
}

extern "C" bie_status bie_backward(bie_ctx* c, const double* omega, const double* gU,
                                   const double* ellipses_host, const bie_grads* g,
                                   const bie_solve_opts* opts, bie_solve_info* info) {
  BIE_NVTX("bie_backward");
  if (!c) return BIE_ERR_ARG;
  if (!c->assembled || !c->have_flow || c->variant != 0)
    return ctx_fail(c, BIE_ERR_STATE, "bie_backward: assemble (eq. AB:cor), set_flow and solve first");
  if (!omega || !gU || !g) return ctx_fail(c, BIE_ERR_ARG, "bie_backward: null pointer");
  const int nobs = c->nb - 2;
  if (g->g_shape && nobs > 0 && !ellipses_host)
    return ctx_fail(c, BIE_ERR_ARG, "bie_backward: g_shape needs the ellipse parameters");
  bie_solve_opts o;
  bie_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > 1000 || o.max_cycles < 1)
    return ctx_fail(c, BIE_ERR_ARG, "bie_backward: bad options");
  o.x0 = 0;   // the adjoint solution has no caller-side guess
  EllParams E;
  memset(&E, 0, sizeof(E));
  if (g->g_shape && nobs > 0) {
    for (int j = 0; j < nobs; ++j) {
      for (int f = 0; f < 5; ++f) {
        const double v = ellipses_host[5 * j + f];
        if (!std::isfinite(v)) return ctx_fail(c, BIE_ERR_ARG, "bie_backward: ellipse parameter not finite");
        E.p[j][f] = v;
      }
    }
  }
  cudaSetDevice(c->device);
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  const int N = c->N, M0 = c->M[0];
  const long long ld = c->ld;
  const int nch = (M0 + VT_ROWS - 1) / VT_ROWS;
  const int ntile = (N + ADJ_TILE - 1) / ADJ_TILE;
  const int nX = 2 * N + M0;
  double *U, *nbar, *vtpart, *xin, *rhs, *mu, *part, *gphit_buf;
  double2 *dY, *dX1, *dX2, *gnode, *gzcp, *gz, *gzp, *gzpp, *gzc, *tmp;
  double4_16a* coef;
  float4* coefdf;
  BIE_GET(c, double, "adj_U", M0, U);
  BIE_GET(c, double, "adj_nbar", M0, nbar);
  BIE_GET(c, double, "adj_vtpart", (size_t)nch * ld, vtpart);
  BIE_GET(c, double, "adj_xin", nX, xin);
  BIE_GET(c, double2, "adj_Y", nX, dY);
  BIE_GET(c, double2, "adj_X1", nX, dX1);
  BIE_GET(c, double2, "adj_X2", nX, dX2);
  BIE_GET(c, double, "adj_rhs", ld, rhs);
  BIE_GET(c, double, "adj_mu", ld, mu);
  BIE_GET(c, double4_16a, "adj_coef", N, coef);
  BIE_GET(c, float4, "adj_coefdf", 2 * (size_t)N, coefdf);
  BIE_GET(c, double, "adj_part", 4 * (size_t)ntile * N, part);
  BIE_GET(c, double2, "adj_gnode", 3 * (size_t)N, gnode);
  BIE_GET(c, double2, "adj_gzcp", (size_t)(nobs > 0 ? nobs : 1) * N, gzcp);
  BIE_GET(c, double2, "adj_gz", N, gz);
  BIE_GET(c, double2, "adj_gzp", N, gzp);
  BIE_GET(c, double2, "adj_gzpp", N, gzpp);
  BIE_GET(c, double2, "adj_gzc", nobs > 0 ? nobs : 1, gzc);
  BIE_GET(c, double2, "adj_tmp", N, tmp);
  BIE_GET(c, double, "adj_gphit", M0, gphit_buf);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  const double2* z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double2* d2z64 = (const double2*)ctx_buf(c, "d2zeta", sizeof(double2) * N, &oom);
  const double* wgt64 = (const double*)ctx_buf(c, "wgt64", sizeof(double) * ld, &oom);
  const int* blk = (const int*)ctx_buf(c, "blk", sizeof(int) * ld, &oom);
  AdjArgs a;
  memset(&a, 0, sizeof(a));
  a.N = N;
  a.ntile = ntile;
  a.blk = blk;
  a.z64 = z64;
  a.nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  a.nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  a.nZp = (const float4*)ctx_buf(c, "nZp", sizeof(float4) * N, &oom);
  a.nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  a.P64 = (const double2*)ctx_buf(c, "P64", sizeof(double2) * N, &oom);
  a.Q64 = (const double2*)ctx_buf(c, "Q64", sizeof(double2) * N, &oom);
  a.Zp64 = dz64;
  a.coef = coef;
  a.coefdf = coefdf;
  a.part = part;
  a.near2 = 0.01f;
  const size_t VN = (size_t)local_vrows(c) * ld;   // the surface rows stored here
  const bool f64 = c->precision == BIE_FP64;
  const double* Vf64 = nullptr;
  const float *Vhi = nullptr, *Vlo = nullptr;
  if (f64) Vf64 = (const double*)ctx_buf(c, "V_f64", sizeof(double) * VN, &oom);
  else {
    Vhi = (const float*)ctx_buf(c, "V_hi", sizeof(float) * VN, &oom);
    Vlo = (const float*)ctx_buf(c, "V_lo", sizeof(float) * VN, &oom);
  }
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_backward: buffers");

  // 1. U of the forward solution and Nbar
  bie_status s = velocity_run(c, omega, U, nullptr);
  if (s != BIE_OK) return s;
  k_adj_nbar<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, gU, dz64, nbar);
  BIE_LAUNCH_CHECK(c, "k_adj_nbar");
  // 2. W V^T Nbar, then omegabar by the DFT: jobs for (W V^T Nbar) per boundary,
  //    Nbar (|k| symbol) and omega (for omega')
  const int nv = local_vrows(c);
  const int nchl = (nv + VT_ROWS - 1) / VT_ROWS;   // chunks of the stored surface rows
  int nsum = nch;
  if (nchl > 0) {
    dim3 gv((unsigned)((N + 255) / 256), (unsigned)nchl);
    if (f64) k_adj_vt<1><<<gv, 256, 0, c->stream>>>(N, c->row0, c->row0 + nv, ld, Vf64, Vhi, Vlo, nbar, vtpart);
    else k_adj_vt<0><<<gv, 256, 0, c->stream>>>(N, c->row0, c->row0 + nv, ld, Vf64, Vhi, Vlo, nbar, vtpart);
    BIE_LAUNCH_CHECK(c, "k_adj_vt");
  }
  if (partitioned(c)) {   // V^T Nbar = sum over the parts of their rows' contributions
    if (nchl > 0) {
      k_adj_vt_sum<<<(N + 255) / 256, 256, 0, c->stream>>>(N, ld, nchl, vtpart);
      BIE_LAUNCH_CHECK(c, "k_adj_vt_sum");
    } else {
      BIE_CUDA_TRY(c, cudaMemsetAsync(vtpart, 0, sizeof(double) * N, c->stream));
    }
    s = part_allreduce(c, vtpart, N);
    if (s != BIE_OK) return s;
    nsum = 1;
  }
  k_adj_dft_in<<<(nX + 255) / 256, 256, 0, c->stream>>>(N, M0, ld, nsum, vtpart, wgt64, nbar, omega, xin);
  BIE_LAUNCH_CHECK(c, "k_adj_dft_in");
  {
    DftJobs J1, J2;
    memset(&J1, 0, sizeof(J1));
    memset(&J2, 0, sizeof(J2));
    int t = 0;
    for (int k = 0; k < c->nb; ++k) {
      const int M = c->M[k], M1 = c->fft_m1[k], o0 = c->off[k];
      J1.j[J1.n++] = DftJob{M, M1, M / M1, o0, o0, o0, 0, t};
      J2.j[J2.n++] = DftJob{M, M1, M / M1, o0, o0, o0, 1, t};
      t += M;
    }
    J1.j[J1.n++] = DftJob{M0, c->fft_m1[0], M0 / c->fft_m1[0], N, N, 0, 0, t};
    J2.j[J2.n++] = DftJob{M0, c->fft_m1[0], M0 / c->fft_m1[0], N, N, 0, 2, t};
    t += M0;
    for (int k = 0; k < c->nb; ++k) {
      const int M = c->M[k], M1 = c->fft_m1[k], o0 = c->off[k];
      J1.j[J1.n++] = DftJob{M, M1, M / M1, N + M0 + o0, N + M0 + o0, o0, 0, t};
      J2.j[J2.n++] = DftJob{M, M1, M / M1, N + M0 + o0, N + M0 + o0, o0, 1, t};
      t += M;
    }
    J1.total = J2.total = t;
    s = dft_pass(c, J1, xin, nullptr, tw, dY, dX1);
    if (s != BIE_OK) return s;
    s = dft_pass(c, J2, nullptr, dX1, tw, dY, dX2);
    if (s != BIE_OK) return s;
  }
  k_adj_rhs<<<(N + 255) / 256, 256, 0, c->stream>>>(B, dX2, omega, nbar, rhs, coef);
  BIE_LAUNCH_CHECK(c, "k_adj_rhs");
  // 3. adjoint system on the transposed storage
  c->assembled = false;
  s = asm_run(c, c->precision, 1);
  if (s != BIE_OK) return s;
  c->assembled = true;
  c->transposed = true;
  const bie_status ss = solve_system(c, &o, mu, rhs, info);
  if (ss != BIE_OK && ss != BIE_ERR_NOCONV) return ss;
  k_adj_lambda<<<(N + 255) / 256, 256, 0, c->stream>>>(N, M0, mu, wgt64, coef, coefdf, g->lambda,
                                                       g->g_phit ? g->g_phit : gphit_buf);
  BIE_LAUNCH_CHECK(c, "k_adj_lambda");
  // 4. geometry terms
  const unsigned npairs = (unsigned)((long long)ntile * (ntile + 1) / 2);
  if (f64) k_adj_pairs<double><<<npairs, 256, 0, c->stream>>>(a);
  else k_adj_pairs<dfl><<<npairs, 256, 0, c->stream>>>(a);
  BIE_LAUNCH_CHECK(c, "k_adj_pairs");
  k_adj_node<<<(N + 255) / 256, 256, 0, c->stream>>>(B, F, z64, dz64, d2z64, coef, gU, U, gnode, gzcp);
  BIE_LAUNCH_CHECK(c, "k_adj_node");
  k_adj_reduce<<<(N + 255) / 256, 256, 0, c->stream>>>(N, ntile, part, gnode, gz, gzp, gzpp);
  BIE_LAUNCH_CHECK(c, "k_adj_reduce");
  if (nobs > 0) {
    k_adj_zc<<<nobs, 256, 0, c->stream>>>(N, gzcp, gzc);
    BIE_LAUNCH_CHECK(c, "k_adj_zc");
  }
  const size_t cb = sizeof(double2) * (size_t)N;
  if (g->g_zeta) BIE_CUDA_TRY(c, cudaMemcpyAsync(g->g_zeta, gz, cb, cudaMemcpyDeviceToDevice, c->stream));
  if (g->g_dzeta) BIE_CUDA_TRY(c, cudaMemcpyAsync(g->g_dzeta, gzp, cb, cudaMemcpyDeviceToDevice, c->stream));
  if (g->g_d2zeta)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(g->g_d2zeta, gzpp, cb, cudaMemcpyDeviceToDevice, c->stream));
  if (g->g_zc && nobs > 0)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(g->g_zc, gzc, sizeof(double2) * nobs, cudaMemcpyDeviceToDevice, c->stream));
  // 5. chains
  if (g->g_node) {
    // g = gzeta - D(gzeta' - D gzeta'')
    s = spectral_d(c, gzpp, tw, dY, dX1, dX2);
    if (s != BIE_OK) return s;
    k_adj_axpy_d<<<(N + 255) / 256, 256, 0, c->stream>>>(B, gzp, dX2, tmp);
    BIE_LAUNCH_CHECK(c, "k_adj_axpy_d");
    s = spectral_d(c, tmp, tw, dY, dX1, dX2);
    if (s != BIE_OK) return s;
    k_adj_axpy_d<<<(N + 255) / 256, 256, 0, c->stream>>>(B, gz, dX2, (double2*)g->g_node);
    BIE_LAUNCH_CHECK(c, "k_adj_axpy_d");
  }
  if (g->g_shape && nobs > 0) {
    k_adj_shape<<<nobs, 256, 0, c->stream>>>(B, E, gz, gzp, gzpp, gzc, g->g_shape);
    BIE_LAUNCH_CHECK(c, "k_adj_shape");
  }
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return ss;
}
