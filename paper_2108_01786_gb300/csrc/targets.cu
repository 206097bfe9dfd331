// Velocity u - i v = Phi'(z) on the boundaries and at points of the fluid
// (Sec. 5.1 and App. F).
//
//  * Boundary values Phi'(zeta_k(alpha_m)) = (phi_s - i phi_n) s_alpha / zeta_k'
//    (eq. phi:prime) with s phi_n, s phi_s from eqs. dphij:dnk and dphij:dsk,
//    gamma_0 = -omega_0', gamma_j = omega_j' (eq. gam:def).  Every boundary node
//    is a target; the sources are all nodes (double-float, matrix-free).
//  * Far targets: the trapezoidal Cauchy sums of eqs. Phi:j:prime and
//    Phi:0:prime plus Phi_mv' (FP32; accurate to single precision once the
//    target is a few node spacings from every boundary).
//  * Near targets: the Helsing-Ojala ratio of eq. helsing:quad over the
//    boundary values, with the free surface entering with -zeta_0' (positive
//    orientation of the boundary of Omega), in double-float.
#include <cstring>

#include "common.cuh"
#include "nvtx.cuh"
#include "dft.cuh"
#include "pair_kernel.cuh"
#include "df2.cuh"

#define BND_CH 512
#define BND_FIELDS 5   // Z0.re Z0.im Z1.re Z1.im tsum

// gamma_l / M_l and H gamma_l (double-float) from the two inverse DFTs:
// X2[0..N) = DFT-side of i k omega-hat (-> omega'), X2[N..2N) of |k| omega-hat.
__global__ void k_gamma_extract(Blocks B, const double2* __restrict__ X2, float2* __restrict__ gc,
                                float2* __restrict__ hg, float* __restrict__ cf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.N) return;
  int k = 0;
  while (k + 1 < B.nb && t >= B.off[k + 1]) ++k;
  const double M = (double)B.M[k];
  const double sg = (k == 0) ? -1.0 : 1.0;
  const double wp = X2[t].x / M;              // omega'
  const double hw = X2[B.N + t].x / M;        // H omega'
  const dfl g = df_from_double(sg * wp / M);  // gamma / M
  gc[t] = make_float2(g.hi, g.lo);
  const dfl h = df_from_double(sg * hw);      // H gamma
  hg[t] = make_float2(h.hi, h.lo);
  cf[t] = (float)(wp / M);                    // omega' / M (far-field sums)
}

// Partial sums for boundary targets m over a chunk of sources l != m:
//   Z0 = sum_{l on Gamma_0} G_ml c_l,  Z1 = sum_{l off Gamma_0} G_ml c_l,
//   tsum = sum_{l on m's boundary} 1/2 cot(pi (i_m - i_l)/M_k) c_l,
// G_ml = 1/2 cot((zeta_l - zeta_m)/2), c_l = gamma_l / M_l.
__global__ void __launch_bounds__(256) k_bnd_partial(Blocks B, const float4* __restrict__ nP,
                                                     const float4* __restrict__ nQ,
                                                     const float4* __restrict__ nPQc,
                                                     const double2* __restrict__ z64,
                                                     const int* __restrict__ blk,
                                                     const float2* __restrict__ gc,
                                                     const float2* __restrict__ Tall, float near2,
                                                     float2* __restrict__ part) {
  __shared__ float4 sP[BND_CH];
  __shared__ float2 sPc[BND_CH];
  __shared__ double2 sZ[BND_CH];
  __shared__ float2 sC[BND_CH];
  __shared__ int sB[BND_CH];
  const int N = B.N;
  const int s0 = blockIdx.y * BND_CH;
  const int ns = min(BND_CH, N - s0);
  for (int t = threadIdx.x; t < ns; t += blockDim.x) {
    sP[t] = nP[s0 + t];
    const float4 pq = nPQc[s0 + t];
    sPc[t] = make_float2(pq.x, pq.y);
    sZ[t] = z64[s0 + t];
    sC[t] = gc[s0 + t];
    sB[t] = blk[s0 + t];
  }
  __syncthreads();
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const float4 qv = nQ[m];
  const cx<dfl> Q = {{qv.x, qv.y}, {qv.z, qv.w}};
  const float4 qc4 = nPQc[m];
  const float2 Qc = make_float2(qc4.z, qc4.w);
  const double2 zm = z64[m];
  const int km = blk[m];
  const int om = B.off[km], Mk = B.M[km], im = m - om;
  dfl Z0r = {0, 0}, Z0i = {0, 0}, Z1r = {0, 0}, Z1i = {0, 0}, ts = {0, 0};
  for (int t = 0; t < ns; ++t) {
    const int l = s0 + t;
    if (l == m) continue;
    const float4 pv = sP[t];
    const cx<dfl> P = {{pv.x, pv.y}, {pv.z, pv.w}};
    const cx<dfl> G = half_cot_pair<dfl>(P, Q, sPc[t], Qc, sZ[t], zm, near2);
    const float2 cv = sC[t];
    const dfl c = {cv.x, cv.y};
    const dfl gr = G.re * c, gi = G.im * c;
    const int bl = sB[t];
    if (bl == 0) {
      Z0r = Z0r + gr;
      Z0i = Z0i + gi;
    } else {
      Z1r = Z1r + gr;
      Z1i = Z1i + gi;
    }
    if (bl == km) {
      int idx = im - (l - om);
      if (idx < 0) idx += Mk;
      const float2 tv = Tall[om + idx];
      ts = ts + dfl{tv.x, tv.y} * c;
    }
  }
  float2* p = part + (size_t)blockIdx.y * BND_FIELDS * N;
  p[0 * (size_t)N + m] = make_float2(Z0r.hi, Z0r.lo);
  p[1 * (size_t)N + m] = make_float2(Z0i.hi, Z0i.lo);
  p[2 * (size_t)N + m] = make_float2(Z1r.hi, Z1r.lo);
  p[3 * (size_t)N + m] = make_float2(Z1i.hi, Z1i.lo);
  p[4 * (size_t)N + m] = make_float2(ts.hi, ts.lo);
}

// Phi'(zeta_m) from the partial sums (eqs. dphij:dnk, dphij:dsk, phi:prime):
//   C_ml = zeta_m' 1/2 cot((zeta_m - zeta_l)/2) - [same boundary] 1/2 cot((alpha_m - beta_l)/2)
//        = -zeta_m' G_ml - [same boundary] T,   C_mm = zeta''/(2 zeta')
//   A0 = sum_{l on Gamma_0} C c,  A1 = sum_{l off Gamma_0} C c
//   s phi_n = Re{Phi_mv' i zeta'} + Re A0 + Im A1 + [k=0] 1/2 H gamma_0 - [k>=1] 1/2 gamma_k
//   s phi_s = Re{Phi_mv' zeta'}   + Im A0 - Re A1 + [k=0] 1/2 gamma_0   - [k>=1] 1/2 H gamma_k
__global__ void k_bnd_finish(Blocks B, FlowParams F, int nchunk, const float2* __restrict__ part,
                             const double2* __restrict__ z64, const double2* __restrict__ dz64,
                             const double2* __restrict__ d2z64, const int* __restrict__ blk,
                             const float2* __restrict__ gc, const float2* __restrict__ hg,
                             double2* __restrict__ f64, float4* __restrict__ fdf) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= B.N) return;
  const int N = B.N;
  dfl acc[BND_FIELDS];
  for (int f = 0; f < BND_FIELDS; ++f) acc[f] = {0.f, 0.f};
  for (int ch = 0; ch < nchunk; ++ch) {
    const float2* p = part + (size_t)ch * BND_FIELDS * N;
    for (int f = 0; f < BND_FIELDS; ++f) {
      const float2 v = p[(size_t)f * N + m];
      acc[f] = acc[f] + dfl{v.x, v.y};
    }
  }
  const double Z0r = df_to_double(acc[0]), Z0i = df_to_double(acc[1]);
  const double Z1r = df_to_double(acc[2]), Z1i = df_to_double(acc[3]);
  const double ts = df_to_double(acc[4]);
  const int k = blk[m];
  const double Mk = (double)B.M[k];
  const double2 zp = dz64[m], zpp = d2z64[m], zm = z64[m];
  const double cm = df_to_double(dfl{gc[m].x, gc[m].y});
  const double gam = cm * Mk;
  const double hgam = df_to_double(dfl{hg[m].x, hg[m].y});
  // -zeta' Z
  double A0r = -(zp.x * Z0r - zp.y * Z0i), A0i = -(zp.x * Z0i + zp.y * Z0r);
  double A1r = -(zp.x * Z1r - zp.y * Z1i), A1i = -(zp.x * Z1i + zp.y * Z1r);
  // diagonal term zeta''/(2 zeta') c_m
  const double den = 2.0 * (zp.x * zp.x + zp.y * zp.y);
  const double dre = (zpp.x * zp.x + zpp.y * zp.y) / den, dim = (zpp.y * zp.x - zpp.x * zp.y) / den;
  if (k == 0) {
    A0r += -ts + dre * cm;
    A0i += dim * cm;
  } else {
    A1r += -ts + dre * cm;
    A1i += dim * cm;
  }
  // Phi_mv'(zeta) = V1 + sum_j a_j (1/2 - i 1/2 cot((zeta - z_j)/2))
  double pr = F.V1, pi = 0.0;
  for (int j = 2; j < F.nb; ++j) {
    const double ux = zm.x - F.zc[j - 2].x, uy = zm.y - F.zc[j - 2].y;
    double s, c;
    sincos(ux, &s, &c);
    const double e = exp(-uy);
    const double qr = e * c - 1.0, qi = e * s;      // e^{iu} - 1
    const double n2 = qr * qr + qi * qi;
    const double hr = qi / n2, hi = 0.5 + qr / n2;  // 1/2 cot(u/2) = i/2 + i/q
    pr += F.a[j - 2] * (0.5 + hi);                  // 1/2 - i (hr + i hi)
    pi += F.a[j - 2] * (-hr);
  }
  const double mvn = -(pr * zp.y + pi * zp.x);      // Re{Phi_mv' i zeta'}
  const double mvs = pr * zp.x - pi * zp.y;         // Re{Phi_mv' zeta'}
  double sn = mvn + A0r + A1i, ss = mvs + A0i - A1r;
  if (k == 0) {
    sn += 0.5 * hgam;
    ss += 0.5 * gam;
  } else {
    sn -= 0.5 * gam;
    ss -= 0.5 * hgam;
  }
  // (ss - i sn) / zeta'
  const double n = zp.x * zp.x + zp.y * zp.y;
  const double fr = (ss * zp.x - sn * zp.y) / n, fi = (-sn * zp.x - ss * zp.y) / n;
  f64[m] = make_double2(fr, fi);
  const dfl a = df_from_double(fr), b = df_from_double(fi);
  fdf[m] = make_float4(a.hi, a.lo, b.hi, b.lo);
}

// Far targets (FP32): Phi'(z) = Phi_mv'(z) + sum_{l off Gamma_0} H_l c_l - i sum_{l on Gamma_0} H_l c_l,
// H_l = 1/2 cot((zeta_l - z)/2) = i/2 + i/(P_l e^{-iz} - 1), c_l = omega_l'/M_l.
// Also the smallest |zeta_l - z|^2 / h_l^2 (h_l the local node spacing); with
// near_thr2 > 0, targets below it are appended to the Helsing list.
#define FAR_CH 1024

// Over sources [i0, i1) of the chunk: (sr, si) += sum c_l i/d_l, d_l = P_l Q - 1
// = wr + i wi, i/d = (wi + i wr)/|d|^2; optionally the smallest |d|^2 / h_l^2
// (near-target test).
template <bool NEAR>
__device__ __forceinline__ void far_sum(const float4* __restrict__ sP, int i0, int i1, float qr,
                                        float qi, float& sr, float& si, float& dmin) {
#pragma unroll 4
  for (int i = i0; i < i1; ++i) {
    const float4 p = sP[i];
    const float wr = fmaf(p.x, qr, -fmaf(p.y, qi, 1.0f));   // Re(P Q) - 1
    const float wi = fmaf(p.x, qi, p.y * qr);               // Im(P Q)
    const float n2 = fmaf(wr, wr, wi * wi);
    const float q = p.z * rcp_approx(n2);
    if (NEAR) dmin = fminf(dmin, n2 * p.w);
    sr = fmaf(wi, q, sr);
    si = fmaf(wr, q, si);
  }
}

// Far targets (FP32): Phi'(z) = Phi_mv'(z) + sum_{l off Gamma_0} G_l c_l - i sum_{l on Gamma_0} G_l c_l,
// G_l = 1/2 cot((zeta_l - z)/2) = i/2 + i/d_l, c_l = omega_l'/M_l.  The i/2 part
// drops out: sum_l omega_l' = 0 on every boundary (the spectral derivative has
// no mean mode).  The surface and the other boundaries are separate loops
// (no per-source branch).  With NEAR, targets whose nearest node is closer
// than sqrt(near_thr2) local spacings are appended to the Helsing list.
template <bool NEAR>
__global__ void __launch_bounds__(256) k_targets_far(int n, const double2* __restrict__ z, int N,
                                                     int M0, const float4* __restrict__ nP,
                                                     const float* __restrict__ cf,
                                                     const float* __restrict__ hinv2,
                                                     FlowParams F, double2* __restrict__ uv,
                                                     float near_thr2, int* __restrict__ nlist,
                                                     int* __restrict__ ncount) {
  __shared__ float4 sP[FAR_CH];   // (P.re, P.im, c, 1/h^2)
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < n;
  double2 zt = make_double2(0.0, 0.0);
  float qr = 0.f, qi = 0.f;
  if (active) {
    zt = z[t];
    double s, c;
    sincos(zt.x, &s, &c);
    const double e = exp(zt.y);
    qr = (float)(e * c);
    qi = (float)(-e * s);
  }
  float s0r = 0.f, s0i = 0.f, s1r = 0.f, s1i = 0.f, dmin = 3.0e38f;
  for (int b0 = 0; b0 < N; b0 += FAR_CH) {
    const int nb = min(FAR_CH, N - b0);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      const float4 p = nP[b0 + i];
      sP[i] = make_float4(p.x, p.z, cf[b0 + i], NEAR ? hinv2[b0 + i] : 0.f);
    }
    __syncthreads();
    if (!active) continue;
    const int ns = min(nb, max(0, M0 - b0));   // surface sources in this chunk
    far_sum<NEAR>(sP, 0, ns, qr, qi, s0r, s0i, dmin);
    far_sum<NEAR>(sP, ns, nb, qr, qi, s1r, s1i, dmin);
  }
  if (!active) return;
  // Phi_mv'(z) in FP64
  double pr = F.V1, pi = 0.0;
  for (int j = 2; j < F.nb; ++j) {
    const double ux = zt.x - F.zc[j - 2].x, uy = zt.y - F.zc[j - 2].y;
    double s, c;
    sincos(ux, &s, &c);
    const double e = exp(-uy);
    const double wr = e * c - 1.0, wi = e * s;
    const double n2 = wr * wr + wi * wi;
    const double hr = wi / n2, hi = 0.5 + wr / n2;
    pr += F.a[j - 2] * (0.5 + hi);
    pi += F.a[j - 2] * (-hr);
  }
  // sum G c = i sum c/d = (S.re, S.im) with S = (wi q, wr q); -i S0 = (S0.im, -S0.re)
  uv[t] = make_double2(pr + (double)s1r + (double)s0i, pi + (double)s1i - (double)s0r);
  if (NEAR && dmin < near_thr2) {
    const int slot = atomicAdd(ncount, 1);
    nlist[slot] = t;
  }
}

// Helsing-Ojala (eq. helsing:quad): Phi'(z) = sum lam f / sum lam,
// lam_l = (sigma_l / M_l) zeta_l' 1/2 cot((zeta_l - z)/2), sigma = -1 on the
// surface, +1 elsewhere; a target on a node returns the node value.  Each
// target's source sums are shared by HEL_SPLIT consecutive lanes (strided
// sources, a fixed shuffle tree), HEL_TPB targets per 256-thread CTA.
#define HEL_CH 512
#define HEL_SPLIT 8
#define HEL_TPB (256 / HEL_SPLIT)
__device__ __forceinline__ dfl hel_group_sum(dfl v) {
#pragma unroll
  for (int o = HEL_SPLIT / 2; o > 0; o >>= 1) {
    const dfl u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = v + u;
  }
  return v;
}

// Two sources per lane at once, in the two lanes of the packed double-float
// arithmetic (df2): a chunk's sources are staged pair-major, source i of the
// lane's stride beside source i + HEL_SPLIT, so one float4 load gives a
// quantity for both.  Per pair of sources: d = P Q - 1 and |d|^2, H = i/2 +
// i/d, lam = H E and lam f each as combined double-float products, the sums
// accumulated inside the last ones.
struct HelPk {
  float4 Pr, Pi, Er, Ei, Fr, Fi;   // (hi a, hi b, lo a, lo b) of each component
};
__device__ __forceinline__ df2 hel_pk(const float4& v) { return {f2(v.x, v.y), f2(v.z, v.w)}; }

__global__ void __launch_bounds__(256) k_targets_helsing(int n, const int* __restrict__ list,
                                                         const int* __restrict__ count,
                                                         const double2* __restrict__ z, int N,
                                                         const float4* __restrict__ nP,
                                                         const float4* __restrict__ nEw,
                                                         const float4* __restrict__ fdf,
                                                         double2* __restrict__ uv) {
  __shared__ HelPk sK[HEL_CH / 2];
  const int cnt = list ? *count : n;
  // the grid covers every target; CTAs past the near list have nothing to do
  // (returning here keeps them from staging every source chunk)
  if ((int)(blockIdx.x * HEL_TPB) >= cnt) return;
  const int t = blockIdx.x * HEL_TPB + (int)threadIdx.x / HEL_SPLIT;
  const int sub = (int)threadIdx.x % HEL_SPLIT;
  const bool active = t < cnt;
  const int tg = active ? (list ? list[t] : t) : 0;
  df2 Qr = {f2(0.f), f2(0.f)}, Qi = {f2(0.f), f2(0.f)};
  if (active) {
    const double2 zt = z[tg];
    double s, c;
    sincos(zt.x, &s, &c);
    const double e = exp(zt.y);
    const dfl qr = df_from_double(e * c), qi = df_from_double(-e * s);
    Qr = {f2(qr.hi), f2(qr.lo)};
    Qi = {f2(qi.hi), f2(qi.lo)};
  }
  const df2 nQi = d2_neg(Qi);
  df2 nr = {f2(0.f), f2(0.f)}, ni = nr, dr = nr, di = nr;
  int hit = -1;
  for (int b0 = 0; b0 < N; b0 += HEL_CH) {
    const int nb = min(HEL_CH, N - b0);
    const int npk = (nb + 2 * HEL_SPLIT - 1) / (2 * HEL_SPLIT) * HEL_SPLIT;   // staged pairs
    __syncthreads();
    for (int p = threadIdx.x; p < npk; p += blockDim.x) {
      // pair p holds sources ia = 16 (p / 8) + p % 8 and ib = ia + 8 of the chunk
      const int ia = (p / HEL_SPLIT) * 2 * HEL_SPLIT + p % HEL_SPLIT, ib = ia + HEL_SPLIT;
      const bool oka = ia < nb, okb = ib < nb;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      // a source past the chunk repeats a real source's position with zero weight and value
      const float4 pa = nP[b0 + (oka ? ia : 0)];
      const float4 ea = oka ? nEw[b0 + ia] : z4, fa = oka ? fdf[b0 + ia] : z4;
      const float4 pb = okb ? nP[b0 + ib] : pa;
      const float4 eb = okb ? nEw[b0 + ib] : z4, fb = okb ? fdf[b0 + ib] : z4;
      HelPk k;
      k.Pr = make_float4(pa.x, pb.x, pa.y, pb.y);
      k.Pi = make_float4(pa.z, pb.z, pa.w, pb.w);
      k.Er = make_float4(ea.x, eb.x, ea.y, eb.y);
      k.Ei = make_float4(ea.z, eb.z, ea.w, eb.w);
      k.Fr = make_float4(fa.x, fb.x, fa.y, fb.y);
      k.Fi = make_float4(fa.z, fb.z, fa.w, fb.w);
      sK[p] = k;
    }
    __syncthreads();
    if (!active) continue;
    for (int p = sub; p < npk; p += HEL_SPLIT) {
      const HelPk k = sK[p];
      const df2 Pr = hel_pk(k.Pr), Pi = hel_pk(k.Pi);
      // d = P Q - 1
      const df2 d_r = d2_dot2<true>(Pr, Qr, Pi, nQi, f2(-1.f), f2(0.f));
      const df2 d_i = d2_dot2<false>(Pr, Qi, Pi, Qr, f2(0.f), f2(0.f));
      const df2 n2 = d2_dot2<false>(d_r, d_r, d_i, d_i, f2(0.f), f2(0.f));
      if (n2.hi.x < 1e-28f || n2.hi.y < 1e-28f) {   // the target sits on a node
        const int ia = (p / HEL_SPLIT) * 2 * HEL_SPLIT + p % HEL_SPLIT;
        if (n2.hi.x < 1e-28f && ia < nb) hit = b0 + ia;
        if (n2.hi.y < 1e-28f && ia + HEL_SPLIT < nb) hit = b0 + ia + HEL_SPLIT;
        continue;
      }
      const df2 inv = d2_rcp(n2);
      const df2 Hr = d2_mul(d_i, inv);                   // Re(i/2 + i/d)
      const df2 Hi = d2_mul_addf(d_r, inv, f2(0.5f));   // Im(i/2 + i/d)
      const df2 Er = hel_pk(k.Er), Ei = hel_pk(k.Ei);
      const df2 lr = d2_dot2<false>(Hr, Er, d2_neg(Hi), Ei, f2(0.f), f2(0.f));   // lam = H E
      const df2 li = d2_dot2<false>(Hr, Ei, Hi, Er, f2(0.f), f2(0.f));
      const df2 Fr = hel_pk(k.Fr), Fi = hel_pk(k.Fi);
      nr = d2_dot2<true>(lr, Fr, d2_neg(li), Fi, nr.hi, nr.lo);   // += Re(lam f)
      ni = d2_dot2<true>(lr, Fi, li, Fr, ni.hi, ni.lo);           // += Im(lam f)
      dr = d2_add(dr, lr);
      di = d2_add(di, li);
    }
  }
  // the two lanes of every sum, then the lanes of a group (inactive groups carry zeros)
  dfl snr = dfl{nr.hi.x, nr.lo.x} + dfl{nr.hi.y, nr.lo.y};
  dfl sni = dfl{ni.hi.x, ni.lo.x} + dfl{ni.hi.y, ni.lo.y};
  dfl sdr = dfl{dr.hi.x, dr.lo.x} + dfl{dr.hi.y, dr.lo.y};
  dfl sdi = dfl{di.hi.x, di.lo.x} + dfl{di.hi.y, di.lo.y};
  snr = hel_group_sum(snr);
  sni = hel_group_sum(sni);
  sdr = hel_group_sum(sdr);
  sdi = hel_group_sum(sdi);
#pragma unroll
  for (int o = HEL_SPLIT / 2; o > 0; o >>= 1) hit = max(hit, __shfl_xor_sync(0xffffffffu, hit, o));
  if (!active || sub != 0) return;
  if (hit >= 0) {
    const float4 fv = fdf[hit];
    uv[tg] = make_double2((double)fv.x + (double)fv.y, (double)fv.z + (double)fv.w);
    return;
  }
  const double Nr = df_to_double(snr), Ni = df_to_double(sni), Dr = df_to_double(sdr), Di = df_to_double(sdi);
  const double D2 = Dr * Dr + Di * Di;
  uv[tg] = make_double2((Nr * Dr + Ni * Di) / D2, (Ni * Dr - Nr * Di) / D2);
}

// per node: sigma zeta'/M (double-float complex) and 1/h^2 with h = |zeta'| 2 pi / M
__global__ void k_node_weights(Blocks B, const double2* __restrict__ dz, float4* __restrict__ nEw,
                               float* __restrict__ hinv2) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= B.N) return;
  int k = 0;
  while (k + 1 < B.nb && l >= B.off[k + 1]) ++k;
  const double sg = (k == 0) ? -1.0 : 1.0;
  const double M = (double)B.M[k];
  const double2 d = dz[l];
  const dfl er = df_from_double(sg * d.x / M), ei = df_from_double(sg * d.y / M);
  nEw[l] = make_float4(er.hi, er.lo, ei.hi, ei.lo);
  const double h = sqrt(d.x * d.x + d.y * d.y) * (2.0 * M_PI / M);
  hinv2[l] = (float)(1.0 / (h * h));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static bie_status boundary_values(bie_ctx* c, const double* omega, double2** f64_out,
                                  float4** fdf_out, float** cf_out) {
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  const int N = c->N;
  const int nchunk = (N + BND_CH - 1) / BND_CH;
  double2 *dY, *dX1, *dX2, *f64;
  float2 *gc, *hg, *part;
  float4* fdf;
  float* cf;
  BIE_GET(c, double2, "tg_Y", 2 * N, dY);
  BIE_GET(c, double2, "tg_X1", N, dX1);
  BIE_GET(c, double2, "tg_X2", 2 * N, dX2);
  BIE_GET(c, float2, "tg_gc", N, gc);
  BIE_GET(c, float2, "tg_hg", N, hg);
  BIE_GET(c, float, "tg_cf", N, cf);
  BIE_GET(c, float2, "tg_part", (size_t)nchunk * BND_FIELDS * N, part);
  BIE_GET(c, double2, "tg_f64", N, f64);
  BIE_GET(c, float4, "tg_fdf", N, fdf);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  const float2* Tall = (const float2*)ctx_buf(c, "Tall", sizeof(float2) * N, &oom);
  const float4* nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  const float4* nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  const float4* nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  const double2* z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double2* d2z64 = (const double2*)ctx_buf(c, "d2zeta", sizeof(double2) * N, &oom);
  const int* blk = (const int*)ctx_buf(c, "blk", sizeof(int) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "targets: buffers");
  // omega' and H omega' on every boundary
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  int s1 = 0, s2 = 0;
  for (int k = 0; k < c->nb; ++k) {
    const int M = c->M[k], M1 = c->fft_m1[k], o = c->off[k];
    J1.j[J1.n++] = DftJob{M, M1, M / M1, o, o, o, 0, s1};
    s1 += M;
  }
  for (int k = 0; k < c->nb; ++k) {
    const int M = c->M[k], M1 = c->fft_m1[k], o = c->off[k];
    J2.j[J2.n++] = DftJob{M, M1, M / M1, o, o, o, 1, s2};
    s2 += M;
  }
  for (int k = 0; k < c->nb; ++k) {
    const int M = c->M[k], M1 = c->fft_m1[k], o = c->off[k];
    J2.j[J2.n++] = DftJob{M, M1, M / M1, o, N + o, o, 2, s2};
    s2 += M;
  }
  J1.total = s1;
  J2.total = s2;
  k_dft_a<<<dft_grid((s1 + 255) / 256), 256, 0, c->stream>>>(J1, omega, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid((s1 + 255) / 256), 256, 0, c->stream>>>(J1, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid((s2 + 255) / 256), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid((s2 + 255) / 256), 256, 0, c->stream>>>(J2, dY, tw, dX2);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_gamma_extract<<<(N + 255) / 256, 256, 0, c->stream>>>(B, dX2, gc, hg, cf);
  BIE_LAUNCH_CHECK(c, "k_gamma_extract");
  k_bnd_partial<<<dim3((N + 255) / 256, nchunk), 256, 0, c->stream>>>(B, nP, nQ, nPQc, z64, blk, gc,
                                                                     Tall, 0.01f, part);
  BIE_LAUNCH_CHECK(c, "k_bnd_partial");
  k_bnd_finish<<<(N + 255) / 256, 256, 0, c->stream>>>(B, F, nchunk, part, z64, dz64, d2z64, blk, gc,
                                                       hg, f64, fdf);
  BIE_LAUNCH_CHECK(c, "k_bnd_finish");
  *f64_out = f64;
  *fdf_out = fdf;
  if (cf_out) *cf_out = cf;
  return BIE_OK;
}

extern "C" bie_status bie_boundary_velocity(bie_ctx* c, const double* omega_dev, double* f_dev) {
  BIE_NVTX("bie_boundary_velocity");
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom || !c->have_flow)
    return ctx_fail(c, BIE_ERR_STATE, "bie_boundary_velocity: geometry/flow missing");
  if (!omega_dev || !f_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_boundary_velocity: null pointer");
  cudaSetDevice(c->device);
  double2* f64;
  float4* fdf;
  bie_status s = boundary_values(c, omega_dev, &f64, &fdf, nullptr);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(f_dev, f64, sizeof(double2) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  return BIE_OK;
}

bie_status boundary_potential_run(bie_ctx* c, const double* omega, double2* out);

// (re, im) in FP64 -> (re.hi, re.lo, im.hi, im.lo) double-float
__global__ void k_c_to_df(int n, const double2* __restrict__ v, float4* __restrict__ o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dfl r = df_from_double(v[i].x), m = df_from_double(v[i].y);
  o[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
}

// Phi~(z) at points of Omega: Helsing-Ojala quadrature (eq. helsing:quad)
// applied to the boundary values of Phi~ from the Plemelj formula; Phi~ is
// analytic and single valued in Omega, so the ratio is exact up to the
// trapezoidal rule near and far from the boundaries alike.
extern "C" bie_status bie_eval_potential(bie_ctx* c, const double* omega_dev, long long n,
                                         const double* z_dev, double* phi_dev) {
  BIE_NVTX("bie_eval_potential");
  if (!c) return BIE_ERR_ARG;
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_eval_potential: not assembled");
  if (c->transposed || c->variant != 0)
    return ctx_fail(c, BIE_ERR_STATE,
                    "bie_eval_potential: storage must hold the operator of eq. lin:sys; assemble again");
  if (n < 0 || n > (1LL << 30) || (n > 0 && (!omega_dev || !z_dev || !phi_dev)))
    return ctx_fail(c, BIE_ERR_ARG, "bie_eval_potential: bad argument");
  if (n == 0) return BIE_OK;
  cudaSetDevice(c->device);
  const Blocks B = make_blocks(c);
  const int N = c->N;
  double2* bnd;
  float4 *fdf, *nEw;
  float* hinv2;
  BIE_GET(c, double2, "ep_bnd", N, bnd);
  BIE_GET(c, float4, "ep_fdf", N, fdf);
  BIE_GET(c, float4, "tg_nEw", N, nEw);
  BIE_GET(c, float, "tg_hinv2", N, hinv2);
  bool oom = false;
  const float4* nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_eval_potential: buffers");
  bie_status s = boundary_potential_run(c, omega_dev, bnd);
  if (s != BIE_OK) return s;
  k_c_to_df<<<(N + 255) / 256, 256, 0, c->stream>>>(N, bnd, fdf);
  BIE_LAUNCH_CHECK(c, "k_c_to_df");
  k_node_weights<<<(N + 255) / 256, 256, 0, c->stream>>>(B, dz64, nEw, hinv2);
  BIE_LAUNCH_CHECK(c, "k_node_weights");
  k_targets_helsing<<<(unsigned)((n + HEL_TPB - 1) / HEL_TPB), 256, 0, c->stream>>>(
      (int)n, nullptr, nullptr, (const double2*)z_dev, N, nP, nEw, fdf, (double2*)phi_dev);
  BIE_LAUNCH_CHECK(c, "k_targets_helsing");
  return BIE_OK;
}

extern "C" bie_status bie_eval_velocity(bie_ctx* c, const double* omega_dev, long long n,
                                        const double* z_dev, double* uv_dev, int mode,
                                        double near_spacings, long long* n_near_out) {
  BIE_NVTX("bie_eval_velocity");
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom || !c->have_flow)
    return ctx_fail(c, BIE_ERR_STATE, "bie_eval_velocity: geometry/flow missing");
  if (n < 0 || n > (1LL << 30) || (n > 0 && (!omega_dev || !z_dev || !uv_dev)) || mode < 0 ||
      mode > 2 || (mode == 2 && !(near_spacings > 0.0)))
    return ctx_fail(c, BIE_ERR_ARG, "bie_eval_velocity: bad argument");
  if (n_near_out) *n_near_out = 0;
  if (n == 0) return BIE_OK;
  cudaSetDevice(c->device);
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  const int N = c->N;
  double2* f64;
  float4* fdf;
  float* cf;
  bie_status s = boundary_values(c, omega_dev, &f64, &fdf, &cf);
  if (s != BIE_OK) return s;
  float4* nEw;
  float* hinv2;
  int *nlist, *ncount;
  BIE_GET(c, float4, "tg_nEw", N, nEw);
  BIE_GET(c, float, "tg_hinv2", N, hinv2);
  BIE_GET(c, int, "tg_nlist", n, nlist);
  BIE_GET(c, int, "tg_ncount", 1, ncount);
  bool oom = false;
  const float4* nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "targets: buffers");
  k_node_weights<<<(N + 255) / 256, 256, 0, c->stream>>>(B, dz64, nEw, hinv2);
  BIE_LAUNCH_CHECK(c, "k_node_weights");
  const double2* z = (const double2*)z_dev;
  double2* uv = (double2*)uv_dev;
  const unsigned g = (unsigned)((n + 255) / 256);
  if (mode == 1) {
    k_targets_helsing<<<(unsigned)((n + HEL_TPB - 1) / HEL_TPB), 256, 0, c->stream>>>(
        (int)n, nullptr, nullptr, z, N, nP, nEw, fdf, uv);
    BIE_LAUNCH_CHECK(c, "k_targets_helsing");
    if (n_near_out) *n_near_out = n;
    return BIE_OK;
  }
  BIE_CUDA_TRY(c, cudaMemsetAsync(ncount, 0, sizeof(int), c->stream));
  const float thr2 = mode == 2 ? (float)(near_spacings * near_spacings) : 0.f;
  if (mode == 2)
    k_targets_far<true><<<g, 256, 0, c->stream>>>((int)n, z, N, c->M[0], nP, cf, hinv2, F, uv, thr2,
                                                  nlist, ncount);
  else
    k_targets_far<false><<<g, 256, 0, c->stream>>>((int)n, z, N, c->M[0], nP, cf, hinv2, F, uv, thr2,
                                                   nlist, ncount);
  BIE_LAUNCH_CHECK(c, "k_targets_far");
  if (mode == 2) {
    k_targets_helsing<<<(unsigned)((n + HEL_TPB - 1) / HEL_TPB), 256, 0, c->stream>>>(
        (int)n, nlist, ncount, z, N, nP, nEw, fdf, uv);
    BIE_LAUNCH_CHECK(c, "k_targets_helsing");
    if (n_near_out) {
      int h = 0;
      BIE_CUDA_TRY(c, cudaMemcpyAsync(&h, ncount, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      *n_near_out = h;
    }
  }
  return BIE_OK;
}
