// Time evolution of the graph formulation (Sec. 2, eqs. graph:eta:t and
// phitileq, xi = alpha) on the GPU, the 36th-order filter of eq. filter, and
// the conserved energy of eq. E:formula (Sec. 5.2).
//
// One right-hand-side evaluation: the surface zeta_0 = alpha + i eta with
// zeta_0' and zeta_0'' from spectral derivatives of eta (FP64 four-step DFT),
// the node tables rebuilt, the matrix assembled and the system solved by the
// library's own kernels, then eta_t = s_alpha U and phi~_t of eq. phitileq
// (V = eta_alpha U, C(t) = 0, rho = 1) in one FP64 pass over the surface.
// Classical RK4 advances (eta, phi~); the filter, when asked for, acts on both
// at the end of each step, not in the stages.
//
// The energy needs psi on the surface: psi_0 = 1/2 H omega_0 - G_00 omega_0 +
// sum_j K_0j omega_j + psi_mv (Table 1 rows for the imaginary part, Plemelj
// step of eq. plemelj:ver2), a matrix-free pass over M_0 x N node pairs with
// the assembly's double-float kernel G = 1/2 cot((zeta_l - zeta_m)/2).
#include <cmath>
#include <cstring>
#include <vector>
#include "common.cuh"
#include "nvtx.cuh"
#include "dft.cuh"
#include "pair_kernel.cuh"

namespace {

// node data of the double-float pair kernel (the assembly's tables)
struct PairNodes {
  const float4* nP;     // e^{i zeta} (df complex)
  const float4* nQ;     // e^{-i zeta}
  const float4* nPQc;   // third words of P (x, y) and Q (z, w)
  const float4* nZp;    // zeta' (df complex)
  const float2* Ttab;   // 1/2 cot(pi j / M_0), df
  const double2* z64;
};

__device__ __forceinline__ cx<dfl> ld_cx(const float4* a, int i) {
  const float4 v = a[i];
  return {{v.x, v.y}, {v.z, v.w}};
}

__device__ __forceinline__ dfl df_shfl_sum(dfl v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dfl u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = v + u;
  }
  return v;
}

// y = [eta | phi~] (2 M_0) -> X2 = [eta_alpha | phi~_alpha | eta_alpha_alpha] x M_0
bie_status graph_derivs(bie_ctx* c, const double* y, double2* X2) {
  const int M0 = c->M[0], M1 = c->fft_m1[0], M2 = M0 / M1;
  double2 *dY, *dX1;
  BIE_GET(c, double2, "ev_Y", 3 * (size_t)M0, dY);
  BIE_GET(c, double2, "ev_X1", 2 * (size_t)M0, dX1);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * c->N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "evolve: twiddles");
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  J1.j[J1.n++] = DftJob{M0, M1, M2, 0, 0, 0, 0, 0};
  J1.j[J1.n++] = DftJob{M0, M1, M2, M0, M0, 0, 0, M0};
  J1.total = 2 * M0;
  J2.j[J2.n++] = DftJob{M0, M1, M2, 0, 0, 0, 1, 0};
  J2.j[J2.n++] = DftJob{M0, M1, M2, M0, M0, 0, 1, M0};
  J2.j[J2.n++] = DftJob{M0, M1, M2, 0, 2 * M0, 0, 5, 2 * M0};
  J2.total = 3 * M0;
  k_dft_a<<<dft_grid((J1.total + 255) / 256), 256, 0, c->stream>>>(J1, y, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid((J1.total + 255) / 256), 256, 0, c->stream>>>(J1, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid((J2.total + 255) / 256), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid((J2.total + 255) / 256), 256, 0, c->stream>>>(J2, dY, tw, X2);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  return BIE_OK;
}

// zeta_0 = alpha + i eta, zeta_0' = 1 + i eta_alpha, zeta_0'' = i eta_alpha_alpha
__global__ void k_graph_surface(int M0, const double* __restrict__ eta,
                                const double2* __restrict__ X2, double2* __restrict__ z,
                                double2* __restrict__ dz, double2* __restrict__ d2z) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M0) return;
  const double inv = 1.0 / (double)M0;
  const double alpha = (2.0 * M_PI) * (double)m / (double)M0;
  z[m] = make_double2(alpha, eta[m]);
  dz[m] = make_double2(1.0, X2[m].x * inv);
  d2z[m] = make_double2(0.0, X2[2 * M0 + m].x * inv);
}

// Phi_mv'(z) = V1 + sum_j a_j (1/2 - i/2 cot((z - z_j)/2)) (eq. d:phi:cyl)
__device__ __forceinline__ double2 dphi_mv(const FlowParams& F, double2 z) {
  double re = F.V1, im = 0.0;
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
  return make_double2(re, im);
}

// eta_t = s U; phi~_t = (phi~_a/s) V + (U - dphi_mv/dn) U - |grad phi|^2/2 - g eta + tau theta_a/s
__global__ void k_graph_rhs(int M0, FlowParams F, const double2* __restrict__ z,
                            const double2* __restrict__ dz, const double2* __restrict__ d2z,
                            const double* __restrict__ U, const double2* __restrict__ X2,
                            const double* __restrict__ y, double tau, double g,
                            double* __restrict__ ydot) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M0) return;
  const double2 zp = dz[m];
  const double ea = zp.y;
  const double s = sqrt(1.0 + ea * ea);
  const double u = U[m];
  const double2 dP = dphi_mv(F, z[m]);
  const double dphimv_dn = (-dP.x * zp.y - dP.y * zp.x) / s;   // Re{Phi_mv' i zeta'} / s
  const double phit_a = X2[M0 + m].x / (double)M0;
  const double phi_a = phit_a + (dP.x * zp.x - dP.y * zp.y);  // + Re{Phi_mv' zeta'}
  const double grad2 = (phi_a / s) * (phi_a / s) + u * u;
  const double theta_a = d2z[m].y / (1.0 + ea * ea);
  const double V = ea * u;
  ydot[m] = s * u;
  ydot[M0 + m] = (phit_a / s) * V + (u - dphimv_dn) * u - 0.5 * grad2 - g * y[m] + tau * theta_a / s;
}

__global__ void k_axpy2(int n, const double* __restrict__ y, double a, const double* __restrict__ k,
                        double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = y[i] + a * k[i];
}

// out = a + (a - b) c  (one Aitken-Neville update of the extrapolation table)
__global__ void k_extrap(int n, const double* __restrict__ a, const double* __restrict__ b,
                         double c, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + (a[i] - b[i]) * c;
}

// y += dt/6 (k1 + 2 k2 + 2 k3 + k4)
__global__ void k_rk4_final(int n, double dt, const double* __restrict__ k1,
                            const double* __restrict__ k2, const double* __restrict__ k3,
                            const double* __restrict__ k4, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = y[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

// out = y + h sum_j w_j k_j over up to 12 stage derivatives (a Runge-Kutta
// stage argument or the step's new state, in place: out may be y); every
// term is formed in FP64
struct StageSum {
  const double* k[12];
  double w[12];
  int n;
};
__global__ void k_stage_sum(int n, const double* y, double h, StageSum S, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int j = 0; j < S.n; ++j) acc = fma(S.w[j], S.k[j][i], acc);
  out[i] = y[i] + h * acc;
}

// weights as double-float: w[l] = v[l] / M_k (k the boundary of l) when scaled, else v[l]
__global__ void k_to_df(Blocks B, int n, const double* __restrict__ v, int scaled,
                        float2* __restrict__ w) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  double x = v[l];
  if (scaled) {
    int k = 0;
    while (k + 1 < B.nb && l >= B.off[k + 1]) ++k;
    x /= (double)B.M[k];
  }
  const dfl d = df_from_double(x);
  w[l] = make_float2(d.hi, d.lo);
}

#define PS_THREADS 128

// fixed-order double-float sum over a 128-thread CTA (result in thread 0)
__device__ __forceinline__ dfl df_cta_sum(dfl v, dfl* sh) {
  v = df_shfl_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  dfl t = {0.f, 0.f};
  if (threadIdx.x == 0)
    for (int w = 0; w < PS_THREADS / 32; ++w) t = t + sh[w];
  __syncthreads();
  return t;
}

// psi on the surface, one 128-thread CTA per row m: the sums of the file
// comment with the double-float pair kernel of the assembly (separable far
// field, FP64 node differences near the diagonal); the diagonal term in FP64.
// w = omega_l / M_j as double-float.
__global__ void __launch_bounds__(PS_THREADS)
    k_psi_surface(Blocks B, PairNodes nd, const double2* __restrict__ dz,
                  const double2* __restrict__ d2z, const float2* __restrict__ w,
                  const double* __restrict__ omega, const double2* __restrict__ Hx, FlowParams F,
                  double* __restrict__ psi0) {
  __shared__ dfl sh[PS_THREADS / 32];
  const int M0 = B.M[0], N = B.N;
  const int m = blockIdx.x;
  const cx<dfl> Qm = ld_cx(nd.nQ, m);
  const float4 qc = nd.nPQc[m];
  const float2 Qcm = make_float2(qc.z, qc.w);
  const double2 zm = nd.z64[m];
  dfl acc = {0.f, 0.f};
  for (int l = threadIdx.x; l < N; l += PS_THREADS) {
    if (l == m) continue;   // diagonal added below in FP64
    const float4 pc = nd.nPQc[l];
    const cx<dfl> G = half_cot_pair<dfl>(ld_cx(nd.nP, l), Qm, make_float2(pc.x, pc.y), Qcm,
                                         nd.z64[l], zm, 0.01f);
    const cx<dfl> Zl = ld_cx(nd.nZp, l);
    const dfl wl = {w[l].x, w[l].y};
    if (l < M0) {
      const float2 t = nd.Ttab[(l - m + M0) % M0];
      acc = acc - (cre(Zl, G) - dfl{t.x, t.y}) * wl;
    } else {
      acc = acc + cim(Zl, G) * wl;
    }
  }
  acc = df_cta_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double2 a = d2z[m], b = dz[m];
    const double n2 = b.x * b.x + b.y * b.y;
    double tot = (double)acc.hi + (double)acc.lo -
                 0.5 * (a.x * b.x + a.y * b.y) / n2 * omega[m] / (double)M0;
    double pm = F.V1 * zm.y;
    for (int j = 2; j < F.nb; ++j) {
      const double ux = zm.x - F.zc[j - 2].x, uy = zm.y - F.zc[j - 2].y;
      double sn, cs;
      sincos(ux, &sn, &cs);
      const double e = exp(-uy);
      const double re = 1.0 - e * cs, im = -e * sn;
      pm -= F.a[j - 2] * 0.5 * log(re * re + im * im);   // a_j psi_cyl, psi_cyl = -ln|1 - e^{iz}|
    }
    psi0[m] = 0.5 * Hx[m].x / (double)M0 + tot + pm;
  }
}

// E = mean_m(tau s + g eta^2 xi_a / 2 + psi_0 phi_a / 2) + sum_j a_j psi_j / 2 (rho = 1), one CTA
__global__ void k_energy(int M0, FlowParams F, const double2* __restrict__ z,
                         const double2* __restrict__ dz, const double2* __restrict__ Xd,
                         const double* __restrict__ psi0, const double* __restrict__ psik,
                         double tau, double g, double* __restrict__ E) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) {
    const double2 zp = dz[m];
    const double s = sqrt(zp.x * zp.x + zp.y * zp.y);
    const double2 dP = dphi_mv(F, z[m]);
    const double phi_a = Xd[m].x / (double)M0 + (dP.x * zp.x - dP.y * zp.y);
    const double eta = z[m].y;
    acc += tau * s + 0.5 * g * eta * eta * zp.x + 0.5 * psi0[m] * phi_a;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      double e = t / (double)M0;
      for (int j = 2; j < F.nb; ++j) e += 0.5 * F.a[j - 2] * psik[j - 2];
      *E = e;
    }
  }
}

}  // namespace

// Energy of the state (geometry in the context, phi~ and its solved omega):
// E written to *E_dev (device).
bie_status energy_run(bie_ctx* c, const double* phit, const double* omega, double tau, double g,
                      double* E_dev) {
  BIE_NVTX("energy");
  const int N = c->N, M0 = c->M[0], M1 = c->fft_m1[0], M2 = M0 / M1;
  double2 *dY, *dX1, *dX2;
  double *psi0, *psik;
  BIE_GET(c, double2, "en_Y", 2 * (size_t)M0, dY);
  BIE_GET(c, double2, "en_X1", 2 * (size_t)M0, dX1);
  BIE_GET(c, double2, "en_X2", 2 * (size_t)M0, dX2);
  BIE_GET(c, double, "en_psi0", M0, psi0);
  BIE_GET(c, double, "en_psik", BIE_MAXB, psik);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  const double2* z = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double2* d2z = (const double2*)ctx_buf(c, "d2zeta", sizeof(double2) * N, &oom);
  PairNodes nd;
  nd.nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  nd.nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  nd.nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  nd.nZp = (const float4*)ctx_buf(c, "nZp", sizeof(float4) * N, &oom);
  nd.Ttab = (const float2*)ctx_buf(c, "Ttab", sizeof(float2) * M0, &oom);
  nd.z64 = z;
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "energy: buffers");
  // H omega_0 (mode 4) at [0, M0) and phi~_alpha (mode 1) at [M0, 2 M0):
  // forward passes of omega_0 and phi~ into X1, inverse passes into X2
  DftJobs Jw, Jp, Jb, J2;
  memset(&Jw, 0, sizeof(Jw));
  memset(&Jp, 0, sizeof(Jp));
  memset(&Jb, 0, sizeof(Jb));
  memset(&J2, 0, sizeof(J2));
  Jw.j[Jw.n++] = DftJob{M0, M1, M2, 0, 0, 0, 0, 0};
  Jw.total = M0;
  Jp.j[Jp.n++] = DftJob{M0, M1, M2, 0, M0, 0, 0, 0};
  Jp.total = M0;
  Jb.j[Jb.n++] = DftJob{M0, M1, M2, 0, 0, 0, 0, 0};
  Jb.j[Jb.n++] = DftJob{M0, M1, M2, M0, M0, 0, 0, M0};
  Jb.total = 2 * M0;
  J2.j[J2.n++] = DftJob{M0, M1, M2, 0, 0, 0, 4, 0};
  J2.j[J2.n++] = DftJob{M0, M1, M2, M0, M0, 0, 1, M0};
  J2.total = 2 * M0;
  const unsigned g1 = (unsigned)((M0 + 255) / 256), g2 = (unsigned)((2 * M0 + 255) / 256);
  k_dft_a<<<dft_grid(g1), 256, 0, c->stream>>>(Jw, omega, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_a<<<dft_grid(g1), 256, 0, c->stream>>>(Jp, phit, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(g2), 256, 0, c->stream>>>(Jb, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid(g2), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(g2), 256, 0, c->stream>>>(J2, dY, tw, dX2);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  float2* wdf;
  BIE_GET(c, float2, "en_wdf", N, wdf);
  k_to_df<<<(N + 255) / 256, 256, 0, c->stream>>>(B, N, omega, 1, wdf);
  BIE_LAUNCH_CHECK(c, "k_to_df");
  k_psi_surface<<<M0, PS_THREADS, 0, c->stream>>>(B, nd, dz, d2z, wdf, omega, dX2, F, psi0);
  BIE_LAUNCH_CHECK(c, "k_psi_surface");
  // psi_j = <1_j, omega> for obstacles (eq. psi:k)
  BIE_CUDA_TRY(c, cudaMemsetAsync(psik, 0, sizeof(double) * BIE_MAXB, c->stream));
  if (c->nb > 2) {
    bie_status s = psi_run(c, omega, psik);
    if (s != BIE_OK) return s;
  }
  k_energy<<<1, 1024, 0, c->stream>>>(M0, F, z, dz, dX2 + M0, psi0, psik, tau, g, E_dev);
  BIE_LAUNCH_CHECK(c, "k_energy");
  return BIE_OK;
}

namespace {

// real part / M_0 of the inverse passes (the filter's output)
__global__ void k_take_real_mode(int n, int M0, const double2* __restrict__ X, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = X[i].x / (double)M0;
}

// eq. filter on nv consecutive surface vectors of x (in place)
bie_status filter_run(bie_ctx* c, double* x, int nv) {
  const int M0 = c->M[0], M1 = c->fft_m1[0], M2 = M0 / M1;
  double2 *dY, *dX1;
  BIE_GET(c, double2, "fl_Y", 2 * (size_t)M0, dY);
  BIE_GET(c, double2, "fl_X1", 2 * (size_t)M0, dX1);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * c->N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "filter: twiddles");
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  for (int v = 0; v < nv; ++v) {
    J1.j[J1.n++] = DftJob{M0, M1, M2, v * M0, v * M0, 0, 0, v * M0};
    J2.j[J2.n++] = DftJob{M0, M1, M2, v * M0, v * M0, 0, 6, v * M0};
  }
  J1.total = J2.total = nv * M0;
  const unsigned gb = (unsigned)((nv * M0 + 255) / 256);
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J1, x, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J1, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J2, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_take_real_mode<<<gb, 256, 0, c->stream>>>(nv * M0, M0, dX1, x);
  BIE_LAUNCH_CHECK(c, "k_take_real_mode");
  return BIE_OK;
}

// forward (mode 0) then inverse passes with modes m0, m1 on two stacked
// surface vectors x = [a | b]: out = [D_m0 a | D_m1 b] (real part / M_0 taken by the caller)
bie_status dft_pair(bie_ctx* c, const double* x, int m0, int m1, double2* out) {
  const int M0 = c->M[0], M1 = c->fft_m1[0], M2 = M0 / M1;
  double2 *dY, *dX1;
  BIE_GET(c, double2, "hp_Y", 2 * (size_t)M0, dY);
  BIE_GET(c, double2, "hp_X1", 2 * (size_t)M0, dX1);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * c->N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "dft: twiddles");
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  J1.j[J1.n++] = DftJob{M0, M1, M2, 0, 0, 0, 0, 0};
  J1.j[J1.n++] = DftJob{M0, M1, M2, M0, M0, 0, 0, M0};
  J2.j[J2.n++] = DftJob{M0, M1, M2, 0, 0, 0, m0, 0};
  J2.j[J2.n++] = DftJob{M0, M1, M2, M0, M0, 0, m1, M0};
  J1.total = J2.total = 2 * M0;
  const unsigned gb = (unsigned)((2 * M0 + 255) / 256);
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J1, x, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J1, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J2, dY, tw, out);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  return BIE_OK;
}

// fixed-order sum over a single CTA (blockDim.x a multiple of 32, <= 1024)
__device__ double cta_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;   // every thread
}

// eq. CS:th: C, S, P0 theta, s_alpha; dz = s e^{i theta}; f = [s cos theta - 1 | s sin theta]
// par = {P0 theta, s_alpha}
__global__ void k_hls_a(int M0, const double* __restrict__ Pth, double2* __restrict__ dz,
                        double* __restrict__ f, double* __restrict__ par) {
  __shared__ double red[32];
  double cs = 0.0, sn = 0.0;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) {
    double s1, c1;
    sincos(Pth[m], &s1, &c1);
    cs += c1;
    sn += s1;
  }
  const double C = cta_sum(cs, red) / (double)M0;
  const double S = cta_sum(sn, red) / (double)M0;
  const double p0 = atan2(-S, C);
  const double sa = 1.0 / sqrt(C * C + S * S);
  for (int m = threadIdx.x; m < M0; m += blockDim.x) {
    double s1, c1;
    sincos(Pth[m] + p0, &s1, &c1);
    dz[m] = make_double2(sa * c1, sa * s1);
    f[m] = sa * c1 - 1.0;
    f[M0 + m] = sa * s1;
  }
  if (threadIdx.x == 0) {
    par[0] = p0;
    par[1] = sa;
  }
}

// eq. xi:eta:recon from the antiderivatives A = [xi_aux | eta_aux] (x M_0 in .x),
// theta_alpha in Ta (.x / M_0): zeta, zeta' (already in dz), zeta'' = i theta_alpha zeta'
__global__ void k_hls_b(int M0, const double2* __restrict__ A, const double2* __restrict__ Ta,
                        const double2* __restrict__ dzs, double2* __restrict__ z,
                        double2* __restrict__ dz, double2* __restrict__ d2z) {
  __shared__ double red[32];
  const double inv = 1.0 / (double)M0;
  double acc = 0.0;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) acc += A[M0 + m].x * inv * dzs[m].x;
  const double mean = cta_sum(acc, red) * inv;   // P0[eta_aux xi_alpha]
  const double xi0 = A[0].x * inv;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) {
    const double alpha = (2.0 * M_PI) * (double)m / (double)M0;
    const double2 w = dzs[m];
    const double ta = Ta[m].x * inv;
    z[m] = make_double2(alpha + A[m].x * inv - xi0, A[M0 + m].x * inv - mean);
    dz[m] = w;
    d2z[m] = make_double2(-ta * w.y, ta * w.x);
  }
}

// w = [U | theta_alpha U - P0[theta_alpha U]]
__global__ void k_hls_q(int M0, const double* __restrict__ U, const double2* __restrict__ Ta,
                        double* __restrict__ w) {
  __shared__ double red[32];
  const double inv = 1.0 / (double)M0;
  double acc = 0.0;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) acc += Ta[m].x * inv * U[m];
  const double mean = cta_sum(acc, red) * inv;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) {
    w[m] = U[m];
    w[M0 + m] = Ta[m].x * inv * U[m] - mean;
  }
}

// V = V_aux - V_aux(0) + U(0) eta_alpha(0)/xi_alpha(0); (P theta)_t = P[(U_alpha + V theta_alpha)/s];
// phi~_t by eq. phitileq (C = 0); UV = [U_alpha | V_aux] (x M_0 in .x), Tp = [theta_alpha | phi~_alpha]
__global__ void k_hls_rhs(int M0, FlowParams F, const double2* __restrict__ z,
                          const double2* __restrict__ dz, const double* __restrict__ U,
                          const double2* __restrict__ UV, const double2* __restrict__ Tp,
                          const double* __restrict__ par, double tau, double g,
                          double* __restrict__ ydot) {
  __shared__ double red[32];
  const double inv = 1.0 / (double)M0;
  const double sa = par[1];
  const double V0 = U[0] * dz[0].y / dz[0].x - UV[M0].x * inv;
  double acc = 0.0;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) {
    const double V = UV[M0 + m].x * inv + V0;
    const double tt = (UV[m].x * inv + V * Tp[m].x * inv) / sa;
    ydot[m] = tt;
    acc += tt;
  }
  const double mean = cta_sum(acc, red) * inv;
  for (int m = threadIdx.x; m < M0; m += blockDim.x) {
    ydot[m] -= mean;
    const double V = UV[M0 + m].x * inv + V0;
    const double2 zp = dz[m];
    const double u = U[m];
    const double2 dP = dphi_mv(F, z[m]);
    const double dphimv_dn = (-dP.x * zp.y - dP.y * zp.x) / sa;
    const double phit_a = Tp[M0 + m].x * inv;
    const double phi_a = phit_a + (dP.x * zp.x - dP.y * zp.y);
    const double grad2 = (phi_a / sa) * (phi_a / sa) + u * u;
    const double theta_a = Tp[m].x * inv;
    ydot[M0 + m] = (phit_a / sa) * V + (u - dphimv_dn) * u - 0.5 * grad2 - g * z[m].y +
                   tau * theta_a / sa;
  }
}

// the HLS curve of P theta written into the context's surface nodes; Tp gets
// [theta_alpha | phi~_alpha] for y = [P theta | phi~]
bie_status hls_surface(bie_ctx* c, const double* y, double2* Tp, double* par) {
  const int M0 = c->M[0];
  double2 *dzs, *A;
  double* f;
  BIE_GET(c, double2, "hls_dz", M0, dzs);
  BIE_GET(c, double2, "hls_A", 2 * (size_t)M0, A);
  BIE_GET(c, double, "hls_f", 2 * (size_t)M0, f);
  double2 *z, *dz, *d2z;
  BIE_GET(c, double2, "zeta", c->N, z);
  BIE_GET(c, double2, "dzeta", c->N, dz);
  BIE_GET(c, double2, "d2zeta", c->N, d2z);
  bie_status s = dft_pair(c, y, 1, 1, Tp);
  if (s != BIE_OK) return s;
  k_hls_a<<<1, 1024, 0, c->stream>>>(M0, y, dzs, f, par);
  BIE_LAUNCH_CHECK(c, "k_hls_a");
  s = dft_pair(c, f, 7, 7, A);
  if (s != BIE_OK) return s;
  k_hls_b<<<1, 1024, 0, c->stream>>>(M0, A, Tp, dzs, z, dz, d2z);
  BIE_LAUNCH_CHECK(c, "k_hls_b");
  return geometry_refresh(c);
}

struct StageBufs {
  double *omega, *U, *psi;
};

// y = [eta | phi~] -> ydot = [eta_t | phi~_t]; the context is left holding the
// graph surface of eta, assembled, with omega, U, psi of the solve in sb.
bie_status graph_stage(bie_ctx* c, const double* y, double* ydot, int precision,
                       const bie_solve_opts* o, double tau, double g, const StageBufs& sb,
                       bie_evolve_info* info) {
  BIE_NVTX("graph_stage");
  const int M0 = c->M[0];
  double2* X2;
  BIE_GET(c, double2, "ev_X2", 3 * (size_t)M0, X2);
  bie_status s = graph_derivs(c, y, X2);
  if (s != BIE_OK) return s;
  double2 *z, *dz, *d2z;
  BIE_GET(c, double2, "zeta", c->N, z);
  BIE_GET(c, double2, "dzeta", c->N, dz);
  BIE_GET(c, double2, "d2zeta", c->N, d2z);
  k_graph_surface<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, y, X2, z, dz, d2z);
  BIE_LAUNCH_CHECK(c, "k_graph_surface");
  s = geometry_refresh(c);
  if (s != BIE_OK) return s;
  s = bie_assemble(c, precision);
  if (s != BIE_OK) return s;
  bie_solve_info si;
  memset(&si, 0, sizeof(si));
  s = solve_run(c, y + M0, sb.omega, sb.U, sb.psi, o, &si);
  if (info) {
    info->solves += 1;
    info->gmres_iters += si.iters;
    info->max_rel_resid = fmax(info->max_rel_resid, si.rel_resid);
  }
  if (s != BIE_OK) return s;
  k_graph_rhs<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, make_flow(c), z, dz, d2z, sb.U, X2, y,
                                                       tau, g, ydot);
  BIE_LAUNCH_CHECK(c, "k_graph_rhs");
  return BIE_OK;
}

// y = [P theta | phi~] -> ydot = [(P theta)_t | phi~_t] (HLS formulation)
bie_status hls_stage(bie_ctx* c, const double* y, double* ydot, int precision,
                     const bie_solve_opts* o, double tau, double g, const StageBufs& sb,
                     bie_evolve_info* info) {
  BIE_NVTX("hls_stage");
  const int M0 = c->M[0];
  double2 *Tp, *UV;
  double *par, *w;
  BIE_GET(c, double2, "hls_Tp", 2 * (size_t)M0, Tp);
  BIE_GET(c, double2, "hls_UV", 2 * (size_t)M0, UV);
  BIE_GET(c, double, "hls_par", 4, par);
  BIE_GET(c, double, "hls_w", 2 * (size_t)M0, w);
  bie_status s = hls_surface(c, y, Tp, par);
  if (s != BIE_OK) return s;
  s = bie_assemble(c, precision);
  if (s != BIE_OK) return s;
  bie_solve_info si;
  memset(&si, 0, sizeof(si));
  s = solve_run(c, y + M0, sb.omega, sb.U, sb.psi, o, &si);
  if (info) {
    info->solves += 1;
    info->gmres_iters += si.iters;
    info->max_rel_resid = fmax(info->max_rel_resid, si.rel_resid);
  }
  if (s != BIE_OK) return s;
  k_hls_q<<<1, 1024, 0, c->stream>>>(M0, sb.U, Tp, w);
  BIE_LAUNCH_CHECK(c, "k_hls_q");
  s = dft_pair(c, w, 1, 7, UV);   // [U_alpha | antiderivative of theta_alpha U - mean]
  if (s != BIE_OK) return s;
  bool oom = false;
  const double2* z = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * c->N, &oom);
  const double2* dz = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * c->N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "hls: nodes");
  k_hls_rhs<<<1, 1024, 0, c->stream>>>(M0, make_flow(c), z, dz, sb.U, UV, Tp, par, tau, g, ydot);
  BIE_LAUNCH_CHECK(c, "k_hls_rhs");
  return BIE_OK;
}

typedef bie_status (*StageFn)(bie_ctx*, const double*, double*, int, const bie_solve_opts*,
                              double, double, const StageBufs&, bie_evolve_info*);

// ---------------------------------------------------------------------------
// vortex-sheet formulation: gamma_0,t (Sec. 4, eqs. gam:t:final, gam:t:aux)
// ---------------------------------------------------------------------------

// per-boundary forward (mode 0) and inverse (mode `mode`) DFT of a vector over all N nodes
bie_status dft_blocks(bie_ctx* c, const double* x, int mode, double2* out) {
  const int N = c->N;
  double2 *dY, *dX1;
  BIE_GET(c, double2, "db_Y", N, dY);
  BIE_GET(c, double2, "db_X1", N, dX1);
  bool oom = false;
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "dft: twiddles");
  DftJobs J1, J2;
  memset(&J1, 0, sizeof(J1));
  memset(&J2, 0, sizeof(J2));
  for (int k = 0; k < c->nb; ++k) {
    const int M = c->M[k], M1 = c->fft_m1[k], o = c->off[k];
    J1.j[J1.n++] = DftJob{M, M1, M / M1, o, o, o, 0, o};
    J2.j[J2.n++] = DftJob{M, M1, M / M1, o, o, o, mode, o};
  }
  J1.total = J2.total = N;
  const unsigned gb = (unsigned)((N + 255) / 256);
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J1, x, nullptr, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J1, dY, tw, dX1);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  k_dft_a<<<dft_grid(gb), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
  BIE_LAUNCH_CHECK(c, "k_dft_a");
  k_dft_b<<<dft_grid(gb), 256, 0, c->stream>>>(J2, dY, tw, out);
  BIE_LAUNCH_CHECK(c, "k_dft_b");
  return BIE_OK;
}

// out[m] = sign_k X[m].x / M_k with sign -1 on block 0 when neg0, -1 off block 0 when negs
__global__ void k_take_blocks(Blocks B, const double2* __restrict__ X, int neg0, int negs,
                              double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= B.N) return;
  int k = 0;
  while (k + 1 < B.nb && m >= B.off[k + 1]) ++k;
  double v = X[m].x / (double)B.M[k];
  if ((k == 0 && neg0) || (k > 0 && negs)) v = -v;
  out[m] = v;
}

__global__ void k_gt_sgn(int N, int M0, float* __restrict__ sgn) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < N) sgn[m] = (m < M0) ? 0.5f : -0.5f;
}

// x = [V gamma_0/s | U gamma_0/s], V = eta_alpha U (graph formulation)
__global__ void k_vs_x(int M0, const double2* __restrict__ dz, const double* __restrict__ U,
                       const double* __restrict__ gamma0, double* __restrict__ x) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M0) return;
  const double2 zp = dz[m];
  const double s = sqrt(zp.x * zp.x + zp.y * zp.y);
  const double V = (zp.y / zp.x) * U[m];
  x[m] = V * gamma0[m] / s;
  x[M0 + m] = U[m] * gamma0[m] / s;
}

// S1[m], S2[m] = (1/M_0) sum_l zeta_0'(beta_l)/2 cot((zeta_0(beta_l) - zeta(alpha_m))/2) x_l
// for x = x1, x2, every node m; on the surface the real part is regularised by
// -1/2 cot((beta_l - alpha_m)/2) and the diagonal is zeta''/(2 zeta').  One
// 128-thread CTA per m, double-float pair kernel of the assembly (xd = x as
// double-float); the diagonal term in FP64.
__global__ void __launch_bounds__(PS_THREADS)
    k_surface_sums(int N, int M0, PairNodes nd, const double2* __restrict__ dz,
                   const double2* __restrict__ d2z, const double* __restrict__ x,
                   const float2* __restrict__ xd, double2* __restrict__ S1,
                   double2* __restrict__ S2) {
  __shared__ dfl sh[PS_THREADS / 32];
  const int m = blockIdx.x;
  const cx<dfl> Qm = ld_cx(nd.nQ, m);
  const float4 qc = nd.nPQc[m];
  const float2 Qcm = make_float2(qc.z, qc.w);
  const double2 zm = nd.z64[m];
  const bool surf = m < M0;
  dfl a1r = {0.f, 0.f}, a1i = a1r, a2r = a1r, a2i = a1r;
  for (int l = threadIdx.x; l < M0; l += PS_THREADS) {
    if (surf && l == m) continue;
    const float4 pc = nd.nPQc[l];
    const cx<dfl> G = half_cot_pair<dfl>(ld_cx(nd.nP, l), Qm, make_float2(pc.x, pc.y), Qcm,
                                         nd.z64[l], zm, 0.01f);
    const cx<dfl> Zl = ld_cx(nd.nZp, l);
    dfl tr = cre(Zl, G);
    const dfl ti = cim(Zl, G);
    if (surf) {
      const float2 t = nd.Ttab[(l - m + M0) % M0];
      tr = tr - dfl{t.x, t.y};
    }
    const dfl x1 = {xd[l].x, xd[l].y}, x2 = {xd[M0 + l].x, xd[M0 + l].y};
    a1r = a1r + tr * x1;
    a1i = a1i + ti * x1;
    a2r = a2r + tr * x2;
    a2i = a2i + ti * x2;
  }
  a1r = df_cta_sum(a1r, sh);
  a1i = df_cta_sum(a1i, sh);
  a2r = df_cta_sum(a2r, sh);
  a2i = df_cta_sum(a2i, sh);
  if (threadIdx.x == 0) {
    double s1r = (double)a1r.hi + (double)a1r.lo, s1i = (double)a1i.hi + (double)a1i.lo;
    double s2r = (double)a2r.hi + (double)a2r.lo, s2i = (double)a2i.hi + (double)a2i.lo;
    if (surf) {
      const double2 a = d2z[m], b = dz[m];
      const double n2 = b.x * b.x + b.y * b.y;
      const double tr = 0.5 * (a.x * b.x + a.y * b.y) / n2;
      const double ti = 0.5 * (a.y * b.x - a.x * b.y) / n2;
      s1r += tr * x[m];
      s1i += ti * x[m];
      s2r += tr * x[M0 + m];
      s2i += ti * x[M0 + m];
    }
    const double inv = 1.0 / (double)M0;
    S1[m] = make_double2(s1r * inv, s1i * inv);
    S2[m] = make_double2(s2r * inv, s2i * inv);
  }
}

// R = [Q on the surface | F_k0 gamma_0 on the solids] (eq. gam:t:final bracket, eq. Fk:from:UV)
__global__ void k_vs_R(int N, int M0, const double2* __restrict__ z, const double2* __restrict__ dz,
                       const double2* __restrict__ d2z, const double* __restrict__ U,
                       const double* __restrict__ gamma0, const double* __restrict__ f,
                       const double2* __restrict__ S1, const double2* __restrict__ S2,
                       const double2* __restrict__ Hx, double tau, double g,
                       double* __restrict__ R) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  if (m >= M0) {
    R[m] = S1[m].x - S2[m].y;
    return;
  }
  const double2 zp = dz[m];
  const double s2 = zp.x * zp.x + zp.y * zp.y, s = sqrt(s2);
  const double tx = zp.x / s, ty = zp.y / s;
  const double g0 = gamma0[m];
  const double Wx = f[2 * m] - g0 / (2.0 * s) * tx;        // f = u - i v
  const double Wy = -f[2 * m + 1] - g0 / (2.0 * s) * ty;
  const double V = (zp.y / zp.x) * U[m];
  const double F00 = -0.5 * Hx[M0 + m].x / (double)M0 + S1[m].y + S2[m].x;
  const double ea = zp.y;
  const double theta_a = d2z[m].y / (1.0 + ea * ea);
  R[m] = -0.5 * (Wx * Wx + Wy * Wy) + (V - (Wx * tx + Wy * ty)) * g0 / (2.0 * s) -
         g0 * g0 / (8.0 * s2) + tau * theta_a / s - g * z[m].y - F00;
}

__global__ void k_vs_ydot(int M0, const double2* __restrict__ dz, const double* __restrict__ U,
                          const double* __restrict__ gt, double* __restrict__ ydot) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M0) return;
  const double2 zp = dz[m];
  ydot[m] = sqrt(zp.x * zp.x + zp.y * zp.y) * U[m];
  ydot[M0 + m] = gt[m];
}

// private context holding the gamma_t operator S^T W + diag(+1/2 surface, -1/2 solids)
// (transposed kernels, no -E_k term) on the current geometry
bie_status gt_prepare(bie_ctx* c, int precision) {
  if (c->gt && c->gt_version == c->geom_version && c->gt_precision == precision) return BIE_OK;
  if (!c->gt) {
    bie_ctx* s = nullptr;
    bie_status st = bie_create(&s, c->device, c->stream);
    if (st != BIE_OK) return ctx_fail(c, st, "gamma_t: sub-context");
    c->gt = s;
  }
  bie_ctx* s = c->gt;
  s->stream = c->stream;
  s->nb = c->nb;
  s->N = c->N;
  s->ld = c->ld;
  partition_update(s);   // a private context holds every row
  for (int k = 0; k < BIE_MAXB; ++k) {
    s->M[k] = c->M[k];
    s->fft_m1[k] = c->fft_m1[k];
    s->zc[k] = c->zc[k];
  }
  for (int k = 0; k <= BIE_MAXB; ++k) s->off[k] = c->off[k];
  s->assembled = false;
  s->transposed = false;
  s->asm_noE = true;
  const size_t nbytes = sizeof(double2) * (size_t)s->N;
  double2 *z, *dz, *d2z;
  BIE_GET(s, double2, "zeta", s->N, z);
  BIE_GET(s, double2, "dzeta", s->N, dz);
  BIE_GET(s, double2, "d2zeta", s->N, d2z);
  bool oom = false;
  const double2* cz = (const double2*)ctx_buf(c, "zeta", nbytes, &oom);
  const double2* cdz = (const double2*)ctx_buf(c, "dzeta", nbytes, &oom);
  const double2* cd2z = (const double2*)ctx_buf(c, "d2zeta", nbytes, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "gamma_t: node buffers");
  BIE_CUDA_TRY(c, cudaMemcpyAsync(z, cz, nbytes, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(dz, cdz, nbytes, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(d2z, cd2z, nbytes, cudaMemcpyDeviceToDevice, c->stream));
  bie_status st = geometry_prep(s);
  if (st != BIE_OK) return ctx_fail(c, st, "gamma_t: " + s->err);
  s->have_geom = true;
  float* sgn;
  BIE_GET(s, float, "sgn", s->ld, sgn);
  k_gt_sgn<<<(unsigned)((s->N + 255) / 256), 256, 0, c->stream>>>(s->N, c->M[0], sgn);
  BIE_LAUNCH_CHECK(c, "k_gt_sgn");
  s->solid_version = c->solid_version;   // same solids: their tile pairs are kept
  st = asm_run(s, precision, 1);
  if (st != BIE_OK) return ctx_fail(c, st, "gamma_t: " + s->err);
  s->precision = precision;
  s->assembled = true;
  s->transposed = true;
  c->gt_version = c->geom_version;
  c->gt_precision = precision;
  return BIE_OK;
}

// y = [eta | gamma_0] -> ydot = [eta_t | gamma_0,t] (graph formulation, vortex sheet)
bie_status vs_stage(bie_ctx* c, const double* y, double* ydot, int precision,
                    const bie_solve_opts* o, double tau, double g, const StageBufs& sb,
                    bie_evolve_info* info) {
  BIE_NVTX("vortex_sheet_stage");
  const int M0 = c->M[0], N = c->N;
  double2 *X2, *Xb, *Hx, *S1, *S2;
  double *gam, *f, *x, *R, *r, *gtx;
  BIE_GET(c, double2, "ev_X2", 3 * (size_t)M0, X2);
  BIE_GET(c, double2, "vs_Xb", N, Xb);
  BIE_GET(c, double2, "vs_Hx", 2 * (size_t)M0, Hx);
  BIE_GET(c, double2, "vs_S1", N, S1);
  BIE_GET(c, double2, "vs_S2", N, S2);
  BIE_GET(c, double, "vs_gam", N, gam);
  BIE_GET(c, double, "vs_f", 2 * (size_t)N, f);
  BIE_GET(c, double, "vs_x", 2 * (size_t)M0, x);
  BIE_GET(c, double, "vs_R", N, R);
  BIE_GET(c, double, "vs_r", N, r);
  BIE_GET(c, double, "vs_gt", N, gtx);
  // surface from eta
  bie_status s = graph_derivs(c, y, X2);
  if (s != BIE_OK) return s;
  double2 *z, *dz, *d2z;
  BIE_GET(c, double2, "zeta", N, z);
  BIE_GET(c, double2, "dzeta", N, dz);
  BIE_GET(c, double2, "d2zeta", N, d2z);
  k_graph_surface<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, y, X2, z, dz, d2z);
  BIE_LAUNCH_CHECK(c, "k_graph_surface");
  s = geometry_refresh(c);
  if (s != BIE_OK) return s;
  // U and gamma_1..N (eq. lin:sys2, eq. U:from:gam:j)
  bie_solve_info si;
  memset(&si, 0, sizeof(si));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(gam, y + M0, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  s = bie_vs_normal_velocity(c, y + M0, sb.U, gam + M0, precision, o, &si);
  if (info) {
    info->solves += 1;
    info->gmres_iters += si.iters;
    info->max_rel_resid = fmax(info->max_rel_resid, si.rel_resid);
  }
  if (s != BIE_OK) return s;
  // omega_0 = -d^-1 gamma_0, omega_j = d^-1 gamma_j; grad phi on the boundaries
  const Blocks B = make_blocks(c);
  const unsigned gN = (unsigned)((N + 255) / 256);
  s = dft_blocks(c, gam, 7, Xb);
  if (s != BIE_OK) return s;
  k_take_blocks<<<gN, 256, 0, c->stream>>>(B, Xb, 1, 0, sb.omega);
  BIE_LAUNCH_CHECK(c, "k_take_blocks");
  s = bie_boundary_velocity(c, sb.omega, f);
  if (s != BIE_OK) return s;
  // F_00 and F_k0 (eq. Fk:from:UV): Table 1 sums over the surface and H(U gamma_0/s)
  k_vs_x<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, dz, sb.U, y + M0, x);
  BIE_LAUNCH_CHECK(c, "k_vs_x");
  s = dft_pair(c, x, 1, 4, Hx);
  if (s != BIE_OK) return s;
  bool oom = false;
  PairNodes nd;
  nd.nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  nd.nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  nd.nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  nd.nZp = (const float4*)ctx_buf(c, "nZp", sizeof(float4) * N, &oom);
  nd.Ttab = (const float2*)ctx_buf(c, "Ttab", sizeof(float2) * M0, &oom);
  nd.z64 = z;
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "gamma_t: node tables");
  float2* xd;
  BIE_GET(c, float2, "vs_xd", 2 * (size_t)M0, xd);
  k_to_df<<<(2 * M0 + 255) / 256, 256, 0, c->stream>>>(B, 2 * M0, x, 0, xd);
  BIE_LAUNCH_CHECK(c, "k_to_df");
  k_surface_sums<<<N, PS_THREADS, 0, c->stream>>>(N, M0, nd, dz, d2z, x, xd, S1, S2);
  BIE_LAUNCH_CHECK(c, "k_surface_sums");
  k_vs_R<<<gN, 256, 0, c->stream>>>(N, M0, z, dz, d2z, sb.U, y + M0, f, S1, S2, Hx, tau, g, R);
  BIE_LAUNCH_CHECK(c, "k_vs_R");
  // right-hand sides: d_alpha of the bracket (surface), -d_alpha F_k0 gamma_0 (solids)
  s = dft_blocks(c, R, 1, Xb);
  if (s != BIE_OK) return s;
  k_take_blocks<<<gN, 256, 0, c->stream>>>(B, Xb, 0, 1, r);
  BIE_LAUNCH_CHECK(c, "k_take_blocks");
  // the gamma_t system on its private context
  s = gt_prepare(c, precision);
  if (s != BIE_OK) return s;
  memset(&si, 0, sizeof(si));
  s = solve_system(c->gt, o, gtx, r, &si);
  if (info) {
    info->solves += 1;
    info->gmres_iters += si.iters;
    info->max_rel_resid = fmax(info->max_rel_resid, si.rel_resid);
  }
  if (s != BIE_OK) return ctx_fail(c, s, "gamma_t solve: " + c->gt->err);
  k_vs_ydot<<<(M0 + 255) / 256, 256, 0, c->stream>>>(M0, dz, sb.U, gtx, ydot);
  BIE_LAUNCH_CHECK(c, "k_vs_ydot");
  return BIE_OK;
}



bie_status stage_bufs(bie_ctx* c, StageBufs& sb) {
  BIE_GET(c, double, "ev_omega", c->N, sb.omega);
  BIE_GET(c, double, "ev_U", c->M[0], sb.U);
  BIE_GET(c, double, "ev_psi", BIE_MAXB, sb.psi);
  return BIE_OK;
}

// With a separation limit set, a step starts only while every node stays at
// least that many local node spacings away from the other boundaries.
bie_status separation_guard(bie_ctx* c, const char* who, int step) {
  if (!(c->min_sep > 0.0)) return BIE_OK;
  double r = 0.0;
  int node = 0;
  bie_status s = separation_run(c, &r, &node);
  if (s != BIE_OK) return s;
  if (r < c->min_sep)
    return ctx_fail(c, BIE_ERR_GEOM, std::string(who) + ": before step " + std::to_string(step) +
                                         " node " + std::to_string(node) + " is " +
                                         std::to_string(r) + " node spacings from another boundary");
  return BIE_OK;
}

bie_status evolve_checks(bie_ctx* c, int precision, const bie_solve_opts* opts, bie_solve_opts* o,
                         double tau, double g) {
  if (!c->have_geom || !c->have_flow)
    return ctx_fail(c, BIE_ERR_STATE, "graph evolution: set geometry and flow first");
  if (precision < BIE_FP64 || precision > BIE_FP16_IR)
    return ctx_fail(c, BIE_ERR_ARG, "graph evolution: bad precision");
  if (!std::isfinite(tau) || !std::isfinite(g))
    return ctx_fail(c, BIE_ERR_ARG, "graph evolution: tau and g must be finite");
  bie_default_opts(o);
  if (opts) *o = *opts;
  if (!(o->rtol > 0.0) || o->restart < 1 || o->restart > 1000 || o->max_cycles < 1)
    return ctx_fail(c, BIE_ERR_ARG, "graph evolution: bad options");
  // the first solve starts from zero; the drivers then start every solve
  // from the previous stage's solution (omega, and gamma for the vortex sheet)
  o->x0 = 0;
  return BIE_OK;
}

bie_status one_stage(bie_ctx* c, StageFn stage, const char* who, const double* eta_dev,
                     const double* phit_dev, double tau, double g, int precision,
                     const bie_solve_opts* opts, double* eta_t_dev, double* phit_t_dev,
                     double* omega_dev, double* U_dev) {
  if (!c) return BIE_ERR_ARG;
  if (!eta_dev || !phit_dev || !eta_t_dev || !phit_t_dev)
    return ctx_fail(c, BIE_ERR_ARG, std::string(who) + ": null pointer");
  bie_solve_opts o;
  bie_status s = evolve_checks(c, precision, opts, &o, tau, g);
  if (s != BIE_OK) return s;
  cudaSetDevice(c->device);
  const int M0 = c->M[0];
  double *y, *yd;
  BIE_GET(c, double, "ev_y", 2 * (size_t)M0, y);
  BIE_GET(c, double, "ev_k1", 2 * (size_t)M0, yd);
  StageBufs sb;
  s = stage_bufs(c, sb);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y, eta_dev, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y + M0, phit_dev, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  s = stage(c, y, yd, precision, &o, tau, g, sb, nullptr);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(eta_t_dev, yd, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(phit_t_dev, yd + M0, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  if (omega_dev)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(omega_dev, sb.omega, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  if (U_dev)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(U_dev, sb.U, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

bie_status rk4_drive(bie_ctx* c, StageFn stage, const char* who, double* eta_dev,
                     double* phit_dev, double dt, int nsteps, double tau, double g, int filter,
                     int precision, const bie_solve_opts* opts, double* energies_host,
                     bie_evolve_info* info) {
  if (!c) return BIE_ERR_ARG;
  if (!eta_dev || !phit_dev) return ctx_fail(c, BIE_ERR_ARG, std::string(who) + ": null pointer");
  if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt))
    return ctx_fail(c, BIE_ERR_ARG, std::string(who) + ": nsteps >= 0 and dt > 0 required");
  bie_solve_opts o;
  bie_status s = evolve_checks(c, precision, opts, &o, tau, g);
  if (s != BIE_OK) return s;
  cudaSetDevice(c->device);
  if (info) memset(info, 0, sizeof(*info));
  const int M0 = c->M[0], n2 = 2 * M0;
  double *y, *yt, *k1, *k2, *k3, *k4, *E = nullptr;
  BIE_GET(c, double, "ev_y", n2, y);
  BIE_GET(c, double, "ev_yt", n2, yt);
  BIE_GET(c, double, "ev_k1", n2, k1);
  BIE_GET(c, double, "ev_k2", n2, k2);
  BIE_GET(c, double, "ev_k3", n2, k3);
  BIE_GET(c, double, "ev_k4", n2, k4);
  if (energies_host) BIE_GET(c, double, "ev_E", (size_t)nsteps + 1, E);
  StageBufs sb;
  s = stage_bufs(c, sb);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y, eta_dev, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y + M0, phit_dev, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  const unsigned gb = (unsigned)((n2 + 255) / 256);
#define EV_TRY(x)            \
  do {                       \
    s = (x);                 \
    if (s != BIE_OK) return s; \
  } while (0)
  for (int n = 0; n < nsteps; ++n) {
    EV_TRY(stage(c, y, k1, precision, &o, tau, g, sb, info));
    o.x0 = 1;
    EV_TRY(separation_guard(c, who, n));
    if (E) EV_TRY(energy_run(c, y + M0, sb.omega, tau, g, E + n));
    k_axpy2<<<gb, 256, 0, c->stream>>>(n2, y, 0.5 * dt, k1, yt);
    BIE_LAUNCH_CHECK(c, "k_axpy2");
    EV_TRY(stage(c, yt, k2, precision, &o, tau, g, sb, info));
    k_axpy2<<<gb, 256, 0, c->stream>>>(n2, y, 0.5 * dt, k2, yt);
    BIE_LAUNCH_CHECK(c, "k_axpy2");
    EV_TRY(stage(c, yt, k3, precision, &o, tau, g, sb, info));
    k_axpy2<<<gb, 256, 0, c->stream>>>(n2, y, dt, k3, yt);
    BIE_LAUNCH_CHECK(c, "k_axpy2");
    EV_TRY(stage(c, yt, k4, precision, &o, tau, g, sb, info));
    k_rk4_final<<<gb, 256, 0, c->stream>>>(n2, dt, k1, k2, k3, k4, y);
    BIE_LAUNCH_CHECK(c, "k_rk4_final");
    if (filter) EV_TRY(filter_run(c, y, 2));
    if (info) info->steps += 1;
  }
  if (E) {  // energy of the final state needs its own solve
    EV_TRY(stage(c, y, k1, precision, &o, tau, g, sb, info));
    EV_TRY(energy_run(c, y + M0, sb.omega, tau, g, E + nsteps));
  }
#undef EV_TRY
  BIE_CUDA_TRY(c, cudaMemcpyAsync(eta_dev, y, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(phit_dev, y + M0, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  if (E)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(energies_host, E, sizeof(double) * ((size_t)nsteps + 1),
                                    cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

// One Gragg-Bulirsch-Stoer step of size h: explicit midpoint rule with n =
// 2, 4, 6, 8 substeps (z_1 = y + (h/n) f(y), z_{m+1} = z_{m-1} + 2 (h/n) f(z_m))
// and Aitken-Neville extrapolation in (h/n)^2: order 8.  f0 = f(y) is given.
bie_status gbs8_step(bie_ctx* c, StageFn stage, double* y, const double* f0, double h,
                     int precision, const bie_solve_opts* o, double tau, double g,
                     const StageBufs& sb, bie_evolve_info* info) {
  BIE_NVTX("gbs8_step");
  static const int kSeq[4] = {2, 4, 6, 8};
  const int M0 = c->M[0], n2 = 2 * M0;
  double *A, *B, *C, *fz, *Tp[4], *Tc[4];
  BIE_GET(c, double, "gb_A", n2, A);
  BIE_GET(c, double, "gb_B", n2, B);
  BIE_GET(c, double, "gb_C", n2, C);
  BIE_GET(c, double, "gb_fz", n2, fz);
  const char* np[4] = {"gb_P0", "gb_P1", "gb_P2", "gb_P3"};
  const char* nc[4] = {"gb_C0", "gb_C1", "gb_C2", "gb_C3"};
  for (int k = 0; k < 4; ++k) {
    BIE_GET(c, double, np[k], n2, Tp[k]);
    BIE_GET(c, double, nc[k], n2, Tc[k]);
  }
  const unsigned gb = (unsigned)((n2 + 255) / 256);
  const size_t bytes = sizeof(double) * n2;
  for (int j = 0; j < 4; ++j) {
    const int n = kSeq[j];
    const double hs = h / n;
    double *zm = A, *z = B, *zn = C;
    BIE_CUDA_TRY(c, cudaMemcpyAsync(zm, y, bytes, cudaMemcpyDeviceToDevice, c->stream));
    k_axpy2<<<gb, 256, 0, c->stream>>>(n2, y, hs, f0, z);
    BIE_LAUNCH_CHECK(c, "k_axpy2");
    for (int m = 1; m < n; ++m) {
      bie_status s = stage(c, z, fz, precision, o, tau, g, sb, info);
      if (s != BIE_OK) return s;
      k_axpy2<<<gb, 256, 0, c->stream>>>(n2, zm, 2.0 * hs, fz, zn);
      BIE_LAUNCH_CHECK(c, "k_axpy2");
      double* t = zm;
      zm = z;
      z = zn;
      zn = t;
    }
    BIE_CUDA_TRY(c, cudaMemcpyAsync(Tc[0], z, bytes, cudaMemcpyDeviceToDevice, c->stream));
    for (int k = 1; k <= j; ++k) {
      const double r = (double)n / (double)kSeq[j - k];
      k_extrap<<<gb, 256, 0, c->stream>>>(n2, Tc[k - 1], Tp[k - 1], 1.0 / (r * r - 1.0), Tc[k]);
      BIE_LAUNCH_CHECK(c, "k_extrap");
    }
    for (int k = 0; k < 4; ++k) {
      double* t = Tp[k];
      Tp[k] = Tc[k];
      Tc[k] = t;
    }
  }
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y, Tp[3], bytes, cudaMemcpyDeviceToDevice, c->stream));
  return BIE_OK;
}

// The eighth-order Dormand-Prince scheme of Sec. 7.1 (the 12-stage method
// DOP853 of Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.10): its
// published Butcher tableau, rows a_i1..a_i,i-1 (zeros included).  The
// stages are autonomous here, so the abscissae c_i do not enter.
static const double kDP8A[12][11] = {
    {0},
    {5.26001519587677318785587544488e-2},
    {1.97250569845378994544595329183e-2, 5.91751709536136983633785987549e-2},
    {2.95875854768068491816892993775e-2, 0.0, 8.87627564304205475450678981324e-2},
    {2.41365134159266685502369798665e-1, 0.0, -8.84549479328286085344864962717e-1,
     9.24834003261792003115737966543e-1},
    {3.7037037037037037037037037037e-2, 0.0, 0.0, 1.70828608729473871279604482173e-1,
     1.25467687566822425016691814123e-1},
    {3.7109375e-2, 0.0, 0.0, 1.70252211019544039314978060272e-1, 6.02165389804559606850219397283e-2,
     -1.7578125e-2},
    {3.70920001185047927108779319836e-2, 0.0, 0.0, 1.70383925712239993810214054705e-1,
     1.07262030446373284651809199168e-1, -1.53194377486244017527936158236e-2,
     8.27378916381402288758473766002e-3},
    {6.24110958716075717114429577812e-1, 0.0, 0.0, -3.36089262944694129406857109825e0,
     -8.68219346841726006818189891453e-1, 2.75920996994467083049415600797e1,
     2.01540675504778934086186788979e1, -4.34898841810699588477366255144e1},
    {4.77662536438264365890433908527e-1, 0.0, 0.0, -2.48811461997166764192642586468e0,
     -5.90290826836842996371446475743e-1, 2.12300514481811942347288949897e1,
     1.52792336328824235832596922938e1, -3.32882109689848629194453265587e1,
     -2.03312017085086261358222928593e-2},
    {-9.3714243008598732571704021658e-1, 0.0, 0.0, 5.18637242884406370830023853209e0,
     1.09143734899672957818500254654e0, -8.14978701074692612513997267357e0,
     -1.85200656599969598641566180701e1, 2.27394870993505042818970056734e1,
     2.49360555267965238987089396762e0, -3.0467644718982195003823669022e0},
    {2.27331014751653820792359768449e0, 0.0, 0.0, -1.05344954667372501984066689879e1,
     -2.00087205822486249909675718444e0, -1.79589318631187989172765950534e1,
     2.79488845294199600508499808837e1, -2.85899827713502369474065508674e0,
     -8.87285693353062954433549289258e0, 1.23605671757943030647266201528e1,
     6.43392746015763530355970484046e-1}};
static const double kDP8B[12] = {
    5.42937341165687622380535766363e-2, 0.0, 0.0, 0.0, 0.0, 4.45031289275240888144113950566e0,
    1.89151789931450038304281599044e0, -5.8012039600105847814672114227e0,
    3.1116436695781989440891606237e-1, -1.52160949662516078556178806805e-1,
    2.01365400804030348374776537501e-1, 4.47106157277725905176885569043e-2};

static StageSum stage_sum(double* const* k, const double* w, int n) {
  StageSum S;
  memset(&S, 0, sizeof(S));
  for (int j = 0; j < n; ++j) {
    if (w[j] == 0.0) continue;
    S.k[S.n] = k[j];
    S.w[S.n] = w[j];
    ++S.n;
  }
  return S;
}

// One step of size h: k_1 = f0 = f(y) (given), k_i = f(y + h sum_{j<i} a_ij
// k_j) for i = 2..12 (11 more solves), y <- y + h sum_i b_i k_i.
bie_status dp8_step(bie_ctx* c, StageFn stage, double* y, const double* f0, double h,
                    int precision, const bie_solve_opts* o, double tau, double g,
                    const StageBufs& sb, bie_evolve_info* info) {
  BIE_NVTX("dp8_step");
  const int M0 = c->M[0], n2 = 2 * M0;
  static const char* names[12] = {"dp_k1", "dp_k2", "dp_k3", "dp_k4", "dp_k5", "dp_k6",
                                  "dp_k7", "dp_k8", "dp_k9", "dp_k10", "dp_k11", "dp_k12"};
  double* k[12];
  double* yt;
  k[0] = const_cast<double*>(f0);
  for (int i = 1; i < 12; ++i) BIE_GET(c, double, names[i], n2, k[i]);
  BIE_GET(c, double, "dp_yt", n2, yt);
  const unsigned gb = (unsigned)((n2 + 255) / 256);
  for (int i = 1; i < 12; ++i) {
    k_stage_sum<<<gb, 256, 0, c->stream>>>(n2, y, h, stage_sum(k, kDP8A[i], i), yt);
    BIE_LAUNCH_CHECK(c, "k_stage_sum");
    bie_status s = stage(c, yt, k[i], precision, o, tau, g, sb, info);
    if (s != BIE_OK) return s;
  }
  k_stage_sum<<<gb, 256, 0, c->stream>>>(n2, y, h, stage_sum(k, kDP8B, 12), y);
  BIE_LAUNCH_CHECK(c, "k_stage_sum");
  return BIE_OK;
}

typedef bie_status (*StepFn)(bie_ctx*, StageFn, double*, const double*, double, int,
                             const bie_solve_opts*, double, double, const StageBufs&,
                             bie_evolve_info*);

// Fixed-step driver of a one-step scheme that takes f(y) at the step's start
// (the Gragg-Bulirsch-Stoer or the Dormand-Prince step): the start value also
// feeds the energy monitor.
bie_status step_drive(bie_ctx* c, StageFn stage, StepFn step, const char* who, double* y1_dev,
                      double* phit_dev, double dt, int nsteps, double tau, double g, int filter,
                      int precision, const bie_solve_opts* opts, double* energies_host,
                      bie_evolve_info* info) {
  if (!y1_dev || !phit_dev) return ctx_fail(c, BIE_ERR_ARG, std::string(who) + ": null pointer");
  if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt))
    return ctx_fail(c, BIE_ERR_ARG, std::string(who) + ": nsteps >= 0 and dt > 0 required");
  bie_solve_opts o;
  bie_status s = evolve_checks(c, precision, opts, &o, tau, g);
  if (s != BIE_OK) return s;
  cudaSetDevice(c->device);
  if (info) memset(info, 0, sizeof(*info));
  const int M0 = c->M[0], n2 = 2 * M0;
  double *y, *f0, *E = nullptr;
  BIE_GET(c, double, "ev_y", n2, y);
  BIE_GET(c, double, "ev_k1", n2, f0);
  if (energies_host) BIE_GET(c, double, "ev_E", (size_t)nsteps + 1, E);
  StageBufs sb;
  s = stage_bufs(c, sb);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y, y1_dev, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y + M0, phit_dev, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  for (int n = 0; n <= nsteps; ++n) {
    if (n == nsteps && !E) break;
    s = stage(c, y, f0, precision, &o, tau, g, sb, info);
    if (s != BIE_OK) return s;
    o.x0 = 1;
    if (n < nsteps) {
      s = separation_guard(c, who, n);
      if (s != BIE_OK) return s;
    }
    if (E) {
      s = energy_run(c, y + M0, sb.omega, tau, g, E + n);
      if (s != BIE_OK) return s;
    }
    if (n == nsteps) break;
    s = step(c, stage, y, f0, dt, precision, &o, tau, g, sb, info);
    if (s != BIE_OK) return s;
    if (filter) {
      s = filter_run(c, y, 2);
      if (s != BIE_OK) return s;
    }
    if (info) info->steps += 1;
  }
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y1_dev, y, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(phit_dev, y + M0, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  if (E)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(energies_host, E, sizeof(double) * ((size_t)nsteps + 1),
                                    cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

// Re Phi~ on the solid boundaries from the fluid side: the Plemelj formula
// applied to eq. w123 (Sec. 4: Phi_t - C on the boundaries).  The jump
// (i/2) omega_k of the own boundary is imaginary and drops out; one CTA per
// solid node m (boundary k >= 1), double-float sums over every source l of
//   Im{zeta_l' G} on surface columns, Re{zeta_l' G} on the other solid
//   boundaries, Re{zeta_l' G} - 1/2 cot((beta_l - alpha_m)/2) on boundary k,
// each times omega_l / M_j (G = 1/2 cot((zeta_l - zeta_m)/2)); then the
// diagonal limit Re{zeta''/(2 zeta')} omega_m / M_k and -(1/2) H omega_k (the
// principal value of the subtracted cotangent) in FP64.  Hb holds M_k H omega_k.
__global__ void __launch_bounds__(PS_THREADS)
    k_phi_solid(Blocks B, PairNodes nd, const float2* __restrict__ Tall,
                const double2* __restrict__ dz, const double2* __restrict__ d2z,
                const float2* __restrict__ w, const double* __restrict__ omega,
                const double2* __restrict__ Hb, double2* __restrict__ out) {
  __shared__ dfl sh[PS_THREADS / 32];
  const int M0 = B.M[0], N = B.N;
  const int m = M0 + (int)blockIdx.x;
  int k = 1;
  while (k + 1 < B.nb && m >= B.off[k + 1]) ++k;
  const int ok = B.off[k], Mk = B.M[k];
  const cx<dfl> Qm = ld_cx(nd.nQ, m);
  const float4 qc = nd.nPQc[m];
  const float2 Qcm = make_float2(qc.z, qc.w);
  const double2 zm = nd.z64[m];
  dfl acc = {0.f, 0.f};
  for (int l = threadIdx.x; l < N; l += PS_THREADS) {
    if (l == m) continue;   // diagonal added below in FP64
    const float4 pc = nd.nPQc[l];
    const cx<dfl> G = half_cot_pair<dfl>(ld_cx(nd.nP, l), Qm, make_float2(pc.x, pc.y), Qcm,
                                         nd.z64[l], zm, 0.01f);
    const cx<dfl> Zl = ld_cx(nd.nZp, l);
    const dfl wl = {w[l].x, w[l].y};
    if (l < M0) {
      acc = acc + cim(Zl, G) * wl;
    } else if (l >= ok && l < ok + Mk) {
      int d = l - m;
      if (d < 0) d += Mk;
      const float2 t = Tall[ok + d];
      acc = acc + (cre(Zl, G) - dfl{t.x, t.y}) * wl;
    } else {
      acc = acc + cre(Zl, G) * wl;
    }
  }
  acc = df_cta_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double2 a = d2z[m], b = dz[m];
    const double diag = 0.5 * (a.x * b.x + a.y * b.y) / (b.x * b.x + b.y * b.y);
    out[m].x = (double)acc.hi + (double)acc.lo + diag * omega[m] / (double)Mk -
               0.5 * Hb[m].x / (double)Mk;
  }
}

// The parts of Phi~ on the boundaries that the operator of eq. lin:sys and the
// energy's psi give: Re on Gamma_0 = (A omega)_m, Im on Gamma_0 = psi_0 without
// psi_mv, Im on Gamma_k = (A omega)_m, plus <1_k, omega> on obstacles (the term
// that -E_k removes).
__global__ void k_phi_bound_finish(Blocks B, const double* __restrict__ y,
                                   const double* __restrict__ psi0,
                                   const double* __restrict__ psik, double2* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= B.N) return;
  if (m < B.M[0]) {
    out[m] = make_double2(y[m], psi0[m]);
    return;
  }
  int k = 1;
  while (k + 1 < B.nb && m >= B.off[k + 1]) ++k;
  out[m].y = y[m] + (k >= 2 ? psik[k - 2] : 0.0);
}

}  // namespace

// Phi~ on every boundary node from the fluid side (also used by the target
// evaluation of the potential)
bie_status boundary_potential_run(bie_ctx* c, const double* omega, double2* out) {
  BIE_NVTX("boundary_potential");
  const int N = c->N, M0 = c->M[0];
  double *y, *psi0, *psik;
  double2* Xb;
  float2* wdf;
  BIE_GET(c, double, "bp_y", c->ld, y);
  BIE_GET(c, double, "bp_psi0", M0, psi0);
  BIE_GET(c, double, "bp_psik", BIE_MAXB, psik);
  BIE_GET(c, double2, "bp_Xb", N, Xb);
  BIE_GET(c, float2, "bp_wdf", N, wdf);
  bool oom = false;
  const double2* z = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double2* d2z = (const double2*)ctx_buf(c, "d2zeta", sizeof(double2) * N, &oom);
  const float2* Tall = (const float2*)ctx_buf(c, "Tall", sizeof(float2) * N, &oom);
  PairNodes nd;
  nd.nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  nd.nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  nd.nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  nd.nZp = (const float4*)ctx_buf(c, "nZp", sizeof(float4) * N, &oom);
  nd.Ttab = (const float2*)ctx_buf(c, "Ttab", sizeof(float2) * M0, &oom);
  nd.z64 = z;
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "boundary potential: buffers");
  bie_status s = gemv_apply(c, 1, omega, y);   // full-accuracy storage
  if (s != BIE_OK) return s;
  s = dft_blocks(c, omega, 4, Xb);             // M_k H omega_k on every boundary
  if (s != BIE_OK) return s;
  const Blocks B = make_blocks(c);
  k_to_df<<<(N + 255) / 256, 256, 0, c->stream>>>(B, N, omega, 1, wdf);
  BIE_LAUNCH_CHECK(c, "k_to_df");
  FlowParams F0 = make_flow(c);   // psi_mv left out: Phi~ alone
  F0.V1 = 0.0;
  for (int j = 0; j < BIE_MAXB; ++j) F0.a[j] = 0.0;
  k_psi_surface<<<M0, PS_THREADS, 0, c->stream>>>(B, nd, dz, d2z, wdf, omega, Xb, F0, psi0);
  BIE_LAUNCH_CHECK(c, "k_psi_surface");
  if (N > M0) {
    k_phi_solid<<<N - M0, PS_THREADS, 0, c->stream>>>(B, nd, Tall, dz, d2z, wdf, omega, Xb, out);
    BIE_LAUNCH_CHECK(c, "k_phi_solid");
  }
  BIE_CUDA_TRY(c, cudaMemsetAsync(psik, 0, sizeof(double) * BIE_MAXB, c->stream));
  s = psi_run(c, omega, psik);
  if (s != BIE_OK) return s;
  k_phi_bound_finish<<<(N + 255) / 256, 256, 0, c->stream>>>(B, y, psi0, psik, out);
  BIE_LAUNCH_CHECK(c, "k_phi_bound_finish");
  return BIE_OK;
}

extern "C" {

bie_status bie_boundary_potential(bie_ctx* c, const double* omega_dev, double* phi_dev) {
  BIE_NVTX("bie_boundary_potential");
  if (!c) return BIE_ERR_ARG;
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_boundary_potential: not assembled");
  if (c->transposed || c->variant != 0)
    return ctx_fail(c, BIE_ERR_STATE,
                    "bie_boundary_potential: storage must hold the operator of eq. lin:sys; assemble again");
  if (!omega_dev || !phi_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_boundary_potential: null pointer");
  cudaSetDevice(c->device);
  return boundary_potential_run(c, omega_dev, (double2*)phi_dev);
}

bie_status bie_filter(bie_ctx* c, double* x_dev) {
  BIE_NVTX("bie_filter");
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom) return ctx_fail(c, BIE_ERR_STATE, "bie_filter: no geometry");
  if (!x_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_filter: null pointer");
  cudaSetDevice(c->device);
  return filter_run(c, x_dev, 1);
}

bie_status bie_energy(bie_ctx* c, const double* phit_dev, const double* omega_dev, double tau,
                      double g, double* E_host) {
  BIE_NVTX("bie_energy");
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom || !c->have_flow)
    return ctx_fail(c, BIE_ERR_STATE, "bie_energy: set geometry and flow first");
  if (!phit_dev || !omega_dev || !E_host) return ctx_fail(c, BIE_ERR_ARG, "bie_energy: null pointer");
  cudaSetDevice(c->device);
  double* E;
  BIE_GET(c, double, "en_E", 1, E);
  bie_status s = energy_run(c, phit_dev, omega_dev, tau, g, E);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(E_host, E, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

bie_status bie_graph_rhs(bie_ctx* c, const double* eta_dev, const double* phit_dev, double tau,
                         double g, int precision, const bie_solve_opts* opts, double* eta_t_dev,
                         double* phit_t_dev, double* omega_dev, double* U_dev) {
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_graph_rhs: not available on a row-partitioned context");
  BIE_NVTX("bie_graph_rhs");
  return one_stage(c, graph_stage, "bie_graph_rhs", eta_dev, phit_dev, tau, g, precision, opts,
                   eta_t_dev, phit_t_dev, omega_dev, U_dev);
}

bie_status bie_graph_evolve(bie_ctx* c, double* eta_dev, double* phit_dev, double dt, int nsteps,
                            double tau, double g, int filter, int precision,
                            const bie_solve_opts* opts, double* energies_host,
                            bie_evolve_info* info) {
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_graph_evolve: not available on a row-partitioned context");
  BIE_NVTX("bie_graph_evolve");
  return rk4_drive(c, graph_stage, "bie_graph_evolve", eta_dev, phit_dev, dt, nsteps, tau, g,
                   filter, precision, opts, energies_host, info);
}

bie_status bie_hls_evolve(bie_ctx* c, double* Ptheta_dev, double* phit_dev, double dt, int nsteps,
                          double tau, double g, int filter, int precision,
                          const bie_solve_opts* opts, double* energies_host,
                          bie_evolve_info* info) {
  BIE_NVTX("bie_hls_evolve");
  return rk4_drive(c, hls_stage, "bie_hls_evolve", Ptheta_dev, phit_dev, dt, nsteps, tau, g,
                   filter, precision, opts, energies_host, info);
}

bie_status bie_evolve(bie_ctx* c, int formulation, int integrator, double* y1_dev,
                      double* phit_dev, double dt, int nsteps, double tau, double g, int filter,
                      int precision, const bie_solve_opts* opts, double* energies_host,
                      bie_evolve_info* info) {
  BIE_NVTX("bie_evolve");
  if (!c) return BIE_ERR_ARG;
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_evolve: not available on a row-partitioned context");
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_hls_evolve: not available on a row-partitioned context");
  if (formulation != BIE_FORM_GRAPH && formulation != BIE_FORM_HLS &&
      formulation != BIE_FORM_VS_GRAPH)
    return ctx_fail(c, BIE_ERR_ARG, "bie_evolve: unknown formulation");
  if (integrator != BIE_INT_RK4 && integrator != BIE_INT_GBS8 && integrator != BIE_INT_DP8)
    return ctx_fail(c, BIE_ERR_ARG, "bie_evolve: unknown integrator");
  if (formulation == BIE_FORM_VS_GRAPH && energies_host)
    return ctx_fail(c, BIE_ERR_ARG, "bie_evolve: the energy monitor needs phi~ (not the vortex-sheet state)");
  StageFn st = formulation == BIE_FORM_GRAPH ? graph_stage
               : formulation == BIE_FORM_HLS ? hls_stage : vs_stage;
  if (integrator == BIE_INT_RK4)
    return rk4_drive(c, st, "bie_evolve", y1_dev, phit_dev, dt, nsteps, tau, g, filter, precision,
                     opts, energies_host, info);
  return step_drive(c, st, integrator == BIE_INT_DP8 ? dp8_step : gbs8_step, "bie_evolve", y1_dev,
                    phit_dev, dt, nsteps, tau, g, filter, precision, opts, energies_host, info);
}

bie_status bie_vs_graph_rhs(bie_ctx* c, const double* eta_dev, const double* gamma0_dev, double tau,
                           double g, int precision, const bie_solve_opts* opts, double* eta_t_dev,
                           double* gamma0_t_dev, double* U_dev) {
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_vs_graph_rhs: not available on a row-partitioned context");
  BIE_NVTX("bie_vs_graph_rhs");
  return one_stage(c, vs_stage, "bie_vs_graph_rhs", eta_dev, gamma0_dev, tau, g, precision, opts,
                   eta_t_dev, gamma0_t_dev, nullptr, U_dev);
}

bie_status bie_hls_rhs(bie_ctx* c, const double* Ptheta_dev, const double* phit_dev, double tau,
                       double g, int precision, const bie_solve_opts* opts, double* Ptheta_t_dev,
                       double* phit_t_dev, double* omega_dev, double* U_dev) {
  BIE_NVTX("bie_hls_rhs");
  return one_stage(c, hls_stage, "bie_hls_rhs", Ptheta_dev, phit_dev, tau, g, precision, opts,
                   Ptheta_t_dev, phit_t_dev, omega_dev, U_dev);
}

bie_status bie_hls_curve(bie_ctx* c, const double* Ptheta_dev, double* zeta_dev, double* dzeta_dev,
                         double* d2zeta_dev) {
  if (!c) return BIE_ERR_ARG;
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_hls_rhs: not available on a row-partitioned context");
  if (!c->have_geom) return ctx_fail(c, BIE_ERR_STATE, "bie_hls_curve: no geometry");
  if (!Ptheta_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_hls_curve: null pointer");
  cudaSetDevice(c->device);
  const int M0 = c->M[0];
  double *y, *par;
  double2* Tp;
  BIE_GET(c, double, "ev_y", 2 * (size_t)M0, y);
  BIE_GET(c, double2, "hls_Tp", 2 * (size_t)M0, Tp);
  BIE_GET(c, double, "hls_par", 4, par);
  BIE_CUDA_TRY(c, cudaMemcpyAsync(y, Ptheta_dev, sizeof(double) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemsetAsync(y + M0, 0, sizeof(double) * M0, c->stream));
  bie_status s = hls_surface(c, y, Tp, par);
  if (s != BIE_OK) return s;
  bool oom = false;
  const double2* z = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * c->N, &oom);
  const double2* dz = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * c->N, &oom);
  const double2* d2z = (const double2*)ctx_buf(c, "d2zeta", sizeof(double2) * c->N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_hls_curve: nodes");
  if (zeta_dev)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(zeta_dev, z, sizeof(double2) * M0, cudaMemcpyDeviceToDevice, c->stream));
  if (dzeta_dev)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(dzeta_dev, dz, sizeof(double2) * M0, cudaMemcpyDeviceToDevice, c->stream));
  if (d2zeta_dev)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(d2zeta_dev, d2z, sizeof(double2) * M0, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

}  // extern "C"
