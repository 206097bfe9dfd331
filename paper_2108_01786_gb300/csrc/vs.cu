// Vortex-sheet route to the normal velocity (Sec. 4): given the surface
// vortex-sheet strength gamma_0, solve the solid-boundary system of eq.
// lin:sys2 for gamma_1..gamma_N and evaluate U from eq. U:from:gam:j.
//
// Solid system (rows m on solid boundary k, columns l on solid boundary j):
//   E_ml = Im{zeta_k'(alpha_m) 1/2 cot((zeta_k(alpha_m) - zeta_j(beta_l))/2)}/M_j
//          - 1/2 delta_ml,          diagonal limit Im{zeta''/(2 zeta')}/M_k,
//   rhs_m = -Re{zeta_k'(alpha_m) sum_l 1/2 cot((zeta_k(alpha_m) - zeta_0(beta_l))/2) gamma_0l}/M_0
//           - s d phi_mv/dn (alpha_m),
// i.e. the transposed kernels of eq. KG:tmat with the weights of the source
// boundary.  In terms of the velocity-potential values S (Table 1 kernel
// times M_l) this is S^T W - 1/2 on the solid blocks without the -E_k term:
// the assembly kernel in its transposed mode with every node solid, on a
// private sub-context holding the solid boundaries only, solved by the same
// GMRES / GMRES-IR (no row flip; all diagonal signs -1/2).
//
// U from gamma is the velocity-potential U formula with omega_0' = -gamma_0
// and omega_j' = gamma_j (eqs. gam:def, U:from:gam:j), so the matrix-free
// normal-velocity kernels run on c_l = gamma-derived weights and
// H omega_0' = -H gamma_0.
#include <cstring>

#include "common.cuh"
#include "nvtx.cuh"
#include "dft.cuh"
#include "pair_kernel.cuh"

#define VS_CH 512
#define VS_FIELDS 3   // S.re S.im cs

// Partial sums over a chunk of surface sources l for solid targets m:
//   S = sum_l G_lm c_l,  cs = sum_l c_l,  G_lm = 1/2 cot((zeta_l - zeta_m)/2),
//   c_l = gamma_0l / M_0 (double-float).
__global__ void __launch_bounds__(256) k_vs_rhs_partial(int N, int M0,
                                                        const float4* __restrict__ nP,
                                                        const float4* __restrict__ nQ,
                                                        const float4* __restrict__ nPQc,
                                                        const double2* __restrict__ z64,
                                                        const double* __restrict__ gamma0,
                                                        float near2, float2* __restrict__ part) {
  __shared__ float4 sP[VS_CH];
  __shared__ float2 sPc[VS_CH];
  __shared__ double2 sZ[VS_CH];
  __shared__ float2 sC[VS_CH];
  const int Ns = N - M0;
  const int s0 = blockIdx.y * VS_CH;
  const int ns = min(VS_CH, M0 - s0);
  for (int t = threadIdx.x; t < ns; t += blockDim.x) {
    sP[t] = nP[s0 + t];
    const float4 pq = nPQc[s0 + t];
    sPc[t] = make_float2(pq.x, pq.y);
    sZ[t] = z64[s0 + t];
    const dfl c = df_from_double(gamma0[s0 + t] / (double)M0);
    sC[t] = make_float2(c.hi, c.lo);
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Ns) return;
  const int m = M0 + t;
  const float4 qv = nQ[m];
  const cx<dfl> Q = {{qv.x, qv.y}, {qv.z, qv.w}};
  const float4 qc4 = nPQc[m];
  const float2 Qc = make_float2(qc4.z, qc4.w);
  const double2 zm = z64[m];
  dfl Sr = {0.f, 0.f}, Si = {0.f, 0.f}, cs = {0.f, 0.f};
  for (int i = 0; i < ns; ++i) {
    const float4 pv = sP[i];
    const cx<dfl> P = {{pv.x, pv.y}, {pv.z, pv.w}};
    const cx<dfl> G = half_cot_pair<dfl>(P, Q, sPc[i], Qc, sZ[i], zm, near2);
    const dfl c = {sC[i].x, sC[i].y};
    Sr = Sr + G.re * c;
    Si = Si + G.im * c;
    cs = cs + c;
  }
  float2* p = part + (size_t)blockIdx.y * VS_FIELDS * Ns;
  p[0 * Ns + t] = make_float2(Sr.hi, Sr.lo);
  p[1 * Ns + t] = make_float2(Si.hi, Si.lo);
  p[2 * Ns + t] = make_float2(cs.hi, cs.lo);
}

// rhs_m = Re{zeta_m' S} - s d phi_mv/dn (m), since sum_l 1/2 cot((zeta_m - zeta_l)/2) c_l = -S
__global__ void k_vs_rhs_finish(int N, int M0, int nchunk, FlowParams F,
                                const float2* __restrict__ part, const double2* __restrict__ z64,
                                const double2* __restrict__ dz64, double* __restrict__ rhs) {
  const int Ns = N - M0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Ns) return;
  dfl acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int ch = 0; ch < nchunk; ++ch) {
    const float2* p = part + (size_t)ch * VS_FIELDS * Ns;
    for (int f = 0; f < 2; ++f) acc[f] = acc[f] + dfl{p[f * Ns + t].x, p[f * Ns + t].y};
  }
  const double Sr = df_to_double(acc[0]), Si = df_to_double(acc[1]);
  const int m = M0 + t;
  const double2 zp = dz64[m], zm = z64[m];
  double asum = 0.0;
  for (int j = 2; j < F.nb; ++j) asum += F.a[j - 2];
  double mv = -(F.V1 + 0.5 * asum) * zp.y;
  for (int j = 2; j < F.nb; ++j) {
    const double ux = zm.x - F.zc[j - 2].x, uy = zm.y - F.zc[j - 2].y;
    double s, c;
    sincos(ux, &s, &c);
    const double e = exp(-uy);
    const double qr = e * c - 1.0, qi = e * s;
    const double n2 = qr * qr + qi * qi;
    const double hr = qi / n2, hi = 0.5 + qr / n2;
    mv += F.a[j - 2] * (hr * zp.x - hi * zp.y);
  }
  rhs[t] = (zp.x * Sr - zp.y * Si) - mv;
}

__global__ void k_vs_fill(int n, float v, float* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

// omega'/M weights from gamma: -gamma_0/M_0 on the surface, gamma_j/M_j on
// solids; H omega_0' = -H gamma_0 (X2 = DFT-side of the Hilbert symbol)
__global__ void k_vs_weights(Blocks B, const double* __restrict__ gamma0,
                             const double* __restrict__ gs, const double2* __restrict__ X2,
                             float2* __restrict__ cw, float2* __restrict__ hw0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.N) return;
  int k = 0;
  while (k + 1 < B.nb && t >= B.off[k + 1]) ++k;
  const double M = (double)B.M[k];
  const int M0 = B.M[0];
  const double w = (t < M0) ? -gamma0[t] / M : gs[t - M0] / M;
  const dfl c = df_from_double(w);
  cw[t] = make_float2(c.hi, c.lo);
  if (t < M0) {
    const dfl h = df_from_double(-X2[t].x / (double)M0);
    hw0[t] = make_float2(h.hi, h.lo);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// the sub-context of the solid boundaries (blocks 1..nb-1 of c), no validation
// (c's geometry was validated), every diagonal sign -1/2, assembled in the
// vortex-sheet mode
static bie_status vs_prepare(bie_ctx* c, int precision) {
  // the solid system depends on the solid boundaries only: a moving free
  // surface (the evolution stages) leaves it as it is
  if (c->vs && c->vs_version == c->solid_version && c->vs_precision == precision) return BIE_OK;
  if (!c->vs) {
    bie_ctx* s = nullptr;
    bie_status st = bie_create(&s, c->device, c->stream);
    if (st != BIE_OK) return ctx_fail(c, st, "vortex sheet: sub-context");
    c->vs = s;
  }
  bie_ctx* s = c->vs;
  s->stream = c->stream;
  const int M0 = c->M[0];
  s->nb = c->nb - 1;
  s->N = c->N - M0;
  s->ld = round_up(s->N, BIE_LD_ALIGN);
  partition_update(s);   // a private context holds every row
  s->off[0] = 0;
  for (int k = 0; k < BIE_MAXB; ++k) {
    s->M[k] = (k + 1 < c->nb) ? c->M[k + 1] : 0;
    s->off[k + 1] = s->off[k] + s->M[k];
    s->fft_m1[k] = (k + 1 < BIE_MAXB) ? c->fft_m1[k + 1] : 0;
    s->zc[k] = make_double2(0.0, 0.0);
  }
  s->assembled = false;
  s->transposed = false;
  s->asm_vs = true;
  const size_t nbytes = sizeof(double2) * (size_t)s->N;
  double2 *z, *dz, *d2z;
  BIE_GET(s, double2, "zeta", s->N, z);
  BIE_GET(s, double2, "dzeta", s->N, dz);
  BIE_GET(s, double2, "d2zeta", s->N, d2z);
  bool oom = false;
  const double2* cz = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * c->N, &oom);
  const double2* cdz = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * c->N, &oom);
  const double2* cd2z = (const double2*)ctx_buf(c, "d2zeta", sizeof(double2) * c->N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "vortex sheet: node buffers");
  BIE_CUDA_TRY(c, cudaMemcpyAsync(z, cz + M0, nbytes, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(dz, cdz + M0, nbytes, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(d2z, cd2z + M0, nbytes, cudaMemcpyDeviceToDevice, c->stream));
  bie_status st = geometry_prep(s);
  if (st != BIE_OK) return ctx_fail(c, st, "vortex sheet: " + s->err);
  s->have_geom = true;
  float* sgn;
  BIE_GET(s, float, "sgn", s->ld, sgn);
  k_vs_fill<<<(unsigned)((s->N + 255) / 256), 256, 0, c->stream>>>(s->N, -0.5f, sgn);
  BIE_LAUNCH_CHECK(c, "k_vs_fill");
  s->asm_sig = -1;   // every node of this system is solid: always in full
  st = asm_run(s, precision, 1);
  if (st != BIE_OK) return ctx_fail(c, st, "vortex sheet: " + s->err);
  s->precision = precision;
  s->assembled = true;
  c->vs_version = c->solid_version;
  c->vs_precision = precision;
  return BIE_OK;
}

extern "C" bie_status bie_vs_normal_velocity(bie_ctx* c, const double* gamma0, double* U,
                                             double* gamma_out, int precision,
                                             const bie_solve_opts* opts, bie_solve_info* info) {
  BIE_NVTX("bie_vs_normal_velocity");
  if (!c) return BIE_ERR_ARG;
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_vs_normal_velocity: not available on a row-partitioned context");
  if (!c->have_geom || !c->have_flow)
    return ctx_fail(c, BIE_ERR_STATE, "bie_vs_normal_velocity: geometry/flow missing");
  if (!gamma0 || !U) return ctx_fail(c, BIE_ERR_ARG, "bie_vs_normal_velocity: null pointer");
  if (precision < BIE_FP64 || precision > BIE_FP16_IR)
    return ctx_fail(c, BIE_ERR_ARG, "bie_vs_normal_velocity: bad precision");
  bie_solve_opts o;
  bie_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > 1000 || o.max_cycles < 1)
    return ctx_fail(c, BIE_ERR_ARG, "bie_vs_normal_velocity: bad options");
  o.row_flip = 0;   // every diagonal sign of the solid system is -1/2
  cudaSetDevice(c->device);
  const int N = c->N, M0 = c->M[0], Ns = N - M0;
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  bool oom = false;
  const float4* nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, &oom);
  const float4* nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, &oom);
  const float4* nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, &oom);
  const double2* z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  const double2* tw = (const double2*)ctx_buf(c, "dft_tw", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_vs_normal_velocity: node buffers");
  // 1. right-hand side of the solid system
  const int nch = (M0 + VS_CH - 1) / VS_CH;
  double *rhs, *gs;
  float2* rpart;
  BIE_GET(c, double, "vs_rhs", round_up(Ns, BIE_LD_ALIGN), rhs);
  BIE_GET(c, double, "vs_gamma", round_up(Ns, BIE_LD_ALIGN), gs);
  BIE_GET(c, float2, "vs_rpart", (size_t)nch * VS_FIELDS * Ns, rpart);
  if (Ns > 0) {
    k_vs_rhs_partial<<<dim3((Ns + 255) / 256, nch), 256, 0, c->stream>>>(N, M0, nP, nQ, nPQc, z64,
                                                                         gamma0, 0.01f, rpart);
    BIE_LAUNCH_CHECK(c, "k_vs_rhs_partial");
    k_vs_rhs_finish<<<(Ns + 255) / 256, 256, 0, c->stream>>>(N, M0, nch, F, rpart, z64, dz64, rhs);
    BIE_LAUNCH_CHECK(c, "k_vs_rhs_finish");
    // 2. the solid system
    bie_status st = vs_prepare(c, precision);
    if (st != BIE_OK) return st;
    bie_ctx* s = c->vs;
    if (o.x0 && gamma_out)   // the caller's solid strengths are the initial guess
      BIE_CUDA_TRY(c, cudaMemcpyAsync(gs, gamma_out, sizeof(double) * Ns, cudaMemcpyDeviceToDevice,
                                      c->stream));
    else
      o.x0 = 0;
    const bie_status ss = solve_system(s, &o, gs, rhs, info);
    if (ss != BIE_OK) return ctx_fail(c, ss, "bie_vs_normal_velocity: " + s->err);
  } else if (info) {
    info->iters = 0;
    info->cycles = 0;
    info->converged = 1;
    info->rel_resid = 0.0;
  }
  // 3. H gamma_0 by the DFT, the weights, and U (matrix-free kernels)
  double2 *dY, *dX1, *dX2;
  BIE_GET(c, double2, "dft_Y", N + M0, dY);
  BIE_GET(c, double2, "dft_X1", N, dX1);
  BIE_GET(c, double2, "dft_X2", N + M0, dX2);
  {
    DftJobs J1, J2;
    memset(&J1, 0, sizeof(J1));
    memset(&J2, 0, sizeof(J2));
    const int m1 = c->fft_m1[0];
    J1.j[J1.n++] = DftJob{M0, m1, M0 / m1, 0, 0, 0, 0, 0};
    J2.j[J2.n++] = DftJob{M0, m1, M0 / m1, 0, 0, 0, 4, 0};
    J1.total = J2.total = M0;
    const unsigned g = (unsigned)((M0 + 255) / 256);
    k_dft_a<<<dft_grid(g), 256, 0, c->stream>>>(J1, gamma0, nullptr, tw, dY);
    BIE_LAUNCH_CHECK(c, "k_dft_a");
    k_dft_b<<<dft_grid(g), 256, 0, c->stream>>>(J1, dY, tw, dX1);
    BIE_LAUNCH_CHECK(c, "k_dft_b");
    k_dft_a<<<dft_grid(g), 256, 0, c->stream>>>(J2, nullptr, dX1, tw, dY);
    BIE_LAUNCH_CHECK(c, "k_dft_a");
    k_dft_b<<<dft_grid(g), 256, 0, c->stream>>>(J2, dY, tw, dX2);
    BIE_LAUNCH_CHECK(c, "k_dft_b");
  }
  float2 *cw, *hw0;
  BIE_GET(c, float2, "vel_cw", N, cw);
  BIE_GET(c, float2, "vel_hw0", M0, hw0);
  k_vs_weights<<<(N + 255) / 256, 256, 0, c->stream>>>(B, gamma0, gs, dX2, cw, hw0);
  BIE_LAUNCH_CHECK(c, "k_vs_weights");
  bie_status su = velocity_from_weights(c, cw, hw0, U);
  if (su != BIE_OK) return su;
  if (gamma_out && Ns > 0)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(gamma_out, gs, sizeof(double) * Ns, cudaMemcpyDeviceToDevice,
                                    c->stream));
  return BIE_OK;
}
