// C-ABI entry points, context and workspace management, geometry/node
// preparation and the right-hand side of eq. Awb.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>

#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "nvtx.cuh"

// ---------------------------------------------------------------------------
// context helpers
// ---------------------------------------------------------------------------
bie_status ctx_fail(bie_ctx* c, bie_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

bie_status ctx_cuda(bie_ctx* c, cudaError_t e, const char* where) {
  if (c) c->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  return BIE_ERR_CUDA;
}

void* ctx_buf(bie_ctx* c, const char* name, size_t bytes, bool* oom) {
  *oom = false;
  if (bytes == 0) bytes = 16;
  for (auto& kv : c->bufs) {
    if (kv.first == name) {
      if (kv.second.bytes >= bytes) return kv.second.p;
      cudaFree(kv.second.p);
      kv.second.p = nullptr;
      kv.second.bytes = 0;
      void* p = nullptr;
      if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *oom = true;
        return nullptr;
      }
      kv.second.p = p;
      kv.second.bytes = bytes;
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *oom = true;
    return nullptr;
  }
  c->bufs.push_back({std::string(name), DevBuf{p, bytes}});
  return p;
}

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, fn}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}


// ---------------------------------------------------------------------------
// profiling
// ---------------------------------------------------------------------------
int prof_begin(bie_ctx* c, int kind, int tag) {
  if (!c->profiling) return -1;
  if (c->ev_used + 2 > (int)c->ev_pool.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return -1;
      }
      c->ev_pool.push_back(e);
    }
  }
  const int ev = c->ev_used;
  c->ev_used += 2;
  cudaEventRecord(c->ev_pool[ev], c->stream);
  c->prof_recs.push_back({kind, ev, tag, true});
  return (int)c->prof_recs.size() - 1;
}

void prof_end(bie_ctx* c, int rec) {
  if (rec < 0) return;
  cudaEventRecord(c->ev_pool[c->prof_recs[rec].ev + 1], c->stream);
}

void prof_invalidate_steps(bie_ctx* c, int from_step) {
  // inner products of steps >= from_step in the cycle just finished were
  // skipped on the device (the cycle had converged): do not count them.  Only
  // that cycle's records are open: scan back to the last closed one.
  const int kClosed = -1000000;
  for (auto it = c->prof_recs.rbegin(); it != c->prof_recs.rend(); ++it) {
    if (it->kind != 0) continue;
    if (it->tag == kClosed) break;
    if (it->tag >= from_step) it->valid = false;
    it->tag = kClosed;
  }
}

bie_status prof_collect(bie_ctx* c) {
  if (c->prof_recs.empty()) return BIE_OK;
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (const auto& r : c->prof_recs) {
    if (!r.valid) continue;
    float ms = 0.f;
    BIE_CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev_pool[r.ev], c->ev_pool[r.ev + 1]));
    switch (r.kind) {
      case 0: c->prof.n_gemv_inner++; c->prof.ms_gemv_inner += ms; break;
      case 1: c->prof.n_gemv_full++; c->prof.ms_gemv_full += ms; break;
      case 2: c->prof.n_assemble++; c->prof.ms_assemble += ms; break;
      case 4: c->prof.n_gemv_hi++; c->prof.ms_gemv_hi += ms; break;
      default: c->prof.n_velocity++; c->prof.ms_velocity += ms; break;
    }
  }
  c->prof_recs.clear();
  c->ev_used = 0;
  return BIE_OK;
}

// ---------------------------------------------------------------------------
// node preparation
//   P_l = e^{i zeta_l}, Q_l = e^{-i zeta_l}   (separable form of the kernel:
//        1/2 cot((zeta_l - zeta_m)/2) = i/2 + i/(P_l Q_m - 1), App. E)
//   diag_l = Im{zeta''/(2 zeta')}            (diagonal limit of K_jj, Sec. 3.2)
//   gdiag_l = Re{zeta''/(2 zeta')}           (diagonal limit of G_00 in eq. d:phi:0)
//   wgt_l = 1/M_j                            (trapezoidal weight, Sec. 3.3)
//   sgn_l = -1/2 (surface) or +1/2 (solids)  (eq. lin:sys diagonal)
// ---------------------------------------------------------------------------
__global__ void k_node_prep(Blocks B, const double2* __restrict__ z, const double2* __restrict__ dz,
                            const double2* __restrict__ d2z, int* __restrict__ blk,
                            float* __restrict__ wgt, double* __restrict__ wgt64,
                            float* __restrict__ sgn, float4* __restrict__ nP,
                            float4* __restrict__ nQ, float4* __restrict__ nPQc,
                            float4* __restrict__ nZp,
                            float2* __restrict__ nDiag, double2* __restrict__ P64,
                            double2* __restrict__ Q64, double* __restrict__ diag64,
                            double* __restrict__ gdiag64, long long ld) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= ld) return;
  if (l >= B.N) {
    wgt[l] = 0.f;
    return;
  }
  int k = 0;
  while (k + 1 < B.nb && l >= B.off[k + 1]) ++k;
  blk[l] = k;
  const double w = 1.0 / (double)B.M[k];
  wgt[l] = (float)w;
  wgt64[l] = w;
  sgn[l] = (k == 0) ? -0.5f : 0.5f;
  const double2 zl = z[l];
  double s, c;
  sincos(zl.x, &s, &c);
  const double em = exp(-zl.y), ep = exp(zl.y);
  const double2 P = make_double2(em * c, em * s);
  const double2 Q = make_double2(ep * c, -ep * s);
  P64[l] = P;
  Q64[l] = Q;
  const dfl pr = df_from_double(P.x), pi = df_from_double(P.y);
  const dfl qr = df_from_double(Q.x), qi = df_from_double(Q.y);
  nP[l] = make_float4(pr.hi, pr.lo, pi.hi, pi.lo);
  nQ[l] = make_float4(qr.hi, qr.lo, qi.hi, qi.lo);
  // third words of P and Q: without them every entry of row m would share the
  // rounding error of Q_m (and of P_l down column l), a correlated error that
  // does not average out in the row sums of the residual
  nPQc[l] = make_float4(df_residue(P.x, pr), df_residue(P.y, pi), df_residue(Q.x, qr),
                        df_residue(Q.y, qi));
  const double2 d1 = dz[l], d2 = d2z[l];
  const dfl zr = df_from_double(d1.x), zi = df_from_double(d1.y);
  nZp[l] = make_float4(zr.hi, zr.lo, zi.hi, zi.lo);
  // zeta''/(2 zeta') = d2 conj(d1) / (2 |d1|^2)
  const double den = 2.0 * (d1.x * d1.x + d1.y * d1.y);
  const double re = (d2.x * d1.x + d2.y * d1.y) / den;
  const double im = (d2.y * d1.x - d2.x * d1.y) / den;
  diag64[l] = im;
  const dfl di = df_from_double(im);
  nDiag[l] = make_float2(di.hi, di.lo);
  if (k == 0) gdiag64[l] = re;
}

// Per-boundary tables: DFT twiddles tw[off_k + j] = e^{-2 pi i j / M_k}, and,
// on the surface, T_j = 1/2 cot(pi j / M_0), T_0 = 0 (the Hilbert-regularising
// term of G_00 in eq. d:phi:0).
__global__ void k_spectral_tables(Blocks B, double2* __restrict__ tw, float2* __restrict__ Ttab,
                                  double* __restrict__ T64, float2* __restrict__ Tall) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= B.N) return;
  int k = 0;
  while (k + 1 < B.nb && l >= B.off[k + 1]) ++k;
  const int M = B.M[k];
  const int j = l - B.off[k];
  double s, c;
  sincospi(2.0 * (double)j / (double)M, &s, &c);
  tw[l] = make_double2(c, -s);
  if (Tall) {  // 1/2 cot(pi j / M_k) for every boundary (Hilbert terms on Gamma_k)
    double Tk = 0.0;
    if (j != 0) {
      double s1, c1;
      sincospi((double)j / (double)M, &s1, &c1);
      Tk = 0.5 * c1 / s1;
    }
    const dfl tk = df_from_double(Tk);
    Tall[l] = make_float2(tk.hi, tk.lo);
  }
  if (k == 0) {
    double T = 0.0;
    if (j != 0) {
      double s1, c1;
      sincospi((double)j / (double)M, &s1, &c1);
      T = 0.5 * c1 / s1;
    }
    const dfl tt = df_from_double(T);
    Ttab[l] = make_float2(tt.hi, tt.lo);
    if (T64) T64[l] = T;
  }
}

// ---------------------------------------------------------------------------
// right-hand side, eq. Awb: b_0 = phi~, b_k = -psi_mv(zeta_k),
//   psi_mv(z) = V1 Im z + sum_j a_j psi_cyl(z - z_j),  psi_cyl(z) = -ln|1 - e^{iz}|
// ---------------------------------------------------------------------------
__global__ void k_rhs(Blocks B, FlowParams F, const double2* __restrict__ z,
                      const double* __restrict__ phit, double* __restrict__ b,
                      long long pstride = 0, long long bstride = 0) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= B.N) return;
  phit += blockIdx.y * pstride;   // right-hand side blockIdx.y of a batch
  b += blockIdx.y * bstride;
  if (l < B.M[0]) {
    b[l] = phit[l];
    return;
  }
  const double2 zl = z[l];
  double v = -F.V1 * zl.y;
  for (int j = 2; j < F.nb; ++j) {
    const double ux = zl.x - F.zc[j - 2].x, uy = zl.y - F.zc[j - 2].y;
    double s, c;
    sincos(ux, &s, &c);
    const double e = exp(-uy);
    const double re = 1.0 - e * c, im = -e * s;
    v += F.a[j - 2] * 0.5 * log(re * re + im * im);   // = -a_j psi_cyl
  }
  b[l] = v;
}

// App. B right-hand side: b_0 = phi - V1 xi (given), b_k = psi - V1 eta_k on solid nodes
__global__ void k_rhs_psi(int N, int M0, double V1, const double2* __restrict__ z,
                          const double* __restrict__ phic, const double* __restrict__ psi,
                          double* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  b[i] = (i < M0) ? phic[i] : psi[i - M0] - V1 * z[i].y;
}

// nrhs right-hand sides at once: phi~ column r at phit + r pstride, b at b + r bstride
bie_status rhs_run_many(bie_ctx* c, int nrhs, const double* phit, long long pstride, double* b,
                        long long bstride) {
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  const double2* z;
  BIE_GET(c, double2, "zeta", c->N, z);
  k_rhs<<<dim3((c->N + 255) / 256, nrhs), 256, 0, c->stream>>>(B, F, z, phit, b, pstride, bstride);
  BIE_LAUNCH_CHECK(c, "k_rhs");
  return BIE_OK;
}

bie_status rhs_run(bie_ctx* c, const double* phit, double* b) {
  const Blocks B = make_blocks(c);
  const FlowParams F = make_flow(c);
  const double2* z;
  BIE_GET(c, double2, "zeta", c->N, z);
  k_rhs<<<(c->N + 255) / 256, 256, 0, c->stream>>>(B, F, z, phit, b);
  BIE_LAUNCH_CHECK(c, "k_rhs");
  return BIE_OK;
}

// ---------------------------------------------------------------------------
// geometry validation on a host copy
// ---------------------------------------------------------------------------
// Geometry checks over chunks of 256 nodes of boundary k (grid: chunks x
// boundaries): first node in the chunk with non-finite data, with zeta' = 0,
// that coincides with its successor (periodic image across the seam of the
// surface and the bottom), and the chunk's parts of twice the shoelace area
// and of the advance sum_l Re zeta'_l.  The host takes the minima and adds
// the parts in chunk order (deterministic).
struct GeomCheck {
  int bad_finite, bad_dz, bad_coinc, pad;
  double area2, adv;
};
static const int kGeomChunk = 256;
// N <= 2^17 nodes: at most 2^17 / 256 chunks plus one partial chunk per boundary
static const int kGeomMaxChunks = (1 << 17) / kGeomChunk + BIE_MAXB;

// chunk q of all boundaries belongs to boundary k when co[k] <= q < co[k+1]
struct GeomChunks {
  int co[BIE_MAXB + 1];
};
static GeomChunks geom_chunks(const bie_ctx* c) {
  GeomChunks g;
  g.co[0] = 0;
  for (int k = 0; k < c->nb; ++k) g.co[k + 1] = g.co[k] + (c->M[k] + kGeomChunk - 1) / kGeomChunk;
  return g;
}

__global__ void __launch_bounds__(kGeomChunk) k_validate_geometry(Blocks B, GeomChunks Q,
                                                                  const double2* __restrict__ z,
                                                                  const double2* __restrict__ dz,
                                                                  const double2* __restrict__ d2z,
                                                                  GeomCheck* __restrict__ out) {
  __shared__ int s_fin, s_dz, s_co;
  __shared__ double s_a[kGeomChunk / 32], s_v[kGeomChunk / 32];
  int k = 0;
  while (k + 1 < B.nb && (int)blockIdx.x >= Q.co[k + 1]) ++k;
  const int o = B.off[k], M = B.M[k];
  const int l0 = ((int)blockIdx.x - Q.co[k]) * kGeomChunk;
  if (threadIdx.x == 0) s_fin = s_dz = s_co = INT_MAX;
  __syncthreads();
  double a2 = 0.0, adv = 0.0;
  const int l = l0 + threadIdx.x;
  if (l < M) {
    const double2 zl = z[o + l], dl = dz[o + l], d2 = d2z[o + l];
    if (!isfinite(zl.x) || !isfinite(zl.y) || !isfinite(dl.x) || !isfinite(dl.y) ||
        !isfinite(d2.x) || !isfinite(d2.y))
      atomicMin(&s_fin, l);
    if (dl.x * dl.x + dl.y * dl.y == 0.0) atomicMin(&s_dz, l);
    const int ln = (l + 1) % M;
    const double2 zn = z[o + ln];
    double ex = zn.x - zl.x;
    const double ey = zn.y - zl.y;
    if (k <= 1 && ln == 0) ex += 2.0 * M_PI;   // periodic images of surface/bottom
    if (ex * ex + ey * ey == 0.0) atomicMin(&s_co, l);
    a2 = zl.x * zn.y - zn.x * zl.y;
    adv = dl.x;
  }
  a2 = warp_sum(a2);
  adv = warp_sum(adv);
  if ((threadIdx.x & 31) == 0) {
    s_a[threadIdx.x >> 5] = a2;
    s_v[threadIdx.x >> 5] = adv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tv = 0.0;
    for (int w = 0; w < kGeomChunk / 32; ++w) {
      ta += s_a[w];
      tv += s_v[w];
    }
    GeomCheck g;
    g.bad_finite = s_fin == INT_MAX ? -1 : o + s_fin;
    g.bad_dz = s_dz == INT_MAX ? -1 : s_dz;
    g.bad_coinc = s_co == INT_MAX ? -1 : s_co;
    g.pad = 0;
    g.area2 = ta;
    g.adv = tv;
    out[blockIdx.x] = g;
  }
}

// Enqueue the checks into the host-mapped records (no copy needed).
static bie_status geometry_checks_enqueue(bie_ctx* c) {
  if (!c->geom_host) {
    const size_t bytes = sizeof(GeomCheck) * kGeomMaxChunks;
    cudaError_t e = cudaHostAlloc(&c->geom_host, bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&c->geom_dev, c->geom_host, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (c->geom_host) cudaFreeHost(c->geom_host);
      c->geom_host = c->geom_dev = nullptr;
      return ctx_fail(c, BIE_ERR_CUDA, "geometry checks: pinned buffer");
    }
  }
  const Blocks B = make_blocks(c);
  double2 *z, *dz, *d2z;
  BIE_GET(c, double2, "zeta", c->N, z);
  BIE_GET(c, double2, "dzeta", c->N, dz);
  BIE_GET(c, double2, "d2zeta", c->N, d2z);
  const GeomChunks Q = geom_chunks(c);
  k_validate_geometry<<<Q.co[c->nb], kGeomChunk, 0, c->stream>>>(B, Q, z, dz, d2z,
                                                                 (GeomCheck*)c->geom_dev);
  BIE_LAUNCH_CHECK(c, "k_validate_geometry");
  return BIE_OK;
}

// After the stream has drained: the checks in the order a host loop would
// meet them: non-finite data anywhere first, then per boundary (in order)
// zeta' = 0 or coincident nodes at the first offending node, orientation of
// obstacles, direction of the periodic curves.
static bie_status geometry_checks_result(bie_ctx* c) {
  const GeomChunks Q = geom_chunks(c);
  const GeomCheck* hc = (const GeomCheck*)c->geom_host;
  GeomCheck h[BIE_MAXB];
  auto first_of = [](int a, int b) { return a < 0 ? b : (b < 0 ? a : std::min(a, b)); };
  for (int k = 0; k < c->nb; ++k) {
    GeomCheck t = {-1, -1, -1, 0, 0.0, 0.0};
    for (int q = Q.co[k]; q < Q.co[k + 1]; ++q) {
      const GeomCheck& g = hc[q];
      t.bad_finite = first_of(t.bad_finite, g.bad_finite);
      t.bad_dz = first_of(t.bad_dz, g.bad_dz);
      t.bad_coinc = first_of(t.bad_coinc, g.bad_coinc);
      t.area2 += g.area2;
      t.adv += g.adv;
    }
    h[k] = t;
  }
  int first = -1;
  for (int k = 0; k < c->nb; ++k) first = first_of(first, h[k].bad_finite);
  if (first >= 0)
    return ctx_fail(c, BIE_ERR_GEOM, "non-finite node data at index " + std::to_string(first));
  for (int k = 0; k < c->nb; ++k) {
    const int ldz = h[k].bad_dz, lco = h[k].bad_coinc;
    if (ldz >= 0 && (lco < 0 || ldz <= lco))
      return ctx_fail(c, BIE_ERR_GEOM, "zeta' = 0 on boundary " + std::to_string(k));
    if (lco >= 0)
      return ctx_fail(c, BIE_ERR_GEOM, "coincident nodes on boundary " + std::to_string(k));
    // the sign of the enclosed area tells the orientation of obstacles
    if (k >= 2 && h[k].area2 >= 0.0)
      return ctx_fail(c, BIE_ERR_GEOM,
                      "obstacle " + std::to_string(k) + " is not traversed clockwise");
    // graph-like periodic curves advance by +2 pi per period (left to right)
    if (k <= 1 && h[k].adv <= 0.0)
      return ctx_fail(c, BIE_ERR_GEOM,
                      "boundary " + std::to_string(k) + " must run left to right");
  }
  return BIE_OK;
}

bie_status geometry_prep(bie_ctx* c) {
  const Blocks B = make_blocks(c);
  const long long ld = c->ld;
  double2 *z, *dz, *d2z, *P64, *Q64;
  int* blk;
  float *wgt, *sgn;
  double *wgt64, *diag64, *gdiag64;
  float4 *nP, *nQ, *nPQc, *nZp;
  float2 *nDiag, *Ttab;
  double2* tw;
  BIE_GET(c, double2, "zeta", c->N, z);
  BIE_GET(c, double2, "dzeta", c->N, dz);
  BIE_GET(c, double2, "d2zeta", c->N, d2z);
  BIE_GET(c, int, "blk", ld, blk);
  BIE_GET(c, float, "wgt", ld, wgt);
  BIE_GET(c, double, "wgt64", ld, wgt64);
  BIE_GET(c, float, "sgn", ld, sgn);
  BIE_GET(c, float4, "nP", c->N, nP);
  BIE_GET(c, float4, "nQ", c->N, nQ);
  BIE_GET(c, float4, "nPQc", c->N, nPQc);
  BIE_GET(c, float4, "nZp", c->N, nZp);
  BIE_GET(c, float2, "nDiag", c->N, nDiag);
  BIE_GET(c, double2, "P64", c->N, P64);
  BIE_GET(c, double2, "Q64", c->N, Q64);
  BIE_GET(c, double, "diag64", c->N, diag64);
  BIE_GET(c, double, "gdiag64", c->M[0], gdiag64);
  BIE_GET(c, double2, "dft_tw", c->N, tw);
  BIE_GET(c, float2, "Ttab", c->M[0], Ttab);
  double* T64;
  BIE_GET(c, double, "T64", c->M[0], T64);
  float2* Tall;
  BIE_GET(c, float2, "Tall", c->N, Tall);
  const int nthr = 256;
  k_node_prep<<<(unsigned)((ld + nthr - 1) / nthr), nthr, 0, c->stream>>>(
      B, z, dz, d2z, blk, wgt, wgt64, sgn, nP, nQ, nPQc, nZp, nDiag, P64, Q64, diag64, gdiag64, ld);
  BIE_LAUNCH_CHECK(c, "k_node_prep");
  // the spectral tables depend on the node counts only
  bool same = c->spec_nb == c->nb;
  for (int k = 0; same && k < c->nb; ++k) same = c->spec_M[k] == c->M[k];
  if (!same) {
    c->spec_nb = 0;
    k_spectral_tables<<<(c->N + nthr - 1) / nthr, nthr, 0, c->stream>>>(B, tw, Ttab, T64, Tall);
    BIE_LAUNCH_CHECK(c, "k_spectral_tables");
    for (int k = 0; k < c->nb; ++k) c->spec_M[k] = c->M[k];
    c->spec_nb = c->nb;
  }
  return BIE_OK;
}

// Validate the node arrays now in the library buffers and rebuild every table
// that depends on them (node sizes, flow and obstacle centres unchanged).
bie_status geometry_refresh(bie_ctx* c) {
  c->have_geom = false;
  c->assembled = false;
  c->transposed = false;
  // the checks and the node tables go in together, one wait for both (the
  // tables of a rejected geometry are never used: have_geom stays false)
  bie_status s = geometry_checks_enqueue(c);
  if (s != BIE_OK) return s;
  s = geometry_prep(c);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  s = geometry_checks_result(c);
  if (s != BIE_OK) return s;
  c->have_geom = true;
  c->geom_version += 1;
  return BIE_OK;
}

// Closest approach of two different boundaries, in units of the local node
// spacing h_i = |zeta'_i| 2 pi / M_k at node i: ratio[i] = min_j |zeta_i - zeta_j| / h_i
// over nodes j of the other boundaries (nearest periodic image).  One warp per node.
__global__ void k_separation(Blocks B, const double2* __restrict__ z, const double2* __restrict__ dz,
                             float* __restrict__ ratio) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B.N) return;
  const int i = warp;
  int ki = 0;
  while (ki + 1 < B.nb && i >= B.off[ki + 1]) ++ki;
  const double2 zi = z[i];
  float best = 3.0e38f;
  for (int j = lane; j < B.N; j += 32) {
    if (j >= B.off[ki] && j < B.off[ki + 1]) continue;
    double dx = z[j].x - zi.x;
    dx -= 2.0 * M_PI * rint(dx / (2.0 * M_PI));
    const double dy = z[j].y - zi.y;
    best = fminf(best, (float)(dx * dx + dy * dy));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (lane == 0) {
    const double2 d = dz[i];
    const double h = sqrt(d.x * d.x + d.y * d.y) * 2.0 * M_PI / (double)B.M[ki];
    ratio[i] = (float)(sqrt((double)best) / h);
  }
}

bie_status separation_run(bie_ctx* c, double* ratio_min, int* node) {
  const int N = c->N;
  float* ratio;
  BIE_GET(c, float, "sep_ratio", N, ratio);
  bool oom = false;
  const double2* z = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "separation: nodes");
  k_separation<<<(unsigned)((32LL * N + 255) / 256), 256, 0, c->stream>>>(make_blocks(c), z, dz, ratio);
  BIE_LAUNCH_CHECK(c, "k_separation");
  std::vector<float> h(N);
  BIE_CUDA_TRY(c, cudaMemcpyAsync(h.data(), ratio, sizeof(float) * N, cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  int arg = 0;
  for (int i = 1; i < N; ++i)
    if (h[i] < h[arg]) arg = i;
  *ratio_min = h[arg];
  if (node) *node = arg;
  return BIE_OK;
}

// ---------------------------------------------------------------------------
// row partition (bie_set_partition)
// ---------------------------------------------------------------------------
void partition_update(bie_ctx* c) {
  const int N = c->N;
  if (c->part_n <= 1) {
    c->row0 = 0;
    c->row1 = N;
    c->part_R = N;
    return;
  }
  const long long P = c->part_n;
  const long long R = (N + 32 * P - 1) / (32 * P) * 32;
  c->part_R = R;
  c->row0 = (int)std::min<long long>(N, c->part_p * R);
  c->row1 = (int)std::min<long long>(N, (c->part_p + 1) * R);
}

bie_status part_allgather(bie_ctx* c, void* vec, int eb, int limit) {
  if (!partitioned(c)) return BIE_OK;
  const long long R = c->part_R;
  const int r1 = std::min(c->row1, limit);
  const long long n = std::max(0, r1 - c->row0);
  char* st = (char*)c->exch_buf;
  if (n > 0)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(st + (size_t)c->part_p * R * eb, (char*)vec + (size_t)c->row0 * eb,
                                    (size_t)n * eb, cudaMemcpyDeviceToDevice, c->stream));
  const int rc = c->exch(c->exch_user, BIE_EXCH_ALLGATHER, R, eb, (void*)c->stream);
  if (rc != 0) return ctx_fail(c, BIE_ERR_CUDA, "partition: exchange function failed (allgather)");
  BIE_CUDA_TRY(c, cudaMemcpyAsync(vec, st, (size_t)limit * eb, cudaMemcpyDeviceToDevice, c->stream));
  return BIE_OK;
}

bie_status part_allreduce(bie_ctx* c, double* vec, long long n) {
  if (!partitioned(c) || n <= 0) return BIE_OK;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(c->exch_buf, vec, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  const int rc = c->exch(c->exch_user, BIE_EXCH_ALLREDUCE_SUM, n, 8, (void*)c->stream);
  if (rc != 0) return ctx_fail(c, BIE_ERR_CUDA, "partition: exchange function failed (allreduce)");
  BIE_CUDA_TRY(c, cudaMemcpyAsync(vec, c->exch_buf, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  return BIE_OK;
}

static bie_status refuse_partitioned(bie_ctx* c, const char* who) {
  return ctx_fail(c, BIE_ERR_STATE, std::string(who) + ": not available on a row-partitioned context");
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void bie_default_opts(bie_solve_opts* o) {
  if (!o) return;
  o->rtol = 1e-14;
  o->restart = 50;
  o->max_cycles = 40;
  o->inner_tol = 0.0;
  o->row_flip = 1;
  o->x0 = 0;
}

bie_status bie_create(bie_ctx** out, int device, void* cuda_stream) {
  if (!out) return BIE_ERR_ARG;
  *out = nullptr;
  bie_ctx* c = new bie_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete c;
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  e = cudaHostAlloc((void**)&c->status_host, sizeof(SolveStatus), cudaHostAllocDefault);
  if (e != cudaSuccess) {
    delete c;
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  memset(c->status_host, 0, sizeof(SolveStatus));
  e = cudaHostAlloc((void**)&c->slots_host, sizeof(HostSlot) * BIE_NSLOTS, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&c->slots_dev, c->slots_host, 0);
  for (int i = 0; i < BIE_NSLOTS && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&c->evs[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    bie_destroy(c);
    return BIE_ERR_CUDA;
  }
  memset(c->slots_host, 0, sizeof(HostSlot) * BIE_NSLOTS);
  *out = c;
  return BIE_OK;
}

void bie_destroy(bie_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->vs) {
    bie_destroy(c->vs);
    c->vs = nullptr;
  }
  if (c->gt) {
    bie_destroy(c->gt);
    c->gt = nullptr;
  }
  if (c->ms_mirror_host) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFreeHost(c->ms_mirror_host);
    c->ms_mirror_host = nullptr;
  }
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (auto& kv : c->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  if (c->geom_host) cudaFreeHost(c->geom_host);
  if (c->status_host) cudaFreeHost(c->status_host);
  if (c->slots_host) cudaFreeHost(c->slots_host);
  for (int i = 0; i < BIE_NSLOTS; ++i)
    if (c->evs[i]) cudaEventDestroy(c->evs[i]);
  delete c;
}

const char* bie_last_error(const bie_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

bie_status bie_set_geometry(bie_ctx* c, int nb, const int* M_host, const double* zeta_dev,
                            const double* dzeta_dev, const double* d2zeta_dev,
                            const double* zc_host) {
  BIE_NVTX("bie_set_geometry");
  if (!c) return BIE_ERR_ARG;
  c->err.clear();
  if (nb < 2 || nb > BIE_MAXB || !M_host || !zeta_dev || !dzeta_dev || !d2zeta_dev)
    return ctx_fail(c, BIE_ERR_ARG, "bie_set_geometry: bad nb or null pointer");
  if (nb > 2 && !zc_host) return ctx_fail(c, BIE_ERR_ARG, "bie_set_geometry: zc_host is NULL");
  long long N = 0;
  for (int k = 0; k < nb; ++k) {
    if (M_host[k] < 8) return ctx_fail(c, BIE_ERR_ARG, "bie_set_geometry: M_k < 8");
    N += M_host[k];
  }
  if (N > (1LL << 17)) return ctx_fail(c, BIE_ERR_ARG, "bie_set_geometry: N too large");
  cudaSetDevice(c->device);
  c->have_geom = false;
  c->assembled = false;
  c->transposed = false;
  c->nb = nb;
  c->N = (int)N;
  c->ld = round_up(N, BIE_LD_ALIGN);
  partition_update(c);
  c->off[0] = 0;
  for (int k = 0; k < BIE_MAXB; ++k) {
    c->M[k] = k < nb ? M_host[k] : 0;
    c->off[k + 1] = c->off[k] + c->M[k];
  }
  for (int k = 0; k < nb; ++k) {
    int m1 = 1;
    for (int d = 1; (long long)d * d <= c->M[k]; ++d)
      if (c->M[k] % d == 0) m1 = d;
    c->fft_m1[k] = m1;
  }
  for (int j = 0; j < BIE_MAXB; ++j) c->zc[j] = make_double2(0, 0);
  for (int j = 2; j < nb; ++j) c->zc[j - 2] = make_double2(zc_host[2 * (j - 2)], zc_host[2 * (j - 2) + 1]);
  // copy inputs into library-owned buffers
  double2 *z, *dz, *d2z;
  BIE_GET(c, double2, "zeta", N, z);
  BIE_GET(c, double2, "dzeta", N, dz);
  BIE_GET(c, double2, "d2zeta", N, d2z);
  BIE_CUDA_TRY(c, cudaMemcpyAsync(z, zeta_dev, sizeof(double2) * N, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(dz, dzeta_dev, sizeof(double2) * N, cudaMemcpyDeviceToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(d2z, d2zeta_dev, sizeof(double2) * N, cudaMemcpyDeviceToDevice, c->stream));
  c->solid_version += 1;   // any boundary may have changed
  return geometry_refresh(c);
}

bie_status bie_min_separation(bie_ctx* c, double* ratio_host, int* node_host) {
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom) return ctx_fail(c, BIE_ERR_STATE, "bie_min_separation: no geometry");
  if (!ratio_host) return ctx_fail(c, BIE_ERR_ARG, "bie_min_separation: null pointer");
  cudaSetDevice(c->device);
  return separation_run(c, ratio_host, node_host);
}

bie_status bie_set_min_separation(bie_ctx* c, double ratio) {
  if (!c) return BIE_ERR_ARG;
  if (!(ratio >= 0.0) || !std::isfinite(ratio))
    return ctx_fail(c, BIE_ERR_ARG, "bie_set_min_separation: ratio >= 0 required");
  c->min_sep = ratio;
  return BIE_OK;
}

bie_status bie_set_partition(bie_ctx* c, int nparts, int part, void* stage_dev, size_t stage_bytes,
                             bie_exchange_fn exchange, void* user) {
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom) return ctx_fail(c, BIE_ERR_STATE, "bie_set_partition: no geometry");
  if (nparts < 1 || part < 0 || part >= nparts)
    return ctx_fail(c, BIE_ERR_ARG, "bie_set_partition: need 0 <= part < nparts");
  if (nparts > 1 && (!exchange || !stage_dev))
    return ctx_fail(c, BIE_ERR_ARG, "bie_set_partition: exchange function and stage buffer required");
  const int pn = c->part_n, pp = c->part_p;
  c->part_n = nparts;
  c->part_p = nparts > 1 ? part : 0;
  partition_update(c);
  if (nparts > 1 && stage_bytes < (size_t)8 * nparts * (size_t)c->part_R) {
    c->part_n = pn;
    c->part_p = pp;
    partition_update(c);
    return ctx_fail(c, BIE_ERR_ARG, "bie_set_partition: stage buffer smaller than 8 nparts R bytes");
  }
  c->exch = nparts > 1 ? exchange : nullptr;
  c->exch_user = nparts > 1 ? user : nullptr;
  c->exch_buf = nparts > 1 ? stage_dev : nullptr;
  c->exch_bytes = nparts > 1 ? stage_bytes : 0;
  // the stored rows change: nothing of an earlier assembly is kept
  c->assembled = false;
  c->transposed = false;
  c->asm_sig = -1;
  return BIE_OK;
}

bie_status bie_partition_rows(const bie_ctx* c, int* row0, int* row1, long long* rows_per_part) {
  if (!c || !row0 || !row1) return BIE_ERR_ARG;
  if (!c->have_geom) return BIE_ERR_STATE;
  *row0 = c->row0;
  *row1 = c->row1;
  if (rows_per_part) *rows_per_part = c->part_R;
  return BIE_OK;
}

bie_status bie_set_flow(bie_ctx* c, double V1, const double* a_host) {
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom) return ctx_fail(c, BIE_ERR_STATE, "bie_set_flow: no geometry");
  if (c->nb > 2 && !a_host) return ctx_fail(c, BIE_ERR_ARG, "bie_set_flow: a_host is NULL");
  if (!std::isfinite(V1)) return ctx_fail(c, BIE_ERR_ARG, "bie_set_flow: V1 not finite");
  c->V1 = V1;
  for (int j = 0; j < BIE_MAXB; ++j) c->a[j] = 0.0;
  for (int j = 2; j < c->nb; ++j) {
    if (!std::isfinite(a_host[j - 2])) return ctx_fail(c, BIE_ERR_ARG, "bie_set_flow: a_j not finite");
    c->a[j - 2] = a_host[j - 2];
  }
  c->have_flow = true;
  return BIE_OK;
}

bie_status bie_assemble(bie_ctx* c, int precision) {
  BIE_NVTX("bie_assemble");
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom) return ctx_fail(c, BIE_ERR_STATE, "bie_assemble: no geometry");
  if (precision < BIE_FP64 || precision > BIE_FP16_IR)
    return ctx_fail(c, BIE_ERR_ARG, "bie_assemble: bad precision");
  cudaSetDevice(c->device);
  c->assembled = false;
  c->transposed = false;
  bie_status s = asm_run(c, precision, 0);
  if (s != BIE_OK) return s;
  c->precision = precision;
  c->variant = 0;
  c->assembled = true;
  return BIE_OK;
}

bie_status bie_assemble_psi(bie_ctx* c, int precision) {
  BIE_NVTX("bie_assemble_psi");
  if (!c) return BIE_ERR_ARG;
  if (partitioned(c)) return refuse_partitioned(c, "bie_assemble_psi");
  if (!c->have_geom) return ctx_fail(c, BIE_ERR_STATE, "bie_assemble_psi: no geometry");
  if (precision < BIE_FP64 || precision > BIE_FP16_IR)
    return ctx_fail(c, BIE_ERR_ARG, "bie_assemble_psi: bad precision");
  cudaSetDevice(c->device);
  c->assembled = false;
  c->transposed = false;
  c->asm_alt = true;
  bie_status s = asm_run(c, precision, 0);
  c->asm_alt = false;
  if (s != BIE_OK) return s;
  c->precision = precision;
  c->variant = 1;
  c->assembled = true;
  return BIE_OK;
}

bie_status bie_rhs(bie_ctx* c, const double* phit_dev, double* b_dev) {
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom || !c->have_flow) return ctx_fail(c, BIE_ERR_STATE, "bie_rhs: geometry/flow missing");
  if (!phit_dev || !b_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_rhs: null pointer");
  cudaSetDevice(c->device);
  return rhs_run(c, phit_dev, b_dev);
}

bie_status bie_matvec(bie_ctx* c, int which, const double* x_dev, double* y_dev) {
  BIE_NVTX("bie_matvec");
  if (!c) return BIE_ERR_ARG;
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_matvec: not assembled");
  if (c->transposed) return ctx_fail(c, BIE_ERR_STATE, "bie_matvec: storage holds the adjoint operator; assemble again");
  if (!x_dev || !y_dev || (which != 0 && which != 1))
    return ctx_fail(c, BIE_ERR_ARG, "bie_matvec: bad argument");
  cudaSetDevice(c->device);
  return gemv_apply(c, which, x_dev, y_dev);
}

bie_status bie_sample_entries(bie_ctx* c, int which, long n, const long long* rows_dev,
                              const long long* cols_dev, double* out_dev) {
  if (!c) return BIE_ERR_ARG;
  if (partitioned(c)) return refuse_partitioned(c, "bie_sample_entries");
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_sample_entries: not assembled");
  if (c->transposed)
    return ctx_fail(c, BIE_ERR_STATE, "bie_sample_entries: storage holds the adjoint operator; assemble again");
  if (n < 0 || (n > 0 && (!rows_dev || !cols_dev || !out_dev)) || (which != 0 && which != 1))
    return ctx_fail(c, BIE_ERR_ARG, "bie_sample_entries: bad argument");
  if (n == 0) return BIE_OK;
  cudaSetDevice(c->device);
  return sample_run(c, which, n, rows_dev, cols_dev, out_dev);
}

bie_status bie_normal_velocity(bie_ctx* c, const double* omega_dev, double* U_dev, double* psi_dev) {
  BIE_NVTX("bie_normal_velocity");
  if (!c) return BIE_ERR_ARG;
  if (!c->have_geom || !c->have_flow) return ctx_fail(c, BIE_ERR_STATE, "bie_normal_velocity: geometry/flow missing");
  if (!omega_dev || !U_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_normal_velocity: null pointer");
  cudaSetDevice(c->device);
  return velocity_run(c, omega_dev, U_dev, psi_dev);
}

bie_status bie_solve(bie_ctx* c, const double* phit_dev, double* omega_dev, double* U_dev,
                     double* psi_dev, const bie_solve_opts* opts, bie_solve_info* info) {
  BIE_NVTX("bie_solve");
  if (!c) return BIE_ERR_ARG;
  if (!c->assembled || !c->have_flow) return ctx_fail(c, BIE_ERR_STATE, "bie_solve: assemble and set_flow first");
  if (c->transposed) return ctx_fail(c, BIE_ERR_STATE, "bie_solve: storage holds the adjoint operator; assemble again");
  if (c->variant != 0) return ctx_fail(c, BIE_ERR_STATE, "bie_solve: storage holds the App. B operator; use bie_solve_psi");
  if (!phit_dev || !omega_dev || !U_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_solve: null pointer");
  bie_solve_opts o;
  bie_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > 1000 || o.max_cycles < 1)
    return ctx_fail(c, BIE_ERR_ARG, "bie_solve: bad options");
  cudaSetDevice(c->device);
  return solve_run(c, phit_dev, omega_dev, U_dev, psi_dev, &o, info);
}

bie_status bie_solve_b(bie_ctx* c, const double* b_dev, double* omega_dev,
                       const bie_solve_opts* opts, bie_solve_info* info) {
  BIE_NVTX("bie_solve_b");
  if (!c) return BIE_ERR_ARG;
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_solve_b: not assembled");
  if (c->transposed) return ctx_fail(c, BIE_ERR_STATE, "bie_solve_b: storage holds the adjoint operator; assemble again");
  if (!b_dev || !omega_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_solve_b: null pointer");
  bie_solve_opts o;
  bie_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > 1000 || o.max_cycles < 1)
    return ctx_fail(c, BIE_ERR_ARG, "bie_solve_b: bad options");
  cudaSetDevice(c->device);
  return solve_system(c, &o, omega_dev, b_dev, info);
}

bie_status bie_solve_psi(bie_ctx* c, const double* phic_dev, const double* psi_dev,
                         double* omega_dev, double* U_dev, double* a_host,
                         const bie_solve_opts* opts, bie_solve_info* info) {
  BIE_NVTX("bie_solve_psi");
  if (!c) return BIE_ERR_ARG;
  if (partitioned(c)) return refuse_partitioned(c, "bie_solve_psi");
  if (!c->assembled || !c->have_flow || c->variant != 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_solve_psi: bie_assemble_psi and bie_set_flow first");
  if (!phic_dev || !psi_dev || !omega_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_solve_psi: null pointer");
  bie_solve_opts o;
  bie_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > 1000 || o.max_cycles < 1)
    return ctx_fail(c, BIE_ERR_ARG, "bie_solve_psi: bad options");
  cudaSetDevice(c->device);
  const int N = c->N, M0 = c->M[0];
  double *b, *a_dev;
  BIE_GET(c, double, "alt_b", N, b);
  BIE_GET(c, double, "alt_a", BIE_MAXB, a_dev);
  bool oom = false;
  const double2* z = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_solve_psi: nodes");
  k_rhs_psi<<<(N + 255) / 256, 256, 0, c->stream>>>(N, M0, c->V1, z, phic_dev, psi_dev, b);
  BIE_LAUNCH_CHECK(c, "k_rhs_psi");
  bie_status ss = solve_system(c, &o, omega_dev, b, info);
  if (ss != BIE_OK && ss != BIE_ERR_NOCONV) return ss;
  // circulations a_j = <1_j, omega> (App. B), then U with them as the flow's a_j
  double a[BIE_MAXB] = {0};
  if (c->nb > 2) {
    bie_status s = psi_run(c, omega_dev, a_dev);
    if (s != BIE_OK) return s;
    BIE_CUDA_TRY(c, cudaMemcpyAsync(a, a_dev, sizeof(double) * (c->nb - 2), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (a_host) memcpy(a_host, a, sizeof(double) * (c->nb - 2));
  }
  if (U_dev) {
    double saved[BIE_MAXB];
    memcpy(saved, c->a, sizeof(saved));
    for (int j = 0; j < c->nb - 2; ++j) c->a[j] = a[j];
    bie_status s = velocity_run(c, omega_dev, U_dev, nullptr);
    memcpy(c->a, saved, sizeof(saved));
    if (s != BIE_OK) return s;
  }
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return ss;
}

bie_status bie_solve_host(bie_ctx* c, int nb, const int* M_host, const double* zeta_host,
                          const double* dzeta_host, const double* d2zeta_host,
                          const double* zc_host, double V1, const double* a_host,
                          const double* phit_host, int precision, const bie_solve_opts* opts,
                          double* omega_host, double* U_host, double* psi_host,
                          bie_solve_info* info) {
  BIE_NVTX("bie_solve_host");
  if (!c) return BIE_ERR_ARG;
  if (nb < 2 || nb > BIE_MAXB || !M_host || !zeta_host || !dzeta_host || !d2zeta_host ||
      !phit_host || !omega_host || !U_host)
    return ctx_fail(c, BIE_ERR_ARG, "bie_solve_host: bad argument");
  long long N = 0;
  for (int k = 0; k < nb; ++k) {
    if (M_host[k] < 8) return ctx_fail(c, BIE_ERR_ARG, "bie_solve_host: M_k < 8");
    N += M_host[k];
  }
  const int M0 = M_host[0];
  cudaSetDevice(c->device);
  double *hz, *hdz, *hd2z, *hphi, *homega, *hU, *hpsi;
  BIE_GET(c, double, "host_in_zeta", 2 * N, hz);
  BIE_GET(c, double, "host_in_dzeta", 2 * N, hdz);
  BIE_GET(c, double, "host_in_d2zeta", 2 * N, hd2z);
  BIE_GET(c, double, "host_in_phit", M0, hphi);
  BIE_GET(c, double, "host_out_omega", N, homega);
  BIE_GET(c, double, "host_out_U", M0, hU);
  BIE_GET(c, double, "host_out_psi", BIE_MAXB, hpsi);
  BIE_CUDA_TRY(c, cudaMemcpyAsync(hz, zeta_host, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(hdz, dzeta_host, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(hd2z, d2zeta_host, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(hphi, phit_host, sizeof(double) * M0, cudaMemcpyHostToDevice, c->stream));
  if (opts && opts->x0)   // the caller's omega is the initial guess
    BIE_CUDA_TRY(c, cudaMemcpyAsync(homega, omega_host, sizeof(double) * N, cudaMemcpyHostToDevice, c->stream));
  bie_status s = bie_set_geometry(c, nb, M_host, hz, hdz, hd2z, zc_host);
  if (s != BIE_OK) return s;
  s = bie_set_flow(c, V1, a_host);
  if (s != BIE_OK) return s;
  s = bie_assemble(c, precision);
  if (s != BIE_OK) return s;
  bie_status ss = bie_solve(c, hphi, homega, hU, hpsi, opts, info);
  if (ss != BIE_OK && ss != BIE_ERR_NOCONV) return ss;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(omega_host, homega, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaMemcpyAsync(U_host, hU, sizeof(double) * M0, cudaMemcpyDeviceToHost, c->stream));
  if (psi_host && nb > 2)
    BIE_CUDA_TRY(c, cudaMemcpyAsync(psi_host, hpsi, sizeof(double) * (nb - 2), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return ss;
}

bie_status bie_set_profiling(bie_ctx* c, int on) {
  if (!c) return BIE_ERR_ARG;
  cudaSetDevice(c->device);
  if (c->profiling) {
    bie_status s = prof_collect(c);
    if (s != BIE_OK) return s;
  }
  c->profiling = on != 0;
  c->prof = bie_profile{};
  c->prof.enabled = c->profiling ? 1 : 0;
  c->launches = 0;
  return BIE_OK;
}

bie_status bie_get_profile(bie_ctx* c, bie_profile* out) {
  if (!c || !out) return BIE_ERR_ARG;
  cudaSetDevice(c->device);
  bie_status s = prof_collect(c);
  if (s != BIE_OK) return s;
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->prof.enabled = c->profiling ? 1 : 0;
  c->prof.kernel_launches = c->launches;
  const double NN = (double)c->N * (double)c->N;
  const int p = c->precision;
  c->prof.bytes_gemv_inner = NN * (p == BIE_FP64 ? 8.0 : p == BIE_FP32_IR ? 4.0 : 2.0);
  c->prof.bytes_gemv_full = NN * 8.0;
  c->prof.bytes_gemv_hi = NN * 4.0;
  *out = c->prof;
  return BIE_OK;
}

}  // extern "C"
