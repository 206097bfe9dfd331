// Assembly of the matrix of eq. lin:sys and entry sampling.
//
// Stored value of entry (m, l), row m on boundary k, column l on boundary j:
//   S_ml = M_j * (Table-1 kernel)  -  [k == j >= 2]          (the -E_k term folded in)
// so that A_ml = S_ml / M_j + delta_ml s_m with s_m = -1/2 (surface), +1/2 (solids).
// The kernel F = zeta_l' * 1/2 cot((zeta_l - zeta_m)/2) enters as
//   Im F on blocks (0,0) and (k>=1, j>=1)   (K_kj),
//   Re F on (0, j>=1)                       (G_0j),
//  -Re F on (k>=1, 0)                       (-G_k0),
// and the diagonal is the limit Im{zeta''/(2 zeta')} (Sec. 3.2).
// With `transpose` set the same values are stored as S^T: with W = diag(1/M_j)
// and Sigma = diag(s_m), A^T = W S^T + Sigma = W (S^T W + Sigma) W^{-1}, so the
// solver's operator S W + Sigma applied to S^T solves the adjoint system.
//
// Entries are produced in pairs: the kernel 1/2 cot(x/2) is odd, so the
// (m, l) and (l, m) entries share G = 1/2 cot((zeta_l - zeta_m)/2).
// Far field (|d| >= 0.1): separable form of App. E,
//   1/2 cot((zeta_l - zeta_m)/2) = i/2 + i/d,   d = P_l Q_m - 1,
//   P_l = e^{i zeta_l}, Q_m = e^{-i zeta_m}, one complex product per entry.
// Near field (|d| < 0.1, the band around the diagonal and close approaches
// between boundaries): d = e^{i Delta} - 1 is ill-conditioned from P and Q, so
// Delta = zeta_l - zeta_m is formed from the FP64 nodes (reduced mod 2 pi in
// double-double) and d = i Delta E(i Delta) with E(w) = (e^w - 1)/w summed by
// Horner's rule; then i/d = 1/(Delta E).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "pair_kernel.cuh"

struct AsmArgs {
  int N;
  int M0;
  long long ld;
  int ntile;            // tiles per dimension, ceil(N / ATILE)
  const int* blk;
  const double2* z64;
  // double-float node data
  const float4* nP;
  const float4* nQ;
  const float4* nZp;
  const float4* nPQc;   // third words (P.re, P.im, Q.re, Q.im)
  const float2* nDiag;
  const float2* Ttab;   // 1/2 cot(pi j / M_0), df
  // FP64 node data
  const double2* P64;
  const double2* Q64;
  const double2* Zp64;
  const double* diag64;
  const double* gdiag64;  // Re{zeta''/(2 zeta')} on the surface
  const double* T64;      // 1/2 cot(pi j / M_0), FP64
  // outputs: matrix A (N x ld) and the surface U-matrix V (M_0 x ld)
  float* hi;
  float* lo;
  void* h16;
  int kind16;  // 0 none, 1 fp16, 2 bf16
  double* f64;
  float* Vhi;
  float* Vlo;
  double* Vf64;
  float near2;
  int transpose;   // store S^T (the adjoint operator); the U-matrix is left as it is
  int vs;          // vortex-sheet solid system: every node solid, no -E_k term
  int alt;         // App. B operator (eq. A:alt): u_k(m) on columns of obstacle k, no -E_k
  const float2* ualt;     // u_k(m) as double-float, [k - 2][N]
  const double* ualt64;   // u_k(m), FP64, [k - 2][N]
};

#define ATILE 32

template <class R> struct NodeLoad;
template <> struct NodeLoad<dfl> {
  static __device__ __forceinline__ cx<dfl> P(const AsmArgs& a, int l) {
    const float4 v = a.nP[l];
    return {{v.x, v.y}, {v.z, v.w}};
  }
  static __device__ __forceinline__ cx<dfl> Q(const AsmArgs& a, int l) {
    const float4 v = a.nQ[l];
    return {{v.x, v.y}, {v.z, v.w}};
  }
  static __device__ __forceinline__ cx<dfl> Zp(const AsmArgs& a, int l) {
    const float4 v = a.nZp[l];
    return {{v.x, v.y}, {v.z, v.w}};
  }
  static __device__ __forceinline__ dfl Diag(const AsmArgs& a, int l) {
    const float2 v = a.nDiag[l];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ dfl T(const AsmArgs& a, int j) {
    const float2 v = a.Ttab[j];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ dfl Ualt(const AsmArgs& a, int k, int m) {
    const float2 v = a.ualt[(size_t)(k - 2) * a.N + m];
    return {v.x, v.y};
  }
  // K16: the inner storage kind fixed at compile time (0 none, 1 FP16, 2 BF16)
  template <int K16>
  static __device__ __forceinline__ void storeA(const AsmArgs& a, size_t idx, dfl v) {
    a.hi[idx] = v.hi;
    a.lo[idx] = v.lo;
    if (K16 == 1) ((__half*)a.h16)[idx] = __float2half_rn(v.hi);
    else if (K16 == 2) ((__nv_bfloat16*)a.h16)[idx] = __float2bfloat16_rn(v.hi);
  }
  static __device__ __forceinline__ void storeA(const AsmArgs& a, size_t idx, dfl v) {
    if (a.kind16 == 1) storeA<1>(a, idx, v);
    else if (a.kind16 == 2) storeA<2>(a, idx, v);
    else storeA<0>(a, idx, v);
  }
  static __device__ __forceinline__ void storeV(const AsmArgs& a, size_t idx, dfl v) {
    a.Vhi[idx] = v.hi;
    a.Vlo[idx] = v.lo;
  }
};
template <> struct NodeLoad<double> {
  static __device__ __forceinline__ cx<double> P(const AsmArgs& a, int l) {
    const double2 v = a.P64[l];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ cx<double> Q(const AsmArgs& a, int l) {
    const double2 v = a.Q64[l];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ cx<double> Zp(const AsmArgs& a, int l) {
    const double2 v = a.Zp64[l];
    return {v.x, v.y};
  }
  static __device__ __forceinline__ double Diag(const AsmArgs& a, int l) { return a.diag64[l]; }
  static __device__ __forceinline__ double T(const AsmArgs& a, int j) { return a.T64[j]; }
  static __device__ __forceinline__ double Ualt(const AsmArgs& a, int k, int m) {
    return a.ualt64[(size_t)(k - 2) * a.N + m];
  }
  template <int K16>
  static __device__ __forceinline__ void storeA(const AsmArgs& a, size_t idx, double v) {
    a.f64[idx] = v;
  }
  static __device__ __forceinline__ void storeA(const AsmArgs& a, size_t idx, double v) {
    a.f64[idx] = v;
  }
  static __device__ __forceinline__ void storeV(const AsmArgs& a, size_t idx, double v) {
    a.Vf64[idx] = v;
  }
};

__device__ __forceinline__ void tile_of(int t, int T, int& I, int& J) {
  // upper-triangular tiles (I <= J), row-major: row I holds T - I tiles
  int i = (int)floorf((2.0f * T + 1.0f - sqrtf((2.0f * T + 1.0f) * (2.0f * T + 1.0f) - 8.0f * t)) * 0.5f);
  if (i < 0) i = 0;
  while (i > 0 && i * T - i * (i - 1) / 2 > t) --i;
  while ((i + 1) * T - (i + 1) * i / 2 <= t) ++i;
  I = i;
  J = i + (t - (i * T - i * (i - 1) / 2));
}

// One CTA per tile pair {(I,J), (J,I)}, I <= J.  Each unordered node pair
// (m, l) gives G once; A_ml = component of zeta_l' G, A_lm = component of
// -zeta_m' G (the kernel is odd), and on surface rows the U-matrix entries
//   V_rc = -Im{zeta_r' G_rc} (c off the surface),  T_{r-c} + Re{zeta_r' G_rc}
// (c on the surface; T the Hilbert-regularising term), V_rr = -Re{zeta''/(2 zeta')},
// so that s_alpha U_r = [eq. d:phi:mv] + sum_c V_rc omega_c'/M_c - 1/2 H omega_0'.
// Transposed entries go through shared memory for coalesced stores.
template <class R, int K16>
__global__ void __launch_bounds__(256) k_assemble_pairs(AsmArgs a) {
  __shared__ cx<R> sQ[ATILE];
  __shared__ cx<R> sZr[ATILE];
  __shared__ float2 sQc[ATILE];
  __shared__ double2 sZm[ATILE];
  __shared__ R sD[ATILE];
  __shared__ int sB[ATILE];
  __shared__ R sAT[ATILE][ATILE + 1];
  __shared__ R sVT[ATILE][ATILE + 1];
  int I, J;
  tile_of(blockIdx.x, a.ntile, I, J);
  const int m0 = I * ATILE, l0 = J * ATILE;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x < ATILE) {
    const int m = m0 + threadIdx.x;
    if (m < a.N) {
      sQ[threadIdx.x] = NodeLoad<R>::Q(a, m);
      sZr[threadIdx.x] = NodeLoad<R>::Zp(a, m);
      const float4 pq = a.nPQc[m];
      sQc[threadIdx.x] = make_float2(pq.z, pq.w);
      sZm[threadIdx.x] = a.z64[m];
      sD[threadIdx.x] = NodeLoad<R>::Diag(a, m);
      sB[threadIdx.x] = a.blk[m];
    }
  }
  __syncthreads();
  const int l = l0 + tx;
  const bool lok = l < a.N;
  cx<R> P, Zl;
  float2 Pc = make_float2(0.f, 0.f);
  double2 zl = make_double2(0.0, 0.0);
  int bl = -1;
  if (lok) {
    P = NodeLoad<R>::P(a, l);
    Zl = NodeLoad<R>::Zp(a, l);
    const float4 pq = a.nPQc[l];
    Pc = make_float2(pq.x, pq.y);
    zl = a.z64[l];
    bl = a.blk[l];
  }
  const bool diagTile = (I == J);
#pragma unroll 1
  for (int k = 0; k < ATILE / 8; ++k) {
    const int rm = ty + 8 * k;
    const int m = m0 + rm;
    if (!lok || m >= a.N) continue;
    if (diagTile && rm > tx) continue;
    const int bm = sB[rm];
    const size_t iml = (size_t)m * a.ld + l;
    if (m == l) {
      R dv = sD[rm];
      if (bm >= 2 && a.alt) dv = r_add(dv, NodeLoad<R>::Ualt(a, bm, m));
      else if (bm >= 2 && !a.vs) dv = r_addf(dv, -1.0f);
      NodeLoad<R>::template storeA<K16>(a, iml, dv);
      if (m < a.M0 && !a.transpose) NodeLoad<R>::storeV(a, iml, r_neg(r_from_double<R>(a.gdiag64[m])));
      continue;
    }
    const cx<R> G = half_cot_pair<R>(P, sQ[rm], Pc, sQc[rm], zl, sZm[rm], a.near2);
    const cx<R> Zm = sZr[rm];
    const bool sm = !a.vs && bm == 0, sl = !a.vs && bl == 0;
    R Aml, Alm;
    if (sm == sl) {
      Aml = cim(Zl, G);
      Alm = r_neg(cim(Zm, G));
    } else if (sm) {
      Aml = cre(Zl, G);
      Alm = cre(Zm, G);
    } else {
      Aml = r_neg(cre(Zl, G));
      Alm = r_neg(cre(Zm, G));
    }
    if (a.alt) {   // + u_k(row) on every column of obstacle k (stored times M_k)
      if (bl >= 2) Aml = r_add(Aml, NodeLoad<R>::Ualt(a, bl, m));
      if (bm >= 2) Alm = r_add(Alm, NodeLoad<R>::Ualt(a, bm, l));
    } else if (bm == bl && bm >= 2 && !a.vs) {
      Aml = r_addf(Aml, -1.0f);
      Alm = r_addf(Alm, -1.0f);
    }
    if (a.transpose) {
      const R t = Aml;
      Aml = Alm;
      Alm = t;
    }
    NodeLoad<R>::template storeA<K16>(a, iml, Aml);
    sAT[tx][rm] = Alm;
    if ((sm || sl) && !a.transpose) {
      int tj = 0;
      if (sm && sl) {   // both on the surface: 0 <= m, l < M_0
        tj = m - l;
        if (tj < 0) tj += a.M0;
      }
      if (sm) {  // V_ml
        const R v = sl ? r_add(NodeLoad<R>::T(a, tj), cre(Zm, G)) : r_neg(cim(Zm, G));
        NodeLoad<R>::storeV(a, iml, v);
      }
      if (sl) {  // V_lm
        const R v = sm ? r_sub(NodeLoad<R>::T(a, tj == 0 ? 0 : a.M0 - tj), cre(Zl, G)) : cim(Zl, G);
        sVT[tx][rm] = v;
      }
    }
  }
  __syncthreads();
  // transposed block: rows l0 + rl, columns m0 + cm
  const int cm = tx;
  const int mcol = m0 + cm;
#pragma unroll 1
  for (int k = 0; k < ATILE / 8; ++k) {
    const int rl = ty + 8 * k;
    const int lrow = l0 + rl;
    if (lrow >= a.N || mcol >= a.N) continue;
    if (diagTile && cm >= rl) continue;
    const size_t ilm = (size_t)lrow * a.ld + mcol;
    NodeLoad<R>::template storeA<K16>(a, ilm, sAT[rl][cm]);
    if (lrow < a.M0 && !a.transpose) NodeLoad<R>::storeV(a, ilm, sVT[rl][cm]);
  }
}

// zero the padding columns [N, ld) of A (rows < N) and of V (rows < M0)
template <class R>
__global__ void k_zero_pad(AsmArgs a) {
  const int pad = (int)(a.ld - a.N);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pad <= 0 || t >= (long long)a.N * pad) return;
  const int r = (int)(t / pad);
  const size_t idx = (size_t)r * a.ld + a.N + (int)(t % pad);
  NodeLoad<R>::storeA(a, idx, r_from_double<R>(0.0));
  if (r < a.M0 && !a.transpose) NodeLoad<R>::storeV(a, idx, r_from_double<R>(0.0));
}

// u_k(m) of eq. A:alt: phi_cyl(zeta_m - z_k) = arg(1 - e^{i(zeta_m - z_k)}) on
// surface rows, psi_cyl(zeta_m - z_k) = -ln|1 - e^{i(zeta_m - z_k)}| on solid rows
__global__ void k_alt_columns(int N, int nobs, const int* __restrict__ blk,
                              const double2* __restrict__ z, FlowParams F,
                              float2* __restrict__ u, double* __restrict__ u64) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  const double2 zm = z[m];
  for (int k = 0; k < nobs; ++k) {
    double sn, cs;
    sincos(zm.x - F.zc[k].x, &sn, &cs);
    const double e = exp(-(zm.y - F.zc[k].y));
    const double wr = 1.0 - e * cs, wi = -e * sn;          // 1 - e^{i(z - z_k)}
    const double v = (blk[m] == 0) ? atan2(wi, wr) : -0.5 * log(wr * wr + wi * wi);
    const dfl d = df_from_double(v);
    u[(size_t)k * N + m] = make_float2(d.hi, d.lo);
    u64[(size_t)k * N + m] = v;
  }
}

static AsmArgs make_asm_args(bie_ctx* c, bool* oom) {
  AsmArgs a;
  memset(&a, 0, sizeof(a));
  a.N = c->N;
  a.M0 = c->M[0];
  a.ld = c->ld;
  a.ntile = (c->N + ATILE - 1) / ATILE;
  const long long N = c->N;
  bool o = false;
  auto get = [&](const char* name, size_t bytes) {
    bool x = false;
    void* p = ctx_buf(c, name, bytes, &x);
    o = o || x;
    return p;
  };
  a.blk = (const int*)get("blk", sizeof(int) * c->ld);
  a.z64 = (const double2*)get("zeta", sizeof(double2) * N);
  a.nP = (const float4*)get("nP", sizeof(float4) * N);
  a.nQ = (const float4*)get("nQ", sizeof(float4) * N);
  a.nZp = (const float4*)get("nZp", sizeof(float4) * N);
  a.nPQc = (const float4*)get("nPQc", sizeof(float4) * N);
  a.nDiag = (const float2*)get("nDiag", sizeof(float2) * N);
  a.Ttab = (const float2*)get("Ttab", sizeof(float2) * c->M[0]);
  a.P64 = (const double2*)get("P64", sizeof(double2) * N);
  a.Q64 = (const double2*)get("Q64", sizeof(double2) * N);
  a.Zp64 = (const double2*)get("dzeta", sizeof(double2) * N);
  a.diag64 = (const double*)get("diag64", sizeof(double) * N);
  a.gdiag64 = (const double*)get("gdiag64", sizeof(double) * c->M[0]);
  a.T64 = (const double*)get("T64", sizeof(double) * c->M[0]);
  a.near2 = 0.01f;
  *oom = o;
  return a;
}

static const char* kStoreNames[4] = {"A_f64", "A_hi", "A_lo", "A_16"};

bie_status asm_run(bie_ctx* c, int precision, int transpose) {
  c->asm_count += 1;
  // the solid-solid entries (tile pairs with both tiles past the surface) are
  // still in the storage when the solids and the storage layout are unchanged
  const long long sig = (long long)precision | (long long)(transpose ? 1 : 0) << 3 |
                        (long long)(c->asm_vs ? 1 : 0) << 4 | (long long)(c->asm_alt ? 1 : 0) << 5 |
                        (long long)(c->asm_noE ? 1 : 0) << 6 | (long long)c->nb << 8 |
                        (long long)c->N << 16 | (long long)c->M[0] << 40;
  const bool keep_solids = sig == c->asm_sig && c->asm_solid_version == c->solid_version;
  c->asm_sig = -1;   // set again once this assembly is enqueued
  bool oom = false;
  AsmArgs a = make_asm_args(c, &oom);
  a.transpose = transpose;
  a.vs = c->asm_vs ? 1 : 0;
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "assemble: node buffers");
  if (c->asm_alt && c->nb > 2) {
    const int nobs = c->nb - 2;
    float2* u;
    double* u64;
    BIE_GET(c, float2, "alt_u", (size_t)nobs * c->N, u);
    BIE_GET(c, double, "alt_u64", (size_t)nobs * c->N, u64);
    k_alt_columns<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->N, nobs, a.blk, a.z64,
                                                             make_flow(c), u, u64);
    BIE_LAUNCH_CHECK(c, "k_alt_columns");
    a.alt = 1;
    a.ualt = u;
    a.ualt64 = u64;
  } else if (c->asm_alt) {
    a.alt = 1;   // no obstacles: B alone
  }
  if (c->asm_noE) {   // B alone: the App. B path with all-zero columns
    if (c->nb > 2) {
      const int nobs = c->nb - 2;
      float2* u;
      double* u64;
      BIE_GET(c, float2, "noe_u", (size_t)nobs * c->N, u);
      BIE_GET(c, double, "noe_u64", (size_t)nobs * c->N, u64);
      BIE_CUDA_TRY(c, cudaMemsetAsync(u, 0, sizeof(float2) * (size_t)nobs * c->N, c->stream));
      BIE_CUDA_TRY(c, cudaMemsetAsync(u64, 0, sizeof(double) * (size_t)nobs * c->N, c->stream));
      a.ualt = u;
      a.ualt64 = u64;
    }
    a.alt = 1;
  }
  const size_t NN = (size_t)c->N * (size_t)c->ld;
  const size_t VN = (size_t)c->M[0] * (size_t)c->ld;
  // upper-triangular tile pairs in row-major order: the pairs with row tile
  // I < ceil(M_0 / ATILE) (every pair touching a surface node) come first
  const long long T = a.ntile, tS = std::min<long long>(T, (c->M[0] + ATILE - 1) / ATILE);
  const unsigned ntiles = (unsigned)(keep_solids ? tS * T - tS * (tS - 1) / 2 : T * (T + 1) / 2);
  const long long npad = (long long)c->N * (c->ld - c->N);
  const unsigned gpad = (unsigned)((npad + 255) / 256);
  if (precision == BIE_FP64) {
    a.f64 = (double*)ctx_buf(c, kStoreNames[0], sizeof(double) * NN, &oom);
    if (!oom && !transpose) a.Vf64 = (double*)ctx_buf(c, "V_f64", sizeof(double) * VN, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "assemble: FP64 matrix");
    const int pr = prof_begin(c, 2, -1);
    k_assemble_pairs<double, 0><<<ntiles, 256, 0, c->stream>>>(a);
    prof_end(c, pr);
    BIE_LAUNCH_CHECK(c, "k_assemble_pairs<double>");
    if (npad > 0) {
      k_zero_pad<double><<<gpad, 256, 0, c->stream>>>(a);
      BIE_LAUNCH_CHECK(c, "k_zero_pad<double>");
    }
  } else {
    a.hi = (float*)ctx_buf(c, kStoreNames[1], sizeof(float) * NN, &oom);
    if (!oom) a.lo = (float*)ctx_buf(c, kStoreNames[2], sizeof(float) * NN, &oom);
    if (!oom && precision != BIE_FP32_IR) a.h16 = ctx_buf(c, kStoreNames[3], 2 * NN, &oom);
    if (!oom && !transpose) a.Vhi = (float*)ctx_buf(c, "V_hi", sizeof(float) * VN, &oom);
    if (!oom && !transpose) a.Vlo = (float*)ctx_buf(c, "V_lo", sizeof(float) * VN, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "assemble: matrix storage");
    a.kind16 = precision == BIE_FP16_IR ? 1 : (precision == BIE_BF16_IR ? 2 : 0);
    const int pr = prof_begin(c, 2, -1);
    if (a.kind16 == 1) k_assemble_pairs<dfl, 1><<<ntiles, 256, 0, c->stream>>>(a);
    else if (a.kind16 == 2) k_assemble_pairs<dfl, 2><<<ntiles, 256, 0, c->stream>>>(a);
    else k_assemble_pairs<dfl, 0><<<ntiles, 256, 0, c->stream>>>(a);
    prof_end(c, pr);
    BIE_LAUNCH_CHECK(c, "k_assemble_pairs<dfl>");
    if (npad > 0) {
      k_zero_pad<dfl><<<gpad, 256, 0, c->stream>>>(a);
      BIE_LAUNCH_CHECK(c, "k_zero_pad<dfl>");
    }
  }
  c->asm_sig = sig;
  c->asm_solid_version = c->solid_version;
  return BIE_OK;
}

// ---------------------------------------------------------------------------
// entry sampling: A[r, c] = S / M_j + delta * s_m, from the chosen storage
// ---------------------------------------------------------------------------
__global__ void k_sample(int n, long long N, long long ld, int prec, int which,
                         const long long* __restrict__ rows, const long long* __restrict__ cols,
                         const double* __restrict__ f64, const float* __restrict__ hi,
                         const float* __restrict__ lo, const void* __restrict__ h16,
                         const double* __restrict__ wgt64, const float* __restrict__ sgn,
                         double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long r = rows[i], cc = cols[i];
  if (r < 0 || r >= N || cc < 0 || cc >= N) {
    out[i] = nan("");
    return;
  }
  const size_t idx = (size_t)r * ld + cc;
  double s;
  if (prec == BIE_FP64) s = f64[idx];
  else if (which == 1) s = (double)hi[idx] + (double)lo[idx];
  else if (prec == BIE_FP32_IR) s = (double)hi[idx];
  else if (prec == BIE_FP16_IR) s = (double)__half2float(((const __half*)h16)[idx]);
  else s = (double)__bfloat162float(((const __nv_bfloat16*)h16)[idx]);
  double v = s * wgt64[cc];
  if (r == cc) v += (double)sgn[r];
  out[i] = v;
}

bie_status sample_run(bie_ctx* c, int which, long n, const long long* rows, const long long* cols,
                      double* out) {
  bool oom = false;
  const size_t NN = (size_t)c->N * (size_t)c->ld;
  const double* f64 = nullptr;
  const float *hi = nullptr, *lo = nullptr;
  const void* h16 = nullptr;
  if (c->precision == BIE_FP64) f64 = (const double*)ctx_buf(c, kStoreNames[0], sizeof(double) * NN, &oom);
  else {
    hi = (const float*)ctx_buf(c, kStoreNames[1], sizeof(float) * NN, &oom);
    lo = (const float*)ctx_buf(c, kStoreNames[2], sizeof(float) * NN, &oom);
    if (c->precision != BIE_FP32_IR) h16 = ctx_buf(c, kStoreNames[3], 2 * NN, &oom);
  }
  const double* wgt64 = (const double*)ctx_buf(c, "wgt64", sizeof(double) * c->ld, &oom);
  const float* sgn = (const float*)ctx_buf(c, "sgn", sizeof(float) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "sample: buffers");
  k_sample<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
      (int)n, c->N, c->ld, c->precision, which, rows, cols, f64, hi, lo, h16, wgt64, sgn, out);
  BIE_LAUNCH_CHECK(c, "k_sample");
  return BIE_OK;
}
