// Assembly of the matrix of eq. lin:sys (step a2) and entry sampling.
//
// Stored value of entry (m, l), row m on boundary k, column l on boundary j:
//   S_ml = M_j * (Table-1 kernel)  -  [k == j >= 2]          (the -E_k term folded in)
// so that A_ml = S_ml / M_j + delta_ml s_m with s_m = -1/2 (surface), +1/2 (solids).
// The kernel F = zeta_l' * 1/2 cot((zeta_l - zeta_m)/2) enters as
//   Im F on blocks (0,0) and (k>=1, j>=1)   (K_kj),
//   Re F on (0, j>=1)                       (G_0j),
//  -Re F on (k>=1, 0)                       (-G_k0),
// and the diagonal is the limit Im{zeta''/(2 zeta')} (Sec. 3.2).
//
// Far field (|d| >= 0.1): separable form of App. E,
//   1/2 cot((zeta_l - zeta_m)/2) = i/2 + i/d,   d = P_l Q_m - 1,
//   P_l = e^{i zeta_l}, Q_m = e^{-i zeta_m}, one complex product per entry.
// Near field (|d| < 0.1, the band around the diagonal and close approaches
// between boundaries): d = e^{i Delta} - 1 is ill-conditioned from P and Q, so
// Delta = zeta_l - zeta_m is formed from the FP64 nodes (reduced mod 2 pi in
// double-double) and d = i Delta E(i Delta) with E(w) = (e^w - 1)/w summed by
// Horner's rule; then i/d = 1/(Delta E).
#include <cstring>

#include "common.cuh"

#define DFC(x) {(float)(x), (float)((x) - (double)(float)(x))}
// 1/(n+1)!, n = 0..11 : Taylor coefficients of E(w) = (e^w - 1)/w
__constant__ float2 c_taylor_df[12] = {
    DFC(1.0), DFC(1.0 / 2.0), DFC(1.0 / 6.0), DFC(1.0 / 24.0), DFC(1.0 / 120.0),
    DFC(1.0 / 720.0), DFC(1.0 / 5040.0), DFC(1.0 / 40320.0), DFC(1.0 / 362880.0),
    DFC(1.0 / 3628800.0), DFC(1.0 / 39916800.0), DFC(1.0 / 479001600.0)};
__constant__ double c_taylor64[12] = {
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

struct AsmArgs {
  int N;
  long long ld;
  const int* blk;
  const double2* z64;
  // double-float node data
  const float4* nP;
  const float4* nQ;
  const float4* nZp;
  const float4* nPQc;   // third words (P.re, P.im, Q.re, Q.im)
  const float2* nDiag;
  // FP64 node data
  const double2* P64;
  const double2* Q64;
  const double2* Zp64;
  const double* diag64;
  // outputs
  float* hi;
  float* lo;
  void* h16;
  int kind16;  // 0 none, 1 fp16, 2 bf16
  double* f64;
  float near2;
};

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
  static __device__ __forceinline__ void store(const AsmArgs& a, size_t idx, dfl v) {
    a.hi[idx] = v.hi;
    a.lo[idx] = v.lo;
    if (a.kind16 == 1) ((__half*)a.h16)[idx] = __float2half_rn(v.hi);
    else if (a.kind16 == 2) ((__nv_bfloat16*)a.h16)[idx] = __float2bfloat16_rn(v.hi);
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
  static __device__ __forceinline__ void store(const AsmArgs& a, size_t idx, double v) {
    a.f64[idx] = v;
  }
};

// One matrix entry S_ml (see the file header).
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

template <class R>
__device__ __forceinline__ R entry_value(const cx<R>& P, const cx<R>& Zp, const cx<R>& Q,
                                         float2 Pc, float2 Qc, double2 zl, double2 zm, int bl,
                                         int bm, bool diag, const R& dval, float near2) {
  const bool isK = ((bm == 0) == (bl == 0));
  R val;
  if (diag) {
    val = dval;
  } else {
    R wr, wi;
    pq_product(P, Q, Pc, Qc, wr, wi);
    const R dr = r_addf(wr, -1.0f);
    const R n2 = r_add(r_sqr(dr), r_sqr(wi));
    if (r_hi(n2) < near2) {
      const cx<R> Rv = near_R<R>(node_delta(zl, zm));
      const R inv = r_rcp(r_add(r_sqr(Rv.re), r_sqr(Rv.im)));
      // F = zeta'(i/2 + conj(R)/|R|^2)
      if (isK) val = r_add(r_half(Zp.re), r_mul(r_sub(r_mul(Zp.im, Rv.re), r_mul(Zp.re, Rv.im)), inv));
      else val = r_add(r_neg(r_half(Zp.im)), r_mul(r_add(r_mul(Zp.re, Rv.re), r_mul(Zp.im, Rv.im)), inv));
    } else {
      const R inv = r_rcp(n2);
      // F = zeta'(i/2 + i conj(d)/|d|^2)
      if (isK) val = r_add(r_half(Zp.re), r_mul(r_add(r_mul(Zp.re, dr), r_mul(Zp.im, wi)), inv));
      else val = r_add(r_neg(r_half(Zp.im)), r_mul(r_sub(r_mul(Zp.re, wi), r_mul(Zp.im, dr)), inv));
    }
    if (bm != 0 && bl == 0) val = r_neg(val);  // -G_k0
  }
  if (bm == bl && bm >= 2) val = r_addf(val, -1.0f);  // -E_k (times M_k)
  return val;
}

template <class R, int ROWS>
__global__ void __launch_bounds__(256) k_assemble(AsmArgs a) {
  __shared__ cx<R> sQ[ROWS];
  __shared__ float2 sQc[ROWS];
  __shared__ R sD[ROWS];
  __shared__ double2 sZ[ROWS];
  __shared__ int sB[ROWS];
  const int m0 = blockIdx.y * ROWS;
  for (int t = threadIdx.x; t < ROWS; t += blockDim.x) {
    const int m = m0 + t;
    if (m < a.N) {
      sQ[t] = NodeLoad<R>::Q(a, m);
      const float4 pq = a.nPQc[m];
      sQc[t] = make_float2(pq.z, pq.w);
      sD[t] = NodeLoad<R>::Diag(a, m);
      sZ[t] = a.z64[m];
      sB[t] = a.blk[m];
    }
  }
  __syncthreads();
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= a.ld) return;
  if (l >= a.N) {  // zero padding columns
    for (int r = 0; r < ROWS; ++r) {
      const int m = m0 + r;
      if (m >= a.N) break;
      NodeLoad<R>::store(a, (size_t)m * a.ld + l, r_from_double<R>(0.0));
    }
    return;
  }
  const int li = (int)l;
  const cx<R> P = NodeLoad<R>::P(a, li);
  const cx<R> Zp = NodeLoad<R>::Zp(a, li);
  const double2 zl = a.z64[li];
  const int bl = a.blk[li];
  const float4 pqc = a.nPQc[li];
  const float2 Pc = make_float2(pqc.x, pqc.y);
  for (int r = 0; r < ROWS; ++r) {
    const int m = m0 + r;
    if (m >= a.N) break;
    const R v = entry_value<R>(P, Zp, sQ[r], Pc, sQc[r], zl, sZ[r], bl, sB[r], m == li, sD[r],
                               a.near2);
    NodeLoad<R>::store(a, (size_t)m * a.ld + l, v);
  }
}

static AsmArgs make_asm_args(bie_ctx* c, bool* oom) {
  AsmArgs a;
  memset(&a, 0, sizeof(a));
  a.N = c->N;
  a.ld = c->ld;
  const long long N = c->N;
  a.blk = (const int*)ctx_buf(c, "blk", sizeof(int) * c->ld, oom);
  a.z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, oom);
  a.nP = (const float4*)ctx_buf(c, "nP", sizeof(float4) * N, oom);
  a.nQ = (const float4*)ctx_buf(c, "nQ", sizeof(float4) * N, oom);
  a.nZp = (const float4*)ctx_buf(c, "nZp", sizeof(float4) * N, oom);
  a.nPQc = (const float4*)ctx_buf(c, "nPQc", sizeof(float4) * N, oom);
  a.nDiag = (const float2*)ctx_buf(c, "nDiag", sizeof(float2) * N, oom);
  a.P64 = (const double2*)ctx_buf(c, "P64", sizeof(double2) * N, oom);
  a.Q64 = (const double2*)ctx_buf(c, "Q64", sizeof(double2) * N, oom);
  a.Zp64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, oom);
  a.diag64 = (const double*)ctx_buf(c, "diag64", sizeof(double) * N, oom);
  a.near2 = 0.01f;
  return a;
}

static const char* kStoreNames[4] = {"A_f64", "A_hi", "A_lo", "A_16"};

bie_status asm_run(bie_ctx* c, int precision) {
  bool oom = false;
  AsmArgs a = make_asm_args(c, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "assemble: node buffers");
  const size_t NN = (size_t)c->N * (size_t)c->ld;
  constexpr int ROWS = 16;
  const dim3 grid((unsigned)(c->ld / 256 + (c->ld % 256 ? 1 : 0)), (unsigned)((c->N + ROWS - 1) / ROWS));
  if (precision == BIE_FP64) {
    a.f64 = (double*)ctx_buf(c, kStoreNames[0], sizeof(double) * NN, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "assemble: FP64 matrix");
    const int pr = prof_begin(c, 2, -1);
    k_assemble<double, ROWS><<<grid, 256, 0, c->stream>>>(a);
    prof_end(c, pr);
    BIE_LAUNCH_CHECK(c, "k_assemble<double>");
  } else {
    a.hi = (float*)ctx_buf(c, kStoreNames[1], sizeof(float) * NN, &oom);
    if (!oom) a.lo = (float*)ctx_buf(c, kStoreNames[2], sizeof(float) * NN, &oom);
    if (!oom && precision != BIE_FP32_IR) a.h16 = ctx_buf(c, kStoreNames[3], 2 * NN, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "assemble: matrix storage");
    a.kind16 = precision == BIE_FP16_IR ? 1 : (precision == BIE_BF16_IR ? 2 : 0);
    const int pr = prof_begin(c, 2, -1);
    k_assemble<dfl, ROWS><<<grid, 256, 0, c->stream>>>(a);
    prof_end(c, pr);
    BIE_LAUNCH_CHECK(c, "k_assemble<dfl>");
  }
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
