// Matrix-vector products with the stored operator of eq. lin:sys:
//   y_m = sum_l S_ml x_l / M_l + s_m x_m,        s_m = -1/2 (surface) or +1/2,
// optionally followed by the row sign flip of the surface block.
//
// All three variants stream the row-major matrix once from HBM (16-byte
// cache-streaming loads, one warp per row, rows interleaved across CTAs so
// that the last partial wave is spread over all SMs) against a copy of
// x_l / M_l staged in shared memory:
//   k_gemv_lowp  : FP32 / FP16 / BF16 storage, FP32 accumulation (inner GMRES)
//   k_gemv_hilo  : FP32 hi + FP32 lo storage and double-float x, double-float
//                  accumulation on the FP32 pipes (~48-bit residuals)
//   k_gemv_f64   : FP64 storage, FP64 FMA (the plain FP64 scheme)
#include <algorithm>
#include <cstring>

#include "common.cuh"

#include "gemv_dot.cuh"

// ---------------------------------------------------------------------------
// low-precision GEMV: y = D (A x) in FP32, single column panel (ld <= 56K)
// ---------------------------------------------------------------------------
template <class TA, int U>
__global__ void __launch_bounds__(1024, 1)
    k_gemv_lowp(const TA* __restrict__ A, long long ld, int N, int r0, int nrows,
                const float* __restrict__ x, const float* __restrict__ wgt,
                const float* __restrict__ sgn, const int* __restrict__ blk, int rowflip,
                float* __restrict__ y, const int* __restrict__ skip, const float* __restrict__ Vk,
                const float* __restrict__ Ck, int qk, int jdots, double* __restrict__ part1,
                int staged, RightDefl df) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float xs[];
  // optional Gram-Schmidt dots: part1[i][cta] = sum over this CTA's rows of
  // Q_i[m] y_m for i <= jdots and of y_m^2 for i = jdots + 1, with the basis
  // Q_i = C_i (i < qk), V_{i - qk} (i >= qk) (lanes own i = lane, lane + 32)
  __shared__ double red[32][2 * 32 + 1];
  __shared__ float s_xc[BIE_MAXB];   // 3/2 x mean over obstacle k (the product takes P x)
  double d0 = 0.0, d1 = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool defl = df.part != nullptr && df.nobs > 0;
  // the means of x over the obstacles, in a fixed order: the partial sums are
  // loaded before the staging of x and added after it, so their latency hides
  double pv[BIE_NPART / 32];
  const bool mwarp = defl && warp < df.nobs;
  if (mwarp) {
    const double* prow = df.part + (size_t)warp * BIE_PSTRIDE;
#pragma unroll
    for (int q = 0; q < BIE_NPART / 32; ++q) pv[q] = prow[lane + 32 * q];
  }
  {   // x / M_l staged as 16-byte vectors (ld is a multiple of 64), entries past N zero
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* w4 = reinterpret_cast<const float4*>(wgt);
    float4* xs4 = reinterpret_cast<float4*>(xs);
    const int nv4 = (int)(ld >> 2);
#pragma unroll 4
    for (int c = threadIdx.x; c < nv4; c += blockDim.x) {
      const float4 xa = x4[c], wa = w4[c];
      const int e = 4 * c;
      float4 o;
      o.x = e < N ? xa.x * wa.x : 0.f;
      o.y = e + 1 < N ? xa.y * wa.y : 0.f;
      o.z = e + 2 < N ? xa.z * wa.z : 0.f;
      o.w = e + 3 < N ? xa.w * wa.w : 0.f;
      xs4[c] = o;
    }
  }
  if (mwarp) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < BIE_NPART / 32; ++q) t += pv[q];
    t = warp_sum(t);
    const double mu = t * (double)df.invM[warp];
    if (lane == 0) {
      s_xc[warp] = (float)((double)df.coef * mu);
      if (blockIdx.x == 0 && df.mean_out) df.mean_out[warp] = mu;
    }
  }
  __syncthreads();
  if (defl) {   // staged columns of P x: obstacle k's entries lower by 3/2 mu_k / M_k
    for (int k = 0; k < df.nobs; ++k) {
      const float cw = s_xc[k] * df.invM[k];
      for (int c = df.off[k] + threadIdx.x; c < df.off[k + 1]; c += blockDim.x) xs[c] -= cw;
    }
    __syncthreads();
  }
  constexpr int E = Dot16<TA>::E;
  const int nvec = (int)(ld / E);
  // stored rows r0 .. r0 + nrows - 1 (row r0 + ml at ml ld; all rows unless
  // the context is row-partitioned); this CTA takes the chunk ml in
  // [c0, c1), c0 = blockIdx.x R, its warps rows c0 + warp, c0 + warp + 32, ...
  const int R = (nrows + (int)gridDim.x - 1) / (int)gridDim.x;
  const int c0 = blockIdx.x * R, c1 = min(nrows, c0 + R);
  // the basis entries of the chunk's rows for the dots, staged in shared
  // memory after x (sQ[i][t] = Q_i[r0 + c0 + t], Q_i = C_i (i < qk), V_{i-qk})
  // (staged == 0: too large for shared memory, the entries come from L2)
  float* sQ = xs + ld;
  if (part1 && staged) {
    for (int i = warp; i <= jdots; i += (int)(blockDim.x >> 5)) {
      const float* qi = i < qk ? Ck + (size_t)i * ld : Vk + (size_t)(i - qk) * ld;
      for (int t = lane; t < c1 - c0; t += 32) sQ[i * R + t] = qi[r0 + c0 + t];
    }
    __syncthreads();
  }
  const float* vq0 = nullptr;
  const float* vq1 = nullptr;
  if (part1 && !staged) {
    if (lane <= jdots) vq0 = lane < qk ? Ck + (size_t)lane * ld : Vk + (size_t)(lane - qk) * ld;
    if (lane + 32 <= jdots)
      vq1 = lane + 32 < qk ? Ck + (size_t)(lane + 32) * ld : Vk + (size_t)(lane + 32 - qk) * ld;
  }
  for (int ml = c0 + warp; ml < c1; ml += (int)(blockDim.x >> 5)) {
    const int m = r0 + ml;
    const uint4* row = reinterpret_cast<const uint4*>(A + (size_t)ml * ld);
    float acc = 0.f;
    int v = lane;
    for (; v + 32 * (U - 1) < nvec; v += 32 * U) {
      uint4 q[U];
#pragma unroll
      for (int u = 0; u < U; ++u) q[u] = __ldcs(row + v + 32 * u);
#pragma unroll
      for (int u = 0; u < U; ++u) acc = Dot16<TA>::run(acc, q[u], xs + (size_t)(v + 32 * u) * E);
    }
    for (; v < nvec; v += 32) acc = Dot16<TA>::run(acc, __ldcs(row + v), xs + (size_t)v * E);
    acc = warp_sum(acc);
    float xm = x[m];
    if (defl && m >= df.obs0) {   // (P x)_m on an obstacle row
      int k = 0;
      while (k + 1 < df.nobs && m >= df.off[k + 1]) ++k;
      xm -= s_xc[k];
    }
    float r = fmaf(sgn[m], xm, acc);
    if (rowflip && blk[m] == 0) r = -r;
    if (lane == 0) y[m] = r;
    if (part1) {
      const int t = ml - c0;
      if (lane <= jdots + 1) {
        const float q0 = lane <= jdots ? (staged ? sQ[lane * R + t] : vq0[m]) : r;
        d0 += (double)q0 * (double)r;
      }
      if (lane + 32 <= jdots + 1) {
        const float q1 = lane + 32 <= jdots ? (staged ? sQ[(lane + 32) * R + t] : vq1[m]) : r;
        d1 += (double)q1 * (double)r;
      }
    }
  }
  if (part1) {
    red[warp][lane] = d0;
    red[warp][lane + 32] = d1;
    __syncthreads();
    if (threadIdx.x <= jdots + 1) {
      double s = 0.0;
      for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) s += red[w2][threadIdx.x];
      part1[(size_t)threadIdx.x * BIE_PSTRIDE + blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// hi + lo GEMV in double-float: ypart[p][m] = sum_{l in panel p} (hi+lo)_ml xs_l
// ---------------------------------------------------------------------------
template <int U, bool LO>
__global__ void __launch_bounds__(1024, 1)
    k_gemv_hilo(const float* __restrict__ Ahi, const float* __restrict__ Alo, long long ld, int r0,
                int nrows, int panel, const float* __restrict__ xh, const float* __restrict__ xl,
                double* __restrict__ ypart, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float sm[];
  const long long c0 = (long long)blockIdx.y * panel;
  const int pw = (int)min((long long)panel, ld - c0);
  float* sh = sm;
  float* sl = sm + panel;
  {   // 16-byte copies (panel, pw and c0 are multiples of 64)
    const float4* gh = reinterpret_cast<const float4*>(xh + c0);
    const float4* gl = reinterpret_cast<const float4*>(xl + c0);
    float4* s4h = reinterpret_cast<float4*>(sh);
    float4* s4l = reinterpret_cast<float4*>(sl);
#pragma unroll 4
    for (int c = threadIdx.x; c < (pw >> 2); c += blockDim.x) {
      s4h[c] = gh[c];
      s4l[c] = gl[c];
    }
  }
  __syncthreads();
  const int nvec = pw / 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int GW = (blockDim.x >> 5) * gridDim.x;
  const float4* xh4 = reinterpret_cast<const float4*>(sh);
  const float4* xl4 = reinterpret_cast<const float4*>(sl);
  for (int ml = warp * gridDim.x + blockIdx.x; ml < nrows; ml += GW) {
    const int m = r0 + ml;
    const float4* rh = reinterpret_cast<const float4*>(Ahi + (size_t)ml * ld + c0);
    const float4* rl = reinterpret_cast<const float4*>(Alo + (size_t)ml * ld + c0);
    // products and short runs (4U elements) in double-float, each run flushed
    // into an FP64 accumulator: a single 48-bit running sum would lose
    // ~sqrt(n) 2^-49 of the row scale over the n = N/32 terms of a lane
    double acc = 0.0;
    int v = lane;
    for (; v + 32 * (U - 1) < nvec; v += 32 * U) {
      float4 a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = __ldcs(rh + v + 32 * u);
        b[u] = LO ? __ldcs(rl + v + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      dfl run = {0.f, 0.f};
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float4 h = xh4[v + 32 * u], l = xl4[v + 32 * u];
        run = df_acc_prod(run, a[u].x, b[u].x, h.x, l.x);
        run = df_acc_prod(run, a[u].y, b[u].y, h.y, l.y);
        run = df_acc_prod(run, a[u].z, b[u].z, h.z, l.z);
        run = df_acc_prod(run, a[u].w, b[u].w, h.w, l.w);
      }
      acc += (double)run.hi + (double)run.lo;
    }
    for (; v < nvec; v += 32) {
      const float4 a = __ldcs(rh + v);
      const float4 b = LO ? __ldcs(rl + v) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 h = xh4[v], l = xl4[v];
      dfl run = {0.f, 0.f};
      run = df_acc_prod(run, a.x, b.x, h.x, l.x);
      run = df_acc_prod(run, a.y, b.y, h.y, l.y);
      run = df_acc_prod(run, a.z, b.z, h.z, l.z);
      run = df_acc_prod(run, a.w, b.w, h.w, l.w);
      acc += (double)run.hi + (double)run.lo;
    }
    acc = warp_sum(acc);
    if (lane == 0) ypart[(size_t)blockIdx.y * ld + m] = acc;
  }
}

// ---------------------------------------------------------------------------
// FP64 GEMV: ypart[p][m] = sum_{l in panel p} A_ml xs_l
// ---------------------------------------------------------------------------
template <int U>
__global__ void __launch_bounds__(1024, 1)
    k_gemv_f64(const double* __restrict__ A, long long ld, int r0, int nrows, int ncols, int panel,
               const double* __restrict__ x, const double* __restrict__ wgt64,
               double* __restrict__ ypart, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) double smd[];
  const long long c0 = (long long)blockIdx.y * panel;
  const int pw = (int)min((long long)panel, ld - c0);
  for (int c = threadIdx.x; c < pw; c += blockDim.x) {
    const long long cc = c0 + c;
    smd[c] = (cc < ncols) ? x[cc] * wgt64[cc] : 0.0;
  }
  __syncthreads();
  const int nvec = pw / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int GW = (blockDim.x >> 5) * gridDim.x;
  const double2* x2 = reinterpret_cast<const double2*>(smd);
  for (int ml = warp * gridDim.x + blockIdx.x; ml < nrows; ml += GW) {
    const int m = r0 + ml;
    const double2* row = reinterpret_cast<const double2*>(A + (size_t)ml * ld + c0);
    // 2U independent partial sums (fewer additions per accumulator)
    double acc[2 * U];
#pragma unroll
    for (int u = 0; u < 2 * U; ++u) acc[u] = 0.0;
    int v = lane;
    for (; v + 32 * (U - 1) < nvec; v += 32 * U) {
      double2 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = __ldcs(row + v + 32 * u);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const double2 b = x2[v + 32 * u];
        acc[2 * u] = fma(a[u].x, b.x, acc[2 * u]);
        acc[2 * u + 1] = fma(a[u].y, b.y, acc[2 * u + 1]);
      }
    }
    for (; v < nvec; v += 32) {
      const double2 a = __ldcs(row + v), b = x2[v];
      acc[0] = fma(a.x, b.x, acc[0]);
      acc[1] = fma(a.y, b.y, acc[1]);
    }
    double tot = 0.0;
#pragma unroll
    for (int u = 0; u < 2 * U; ++u) tot += acc[u];
    tot = warp_sum(tot);
    if (lane == 0) ypart[(size_t)blockIdx.y * ld + m] = tot;
  }
}

// x (FP64) -> x_l / M_l as double-float, zero-padded to ld
__global__ void k_prep_x_df(int N, long long ld, const double* __restrict__ x,
                            const double* __restrict__ wgt64, float* __restrict__ xh,
                            float* __restrict__ xl, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= ld) return;
  double v = (l < N) ? x[l] * wgt64[l] : 0.0;
  const dfl d = df_from_double(v);
  xh[l] = d.hi;
  xl[l] = d.lo;
}

// Finish: y_m = sum_p ypart[p][m] + s_m x_m ; out = D (b - y) or D y ;
// optional per-slice partial sums of out^2 (slice c = rows [q0 + c S, q0 + (c+1) S)).
__global__ void k_gemv_finish(int q0, int q1, long long ld, int npanel, const double* __restrict__ ypart,
                              const double* __restrict__ x, const float* __restrict__ sgn,
                              const int* __restrict__ blk, int rowflip,
                              const double* __restrict__ b, double* __restrict__ outd,
                              float* __restrict__ outf, double* __restrict__ part_norm,
                              const int* __restrict__ skip, const double* __restrict__ Vk,
                              int jdots, double* __restrict__ part1) {
  if (skip && *skip) return;
  // rows q0 .. q1 - 1 (all rows unless the context is row-partitioned)
  const int S = (q1 - q0 + (int)gridDim.x - 1) / (int)gridDim.x;
  const int r0 = q0 + blockIdx.x * S, r1 = min(q1, r0 + S);
  double acc = 0.0;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
    double y = 0.0;
    for (int p = 0; p < npanel; ++p) y += ypart[(size_t)p * ld + m];
    y += (double)sgn[m] * x[m];
    double o = b ? b[m] - y : y;
    if (rowflip && blk[m] == 0) o = -o;
    if (outd) outd[m] = o;
    if (outf) outf[m] = (float)o;
    acc += o * o;
  }
  if (part1) {  // Gram-Schmidt dots over this slice (FP64 Arnoldi): V_i^T out, |out|^2
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i <= jdots + 1; i += nw) {
      const double* vi = i <= jdots ? Vk + (size_t)i * ld : outd;
      double s = 0.0;
      for (int m = r0 + lane; m < r1; m += 32) s += vi[m] * outd[m];
      s = warp_sum(s);
      if (lane == 0) part1[(size_t)i * BIE_PSTRIDE + blockIdx.x] = s;
    }
  }
  if (part_norm) {
    __shared__ double red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      v = warp_sum(v);
      if (threadIdx.x == 0) part_norm[blockIdx.x] = v;
    }
  }
}

__global__ void k_d2f(int n, long long ld, const double* __restrict__ x, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) y[i] = (i < n) ? (float)x[i] : 0.f;
}
__global__ void k_f2d(int n, const float* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
int gemv_num_ctas();

int gemv_num_ctas() {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  return nsm;
}

// Threads per CTA for a row-streaming product whose CTA takes rows_per_cta rows
// one warp per row: 24..32 warps, the count that minimises rounds x warps (the
// time of a bandwidth-bound CTA whose last round of rows would otherwise run
// with few warps, e.g. 108 rows: 27 warps x 4 rounds instead of 32 x 4 with
// the last round a third full); ties go to more warps.
int gemv_balanced_threads(long long rows_per_cta) {
  if (rows_per_cta <= 0) return 1024;
  int best = 32;
  long long best_cost = ((rows_per_cta + 31) / 32) * 32;
  for (int nw = 31; nw >= 24; --nw) {
    const long long cost = ((rows_per_cta + nw - 1) / nw) * nw;
    if (cost < best_cost) {
      best_cost = cost;
      best = nw;
    }
  }
  return 32 * best;
}

static const int kPanelHilo = 16384;
static const int kPanelF64 = 16384;
static const long long kMaxLdLowp = 56 * 1024;
// dynamic shared memory the inner product may take (of 227 KB per CTA, less
// the 16.8 KB of static reduction space)
static const size_t kGemvSmemMax = 208 * 1024;

// low-precision product: y = D A x (x, y FP32 vectors of length ld)
bie_status gemv_lowp_run_skip(bie_ctx* c, const float* x, float* y, int rowflip, const int* skip,
                              const float* Vk, const float* Ck, int qk, int jdots, double* part1,
                              int* nparts, const RightDefl* defl) {
  RightDefl df;
  if (defl) df = *defl;
  else {
    memset(&df, 0, sizeof(df));
    df.obs0 = c->N;
  }
  const size_t NN = (size_t)local_rows(c) * (size_t)c->ld;
  const int r0 = c->row0, nr = local_rows(c);
  bool oom = false;
  const float* wgt = (const float*)ctx_buf(c, "wgt", sizeof(float) * c->ld, &oom);
  const float* sgn = (const float*)ctx_buf(c, "sgn", sizeof(float) * c->ld, &oom);
  const int* blk = (const int*)ctx_buf(c, "blk", sizeof(int) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv: node buffers");
  if (c->ld > kMaxLdLowp) return ctx_fail(c, BIE_ERR_ARG, "gemv: N too large for the low-precision path");
  const int grid = gemv_num_ctas();
  // x, then (when it fits) the basis entries of each CTA's chunk of rows
  const int Rchunk = (nr + grid - 1) / grid;
  const size_t xbytes = sizeof(float) * c->ld;
  const size_t qbytes = part1 ? sizeof(float) * (size_t)(jdots + 1) * Rchunk : 0;
  const int staged = (part1 && xbytes + qbytes <= kGemvSmemMax) ? 1 : 0;
  const size_t smem = xbytes + (staged ? qbytes : 0);
  const int nt = gemv_balanced_threads(Rchunk);
  if (c->precision == BIE_FP32_IR) {
    const float* A = (const float*)ctx_buf(c, "A_hi", sizeof(float) * NN, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv: A_hi");
    auto kern = k_gemv_lowp<float, 4>;
    BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
    kern<<<grid, nt, smem, c->stream>>>(A, c->ld, c->N, r0, nr, x, wgt, sgn, blk, rowflip, y, skip,
                                          Vk, Ck, qk, jdots, part1, staged, df);
  } else if (c->precision == BIE_FP16_IR) {
    const __half* A = (const __half*)ctx_buf(c, "A_16", 2 * NN, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv: A_16");
    auto kern = k_gemv_lowp<__half, 4>;
    BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
    kern<<<grid, nt, smem, c->stream>>>(A, c->ld, c->N, r0, nr, x, wgt, sgn, blk, rowflip, y, skip,
                                          Vk, Ck, qk, jdots, part1, staged, df);
  } else if (c->precision == BIE_BF16_IR) {
    const __nv_bfloat16* A = (const __nv_bfloat16*)ctx_buf(c, "A_16", 2 * NN, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv: A_16");
    auto kern = k_gemv_lowp<__nv_bfloat16, 4>;
    BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
    kern<<<grid, nt, smem, c->stream>>>(A, c->ld, c->N, r0, nr, x, wgt, sgn, blk, rowflip, y, skip,
                                          Vk, Ck, qk, jdots, part1, staged, df);
  } else {
    return ctx_fail(c, BIE_ERR_STATE, "gemv: no low-precision storage");
  }
  BIE_LAUNCH_CHECK(c, "k_gemv_lowp");
  if (nparts) *nparts = grid;
  return BIE_OK;
}

// full-accuracy product into panel partials: ypart[p][m]; x FP64 (length N)
bie_status gemv_full_partials_skip(bie_ctx* c, const double* x, double** ypart_out, int* npanel_out,
                                   const int* skip, int hi_only) {
  const size_t NN = (size_t)local_rows(c) * (size_t)c->ld;
  const int r0 = c->row0, nr = local_rows(c);
  bool oom = false;
  const double* wgt64 = (const double*)ctx_buf(c, "wgt64", sizeof(double) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv: node buffers");
  const int grid0 = gemv_num_ctas();
  if (c->precision == BIE_FP64) {
    const int npanel = (int)((c->ld + kPanelF64 - 1) / kPanelF64);
    const double* A = (const double*)ctx_buf(c, "A_f64", sizeof(double) * NN, &oom);
    double* ypart = (double*)ctx_buf(c, "ypart", sizeof(double) * c->ld * npanel, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv: f64 buffers");
    const int panel = (int)std::min<long long>(kPanelF64, c->ld);
    const size_t smem = sizeof(double) * panel;
    auto kern = k_gemv_f64<2>;
    BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
    kern<<<dim3(grid0, npanel), gemv_balanced_threads((nr + grid0 - 1) / grid0), smem, c->stream>>>(
        A, c->ld, r0, nr, c->N, panel, x, wgt64, ypart, skip);
    BIE_LAUNCH_CHECK(c, "k_gemv_f64");
    *ypart_out = ypart;
    *npanel_out = npanel;
    return BIE_OK;
  }
  const int npanel = (int)((c->ld + kPanelHilo - 1) / kPanelHilo);
  const float* Ahi = (const float*)ctx_buf(c, "A_hi", sizeof(float) * NN, &oom);
  const float* Alo = (const float*)ctx_buf(c, "A_lo", sizeof(float) * NN, &oom);
  float* xh = (float*)ctx_buf(c, "xs_hi", sizeof(float) * c->ld, &oom);
  float* xl = (float*)ctx_buf(c, "xs_lo", sizeof(float) * c->ld, &oom);
  double* ypart = (double*)ctx_buf(c, "ypart", sizeof(double) * c->ld * npanel, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv: hilo buffers");
  k_prep_x_df<<<(unsigned)((c->ld + 255) / 256), 256, 0, c->stream>>>(c->N, c->ld, x, wgt64, xh, xl, skip);
  BIE_LAUNCH_CHECK(c, "k_prep_x_df");
  const int panel = (int)std::min<long long>(kPanelHilo, c->ld);
  const size_t smem = 2 * sizeof(float) * panel;
  // hi_only: the FP32 part alone (about 2^-24/sqrt(N) of the row scale, enough
  // for an early refinement residual that is still far above the target)
  // (the FP32 part alone reads half the bytes per row: eight 16-byte loads in
  // flight per lane instead of four hi + four lo)
  auto kern = hi_only ? k_gemv_hilo<8, false> : k_gemv_hilo<4, true>;
  BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
  kern<<<dim3(grid0, npanel), gemv_balanced_threads((nr + grid0 - 1) / grid0), smem, c->stream>>>(
      Ahi, Alo, c->ld, r0, nr, panel, xh, xl, ypart, skip);
  BIE_LAUNCH_CHECK(c, "k_gemv_hilo");
  *ypart_out = ypart;
  *npanel_out = npanel;
  return BIE_OK;
}

// out = D (b - A x) (b != NULL) or D A x, plus optional slice partial norms
bie_status gemv_full_finish_skip(bie_ctx* c, const double* ypart, int npanel, const double* x,
                                 int rowflip, const double* b, double* outd, float* outf,
                                 double* part_norm, const int* skip, const double* Vk, int jdots,
                                 double* part1) {
  bool oom = false;
  const float* sgn = (const float*)ctx_buf(c, "sgn", sizeof(float) * c->ld, &oom);
  const int* blk = (const int*)ctx_buf(c, "blk", sizeof(int) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "gemv finish: node buffers");
  k_gemv_finish<<<BIE_NPART, 256, 0, c->stream>>>(c->row0, c->row1, c->ld, npanel, ypart, x, sgn, blk,
                                                   rowflip, b, outd, outf, part_norm, skip, Vk, jdots,
                                                   part1);
  BIE_LAUNCH_CHECK(c, "k_gemv_finish");
  return BIE_OK;
}

bie_status gemv_apply(bie_ctx* c, int which, const double* x, double* y) {
  bool oom = false;
  if (which == 1 || c->precision == BIE_FP64) {
    double* ypart = nullptr;
    int npanel = 0;
    bie_status s = gemv_full_partials_skip(c, x, &ypart, &npanel, nullptr, 0);
    if (s != BIE_OK) return s;
    s = gemv_full_finish_skip(c, ypart, npanel, x, 0, nullptr, y, nullptr, nullptr, nullptr,
                              nullptr, 0, nullptr);
    if (s != BIE_OK) return s;
    return part_allgather(c, y, 8, c->N);   // the other parts' rows
  }
  float* xf = (float*)ctx_buf(c, "mv_xf", sizeof(float) * c->ld, &oom);
  float* yf = (float*)ctx_buf(c, "mv_yf", sizeof(float) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "matvec: buffers");
  k_d2f<<<(unsigned)((c->ld + 255) / 256), 256, 0, c->stream>>>(c->N, c->ld, x, xf);
  BIE_LAUNCH_CHECK(c, "k_d2f");
  bie_status s = gemv_lowp_run_skip(c, xf, yf, 0, nullptr, nullptr, nullptr, 0, 0, nullptr, nullptr,
                                    nullptr);
  if (s != BIE_OK) return s;
  s = part_allgather(c, yf, 4, c->N);   // the other parts' rows
  if (s != BIE_OK) return s;
  k_f2d<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->N, yf, y);
  BIE_LAUNCH_CHECK(c, "k_f2d");
  return BIE_OK;
}

// y[m] = sum_c V_mc x_c / M_c over the M_0 surface rows of the U matrix:
// hi + lo storage with x given as double-float (xh, xl, already divided by
// M_c), or FP64 storage with x = omega' (divided by M_c here).
bie_status vgemv_run(bie_ctx* c, const float* xh, const float* xl, const double* x64,
                     double** ypart_out, int* npanel_out) {
  bool oom = false;
  // surface rows [row0, row0 + nv) of the U-matrix held here (all M_0 unless partitioned)
  const int nv = local_vrows(c);
  const size_t VN = (size_t)nv * (size_t)c->ld;
  const int grid0 = gemv_num_ctas();
  if (c->precision == BIE_FP64) {
    const int npanel = (int)((c->ld + kPanelF64 - 1) / kPanelF64);
    const double* V = (const double*)ctx_buf(c, "V_f64", sizeof(double) * VN, &oom);
    const double* wgt64 = (const double*)ctx_buf(c, "wgt64", sizeof(double) * c->ld, &oom);
    double* ypart = (double*)ctx_buf(c, "vypart", sizeof(double) * c->ld * npanel, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "vgemv: buffers");
    const int panel = (int)std::min<long long>(kPanelF64, c->ld);
    const size_t smem = sizeof(double) * panel;
    auto kern = k_gemv_f64<2>;
    BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
    kern<<<dim3(grid0, npanel), gemv_balanced_threads((nv + grid0 - 1) / grid0), smem, c->stream>>>(
        V, c->ld, c->row0, nv, c->N, panel, x64, wgt64, ypart, nullptr);
    BIE_LAUNCH_CHECK(c, "k_gemv_f64 (U)");
    *ypart_out = ypart;
    *npanel_out = npanel;
    return BIE_OK;
  }
  const int npanel = (int)((c->ld + kPanelHilo - 1) / kPanelHilo);
  const float* Vhi = (const float*)ctx_buf(c, "V_hi", sizeof(float) * VN, &oom);
  const float* Vlo = (const float*)ctx_buf(c, "V_lo", sizeof(float) * VN, &oom);
  double* ypart = (double*)ctx_buf(c, "vypart", sizeof(double) * c->ld * npanel, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "vgemv: buffers");
  const int panel = (int)std::min<long long>(kPanelHilo, c->ld);
  const size_t smem = 2 * sizeof(float) * panel;
  auto kern = k_gemv_hilo<4, true>;
  BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
  kern<<<dim3(grid0, npanel), gemv_balanced_threads((nv + grid0 - 1) / grid0), smem, c->stream>>>(
      Vhi, Vlo, c->ld, c->row0, nv, panel, xh, xl, ypart, nullptr);
  BIE_LAUNCH_CHECK(c, "k_gemv_hilo (U)");
  *ypart_out = ypart;
  *npanel_out = npanel;
  return BIE_OK;
}
