// GMRES(m) with classical Gram-Schmidt applied twice (CGS2), FP64 Hessenberg /
// Givens / triangular solve, and iterative refinement.
//
// The paper solves eq. Awb with restarted GMRES to ||r|| <= 1e-15 ||b|| (Sec.
// 7.4) and gives no further detail; the choices here are: zero initial guess
// (or the caller's, e.g. the previous time step's),
// CGS2, Givens rotations in FP64, convergence judged on the true residual
// computed with the full-accuracy operator.
//
// Refined schemes (BIE_*_IR): each cycle computes r = D(b - A omega) with the
// ~48-bit (hi + lo) operator, runs one GMRES cycle on the low-precision
// operator for A d = r/||r|| to a relative tolerance, and updates
// omega += ||r|| d in FP64.  The plain scheme (BIE_FP64) is restarted GMRES in
// FP64 with the same kernels.  D flips the sign of the free-surface rows when
// row_flip is set.
//
// Vector kernels work on BIE_NPART row slices and reduce partial sums in a
// fixed order (deterministic).  Convergence flags live on the device and are
// copied into host-mapped slots; the host reads a slot only after waiting on
// an event recorded behind the kernel that wrote it, which makes the writes
// visible, so the kernels issue no system-scope fence.  Every
// kernel of an Arnoldi step returns at once when the cycle is already done, so
// the host can enqueue a few steps ahead and read the flags from host-mapped
// memory without draining the stream.
#include <cmath>
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "nvtx.cuh"
#include "krylov.cuh"

bie_status gemv_lowp_run_skip(bie_ctx* c, const float* x, float* y, int rowflip, const int* skip,
                              const float* Vk, int jdots, double* part1, int* nparts);
bie_status gemv_full_partials_skip(bie_ctx* c, const double* x, double** ypart, int* npanel,
                                   const int* skip, int hi_only);
bie_status gemv_full_finish_skip(bie_ctx* c, const double* ypart, int npanel, const double* x,
                                 int rowflip, const double* b, double* outd, float* outf,
                                 double* part_norm, const int* skip, const double* Vk, int jdots,
                                 double* part1);

struct KrylovArgs {
  int N;
  long long ld;
  int m;             // restart length
  double* H;         // (m+1) x m, column j at H + j*(m+1)
  double* cs;
  double* sn;
  double* g;         // m+1
  double* part1;     // (m+2) rows of BIE_PSTRIDE, row i at part1 + i*BIE_PSTRIDE
  int np1;           // number of valid partials in a row of part1
  double* part2;     // same layout, BIE_NPART valid partials
  double* partn;     // NPART
  SolveStatus* st;
  HostSlot* slots;   // host-mapped ring
  int nslots;
  const unsigned char* pf;   // stored matrix that the next inner product streams
  long long pf_bytes;        // leading bytes of it to fetch into L2 per Arnoldi step (0: none)
};

// One thread per CTA asks L2 to fetch this CTA's share of [p, p + bytes) (a
// multiple of 16 bytes from a 16-byte aligned start).  The Gram-Schmidt kernels
// are latency bound and leave HBM idle; the fetched rows are the first ones the
// next inner product reads, so that much of its stream comes from L2.
__device__ __forceinline__ void l2_prefetch_share(const unsigned char* p, long long bytes) {
  const long long share = ((bytes / gridDim.x) + 15) & ~15LL;
  const long long b0 = share * blockIdx.x;
  const long long b1 = b0 + share < bytes ? b0 + share : bytes;
  for (long long o = b0; o < b1; o += 65536) {
    const unsigned n = (unsigned)(b1 - o < 65536 ? b1 - o : 65536);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + o), "r"(n) : "memory");
  }
}

template <class VT> __device__ __forceinline__ bool is_finite_v(VT v) { return isfinite(v); }

// r = D b, partial norms (first cycle, omega = 0)
__global__ void k_init_resid(int N, const double* __restrict__ b, const int* __restrict__ blk,
                             int rowflip, double* __restrict__ r, double* __restrict__ partn) {
  __shared__ double red[32];
  int r0, r1;
  slice_of(N, r0, r1);
  double acc = 0.0;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
    double v = b[m];
    if (rowflip && blk[m] == 0) v = -v;
    r[m] = v;
    acc += v * v;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partn[blockIdx.x] = acc;
}

// partial sums of r^2 over the row slices (a residual made whole by an
// allgather on a row-partitioned context)
__global__ void k_norm_parts(int N, const double* __restrict__ r, double* __restrict__ partn) {
  __shared__ double red[32];
  int r0, r1;
  slice_of(N, r0, r1);
  double acc = 0.0;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) acc += r[m] * r[m];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) partn[blockIdx.x] = acc;
}

// ||D b|| from the partial norms left by k_init_resid, for a solve that starts
// from a given omega (its first residual is not D b).  b = 0 has the solution
// 0: omega is cleared, so the first residual is 0 and the solve stops there.
__global__ void k_set_bnorm(KrylovArgs K, double* __restrict__ x, int slot) {
  double s = 0.0;
  for (int t = threadIdx.x; t < BIE_NPART; t += 32) s += K.partn[t];
  s = warp_sum(s);
  const double bn = sqrt(__shfl_sync(0xffffffffu, s, 0));
  if (bn == 0.0)
    for (int m = threadIdx.x; m < K.N; m += 32) x[m] = 0.0;
  if (threadIdx.x == 0) {
    K.st->bnorm = bn;
    HostSlot* hs = K.slots + (slot % K.nslots);
    hs->rnorm = bn;
  }
}

// Start of a cycle: ||r||, convergence test, v_0 = r/||r||, g = (1, 0, ...).
template <class VT>
__global__ void k_start(KrylovArgs K, const double* __restrict__ r, VT* __restrict__ V,
                        double rtol, double inner_tol, int first, int slot) {
  __shared__ double tot;
  if (threadIdx.x < 32) {
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < BIE_NPART / 32; ++t) s += K.partn[threadIdx.x + 32 * t];
    s = warp_sum(s);
    if (threadIdx.x == 0) tot = s;
  }
  __syncthreads();
  const double rn = sqrt(tot);
  const double bn = first ? rn : K.st->bnorm;
  const bool bad = !isfinite(rn);
  const bool done = bad || rn <= rtol * bn || rn == 0.0;
  if (!done) {
    const double inv = 1.0 / rn;
    int r0, r1;
    slice_of(K.N, r0, r1);
    for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) V[m] = (VT)(r[m] * inv);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    SolveStatus* st = K.st;
    if (first) st->bnorm = rn;
    st->rnorm = rn;
    st->nonfinite = bad ? 1 : 0;
    st->outer_done = done ? 1 : 0;
    st->inner_done = done ? 1 : 0;
    st->iters = 0;
    st->resid_est = 1.0;
    // this cycle needs a reduction to ~rtol ||b|| / ||r||; not below inner_tol
    st->inner_tol = fmax(inner_tol, 0.5 * rtol * bn / fmax(rn, 1e-300));
    K.g[0] = 1.0;
    for (int i = 1; i <= K.m; ++i) K.g[i] = 0.0;
    HostSlot* hs = K.slots + (slot % K.nslots);
    hs->inner_done = st->inner_done;
    hs->outer_done = st->outer_done;
    hs->nonfinite = st->nonfinite;
    hs->iters = 0;
    hs->rnorm = rn;
    hs->resid_est = 1.0;
  }
}

// CGS pass 1: part1[i][c] = sum_{m in slice c} V_i[m] w[m], i = 0..j
template <class VT>
__global__ void k_cgs1(KrylovArgs K, int j, const VT* __restrict__ V, const VT* __restrict__ w) {
  if (K.st->inner_done) return;
  int r0, r1;
  slice_of(K.N, r0, r1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i <= j; i += nw) {
    const VT* vi = V + (size_t)i * K.ld;
    double s = 0.0;
    for (int m = r0 + lane; m < r1; m += 32) s += (double)vi[m] * (double)w[m];
    s = warp_sum(s);
    if (lane == 0) K.part1[(size_t)i * BIE_PSTRIDE + blockIdx.x] = s;
  }
}

// CGS: h = sum part1; w' = w - V h; part2 = V^T w' and ||w'||^2 (each lane sums
// its few terms of a slice in the vector precision, everything after in FP64)
template <class VT>
__global__ void k_cgs2(KrylovArgs K, int j, const VT* __restrict__ V, VT* __restrict__ w) {
  if (K.st->inner_done) return;
  if (K.pf_bytes > 0 && threadIdx.x == 0) l2_prefetch_share(K.pf, K.pf_bytes);
  extern __shared__ double sh[];          // h[0..j]
  reduce_partials(K.part1, j + 1, K.np1, sh);
  __syncthreads();
  int r0, r1;
  slice_of(K.N, r0, r1);
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) w[m] = subtract_basis(w[m], sh, V, K.ld, j, m);
  __syncthreads();   // the slice of w' is rewritten by this CTA only
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i <= j + 1; i += nw) {
    double s = 0.0;
    if (i <= j) {
      const VT* vi = V + (size_t)i * K.ld;
      VT sf = 0;
      for (int m = r0 + lane; m < r1; m += 32) sf += vi[m] * w[m];
      s = (double)sf;
    } else {
      VT sf = 0;
      for (int m = r0 + lane; m < r1; m += 32) sf += w[m] * w[m];
      s = (double)sf;
    }
    s = warp_sum(s);
    if (lane == 0) K.part2[(size_t)i * BIE_PSTRIDE + blockIdx.x] = s;
  }
}

// CGS: h2 = sum part2; beta = sqrt(||w'||^2 - ||h2||^2); v_{j+1} = (w' - V h2)/beta;
// CTA 0 updates the Hessenberg column, applies Givens rotations and tests.
template <class VT>
__global__ void k_cgs3(KrylovArgs K, int j, VT* __restrict__ V, const VT* __restrict__ w,
                       int slot) {
  if (K.st->inner_done) return;
  extern __shared__ double sh[];          // h2[0..j], nrm2 at [j+1], h[...] at [j+2 ...]
  reduce_partials(K.part2, j + 2, BIE_NPART, sh);
  if (blockIdx.x == 0) reduce_partials(K.part1, j + 1, K.np1, sh + (j + 2));
  __syncthreads();
  __shared__ double s_b2;   // ||w'||^2 - ||h2||^2, one warp's sum for the CTA
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i <= j; i += 32) t += sh[i] * sh[i];
    t = warp_sum(t);
    if (threadIdx.x == 0) s_b2 = sh[j + 1] - t;
  }
  __syncthreads();
  const double beta = sqrt(fmax(s_b2, 0.0));
  const bool breakdown = !(beta > 1e-300) || !isfinite(beta);
  if (!breakdown) {
    const double inv = 1.0 / beta;
    int r0, r1;
    slice_of(K.N, r0, r1);
    VT* vn = V + (size_t)(j + 1) * K.ld;
    for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x)
      vn[m] = (VT)((double)subtract_basis(w[m], sh, V, K.ld, j, m) * inv);
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {   // one warp: Hessenberg column and rotations
    const int m = K.m;
    double* Hj = K.H + (size_t)j * (m + 1);
    for (int i = threadIdx.x; i <= j; i += 32) Hj[i] = sh[j + 2 + i] + sh[i];
    __syncwarp();
    const double uj = givens_apply_warp(Hj, K.cs, K.sn, j);
    if (threadIdx.x != 0) return;
    Hj[j] = uj;
    Hj[j + 1] = beta;
    const double rr = hypot(Hj[j], Hj[j + 1]);
    double c = 1.0, s = 0.0;
    if (rr > 0.0) {
      c = Hj[j] / rr;
      s = Hj[j + 1] / rr;
    }
    K.cs[j] = c;
    K.sn[j] = s;
    Hj[j] = rr;
    Hj[j + 1] = 0.0;
    K.g[j + 1] = -s * K.g[j];
    K.g[j] = c * K.g[j];
    SolveStatus* st = K.st;
    const double est = fabs(K.g[j + 1]);
    st->iters = j + 1;
    st->resid_est = est;
    const bool nf = !isfinite(est) || !isfinite(rr);
    if (nf) st->nonfinite = 1;
    if (nf || breakdown || est <= st->inner_tol || j + 1 >= m) st->inner_done = 1;
    HostSlot* hs = K.slots + (slot % K.nslots);
    hs->inner_done = st->inner_done;
    hs->outer_done = st->outer_done;
    hs->nonfinite = st->nonfinite;
    hs->iters = j + 1;
    hs->rnorm = st->rnorm;
    hs->resid_est = est;
  }
}

// omega += ||r|| V y with R y = g (k x k upper triangular, FP64, one warp per CTA)
template <class VT>
__global__ void k_update(KrylovArgs K, const VT* __restrict__ V, double* __restrict__ x) {
  extern __shared__ double y[];
  const int k = K.st->iters;
  if (K.st->outer_done || k <= 0) return;
  const int m = K.m;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = k - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1 + lane; l < k; l += 32) s += K.H[(size_t)l * (m + 1) + i] * y[l];
      s = warp_sum(s);
      if (lane == 0) y[i] = (K.g[i] - s) / K.H[(size_t)i * (m + 1) + i];
      __syncwarp();
    }
  }
  __syncthreads();
  const double scale = K.st->rnorm;
  int r0, r1;
  slice_of(K.N, r0, r1);
  for (int mm = r0 + threadIdx.x; mm < r1; mm += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc += y[i] * (double)V[(size_t)i * K.ld + mm];
    x[mm] += scale * acc;
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static const int kLookahead = 2;
// share of L2 filled with the stored matrix during each step's Gram-Schmidt kernels
static const double kL2PrefetchFrac = 0.25;

template <class VT>
static bie_status enqueue_step(bie_ctx* c, KrylovArgs& K, int j, VT* V, VT* w, int rowflip,
                               const int* skip, size_t sh_h, int slot) {
  const bool ir = c->precision != BIE_FP64;
  const VT* vj = V + (size_t)j * c->ld;
  // the first CGS pass is fused into the matrix-vector product for j < 64;
  // on a row-partitioned context the product covers the local rows only, so
  // the pass runs after the allgather (k_cgs1)
  const bool part = partitioned(c);
  const bool fused = !part && (!ir || j < BIE_FUSED_DOTS);
  const int pr = prof_begin(c, 0, j);
  if (ir) {
    int np = 0;
    bie_status s = gemv_lowp_run_skip(c, (const float*)(const void*)vj, (float*)(void*)w, rowflip,
                                      skip, fused ? (const float*)(const void*)V : nullptr, j,
                                      fused ? K.part1 : nullptr, &np);
    if (s != BIE_OK) return s;
    K.np1 = fused ? np : BIE_NPART;
  } else {
    double* ypart = nullptr;
    int npanel = 0;
    bie_status s = gemv_full_partials_skip(c, (const double*)(const void*)vj, &ypart, &npanel, skip, 0);
    if (s != BIE_OK) return s;
    s = gemv_full_finish_skip(c, ypart, npanel, (const double*)(const void*)vj, rowflip, nullptr,
                              (double*)(void*)w, nullptr, nullptr, skip,
                              fused ? (const double*)(const void*)V : nullptr, j,
                              fused ? K.part1 : nullptr);
    if (s != BIE_OK) return s;
    K.np1 = BIE_NPART;
  }
  prof_end(c, pr);
  if (part) {   // the other parts' rows of w
    bie_status s = part_allgather(c, w, (int)sizeof(VT), c->N);
    if (s != BIE_OK) return s;
  }
  if (!fused) {
    k_cgs1<VT><<<BIE_NPART, 256, 0, c->stream>>>(K, j, V, w);
    BIE_LAUNCH_CHECK(c, "k_cgs1");
  }
  k_cgs2<VT><<<BIE_NPART, 256, sh_h, c->stream>>>(K, j, V, w);
  k_cgs3<VT><<<BIE_NPART, 256, sh_h, c->stream>>>(K, j, V, w, slot);
  BIE_LAUNCH_CHECK(c, "arnoldi step");
  c->launches += 1;  // k_cgs2 above
  BIE_CUDA_TRY(c, cudaEventRecord(c->evs[slot % BIE_NSLOTS], c->stream));
  return BIE_OK;
}

template <class VT>
static bie_status run_solver(bie_ctx* c, const bie_solve_opts* o, double* x, const double* b,
                             bie_solve_info* info) {
  BIE_NVTX("gmres_ir");
  const int m = o->restart;
  const long long ld = c->ld;
  const bool ir = c->precision != BIE_FP64;
  KrylovArgs K;
  memset(&K, 0, sizeof(K));
  K.N = c->N;
  K.ld = ld;
  K.m = m;
  VT *V, *w;
  double* r;
  BIE_GET(c, VT, ir ? "kr_V32" : "kr_V64", (size_t)(m + 1) * ld, V);
  BIE_GET(c, VT, ir ? "kr_w32" : "kr_w64", ld, w);
  BIE_GET(c, double, "kr_r", ld, r);
  BIE_GET(c, double, "kr_H", (size_t)(m + 1) * m, K.H);
  BIE_GET(c, double, "kr_cs", m, K.cs);
  BIE_GET(c, double, "kr_sn", m, K.sn);
  BIE_GET(c, double, "kr_g", m + 1, K.g);
  BIE_GET(c, double, "kr_part1", (size_t)(m + 2) * BIE_PSTRIDE, K.part1);
  BIE_GET(c, double, "kr_part2", (size_t)(m + 2) * BIE_PSTRIDE, K.part2);
  BIE_GET(c, double, "kr_partn", BIE_NPART, K.partn);
  BIE_GET(c, SolveStatus, "kr_status", 1, K.st);
  bool oom = false;
  const int* blk = (const int*)ctx_buf(c, "blk", sizeof(int) * ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "solve: blk");
  K.slots = c->slots_dev;
  K.nslots = BIE_NSLOTS;
  if (ir) {   // low-precision storage read by every inner product
    const bool f32 = c->precision == BIE_FP32_IR;
    const size_t abytes = (f32 ? 4 : 2) * (size_t)local_rows(c) * (size_t)ld;
    K.pf = (const unsigned char*)ctx_buf(c, f32 ? "A_hi" : "A_16", abytes, &oom);
    if (oom) return ctx_fail(c, BIE_ERR_OOM, "solve: stored matrix");
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
    const long long want = (long long)(kL2PrefetchFrac * (double)l2);
    K.pf_bytes = std::min<long long>(want, (long long)abytes) & ~15LL;
  }
  const int* skip = &K.st->inner_done;
  const size_t sh_h = sizeof(double) * (2 * m + 8);
  const int rowflip = o->row_flip ? 1 : 0;
  double inner_tol = o->inner_tol;
  if (inner_tol <= 0.0) {
    inner_tol = c->precision == BIE_FP64     ? 0.0
                : c->precision == BIE_FP32_IR ? 1e-6
                : c->precision == BIE_FP16_IR ? 2e-3
                                              : 1e-2;
  }
  const bool x0 = o->x0 != 0;   // omega holds an initial guess
  if (!x0) BIE_CUDA_TRY(c, cudaMemsetAsync(x, 0, sizeof(double) * c->N, c->stream));
  BIE_CUDA_TRY(c, cudaMemsetAsync(w, 0, sizeof(VT) * ld, c->stream));
  int slot = 0, total_iters = 0, cycles = 0;
  bool converged = false, nonfinite = false, stagnated = false;
  double last_rn = 0.0, bnorm = 0.0, prev_rn = 0.0;
  int stall = 0, bnorm_slot = -1;
  if (x0) {
    k_init_resid<<<BIE_NPART, 256, 0, c->stream>>>(c->N, b, blk, rowflip, r, K.partn);
    BIE_LAUNCH_CHECK(c, "k_init_resid");
    bnorm_slot = slot++;
    k_set_bnorm<<<1, 32, 0, c->stream>>>(K, x, bnorm_slot);
    BIE_LAUNCH_CHECK(c, "k_set_bnorm");
  }
  for (int cycle = 0;; ++cycle) {
    // residual of the current iterate: r = D(b - A omega) with the full operator
    if (cycle == 0 && !x0) {
      k_init_resid<<<BIE_NPART, 256, 0, c->stream>>>(c->N, b, blk, rowflip, r, K.partn);
      BIE_LAUNCH_CHECK(c, "k_init_resid");
    } else {
      double* ypart = nullptr;
      int npanel = 0;
      // while the last residual is above 1e-4 ||b||, the next one (about
      // inner_tol times smaller) only needs a few digits: FP32 part alone
      // (the residual of an initial guess is always taken in full)
      const int hi_only = (ir && cycle > 0 && last_rn > 1e-4 * bnorm) ? 1 : 0;
      const int pr = prof_begin(c, hi_only ? 4 : 1, -1);
      bie_status s = gemv_full_partials_skip(c, x, &ypart, &npanel, nullptr, hi_only);
      if (s != BIE_OK) return s;
      prof_end(c, pr);
      s = gemv_full_finish_skip(c, ypart, npanel, x, rowflip, b, r, nullptr,
                                partitioned(c) ? nullptr : K.partn, nullptr, nullptr, 0, nullptr);
      if (s != BIE_OK) return s;
      if (partitioned(c)) {   // the other parts' rows of r, then its slice norms
        s = part_allgather(c, r, 8, c->N);
        if (s != BIE_OK) return s;
        k_norm_parts<<<BIE_NPART, 256, 0, c->stream>>>(c->N, r, K.partn);
        BIE_LAUNCH_CHECK(c, "k_norm_parts");
      }
    }
    const int start_slot = slot++;
    k_start<VT><<<BIE_NPART, 256, 0, c->stream>>>(K, r, V, o->rtol, inner_tol, cycle == 0 && !x0,
                                                  start_slot);
    BIE_LAUNCH_CHECK(c, "k_start");
    BIE_CUDA_TRY(c, cudaEventRecord(c->evs[start_slot % BIE_NSLOTS], c->stream));
    const int step0 = slot;
    int enq = 0;
    // steps 0..L-1 go in before the start flags are read (they return at once
    // if the cycle is already converged)
    while (enq < m && enq < kLookahead) {
      bie_status s = enqueue_step<VT>(c, K, enq, V, w, rowflip, skip, sh_h, step0 + enq);
      if (s != BIE_OK) return s;
      ++enq;
    }
    BIE_CUDA_TRY(c, cudaEventSynchronize(c->evs[start_slot % BIE_NSLOTS]));
    {
      const HostSlot hs = c->slots_host[start_slot % BIE_NSLOTS];
      last_rn = hs.rnorm;
      if (cycle == 0) bnorm = x0 ? c->slots_host[bnorm_slot % BIE_NSLOTS].rnorm : hs.rnorm;
      if (hs.nonfinite) nonfinite = true;
      else if (hs.outer_done) converged = true;
      // stagnation: three refinement cycles in a row that cut the true residual by < 10%
      if (cycle > 0 && !converged && !nonfinite) {
        stall = (last_rn > 0.9 * prev_rn) ? stall + 1 : 0;
        if (stall >= 3) stagnated = true;
      }
      prev_rn = last_rn;
    }
    int done_steps = 0;
    if (!nonfinite && !converged && !stagnated && cycle < o->max_cycles) {
      for (int j = 0; j < m; ++j) {
        while (enq < m && enq <= j + kLookahead) {
          bie_status s = enqueue_step<VT>(c, K, enq, V, w, rowflip, skip, sh_h, step0 + enq);
          if (s != BIE_OK) return s;
          ++enq;
        }
        BIE_CUDA_TRY(c, cudaEventSynchronize(c->evs[(step0 + j) % BIE_NSLOTS]));
        const HostSlot hs = c->slots_host[(step0 + j) % BIE_NSLOTS];
        if (hs.nonfinite) nonfinite = true;
        if (hs.inner_done) {
          done_steps = hs.iters;
          break;
        }
      }
    }
    slot = step0 + enq;
    prof_invalidate_steps(c, (converged || nonfinite) ? 0 : done_steps);
    if (nonfinite || converged || stagnated || cycle >= o->max_cycles) break;
    if (ir) k_update<float><<<BIE_NPART, 256, sizeof(double) * (m + 1), c->stream>>>(K, (const float*)(const void*)V, x);
    else k_update<double><<<BIE_NPART, 256, sizeof(double) * (m + 1), c->stream>>>(K, (const double*)(const void*)V, x);
    BIE_LAUNCH_CHECK(c, "k_update");
    total_iters += done_steps;
    ++cycles;
  }
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (info) {
    info->iters = total_iters;
    info->cycles = cycles;
    info->converged = converged ? 1 : 0;
    info->rel_resid = bnorm > 0 ? last_rn / bnorm : last_rn;
  }
  if (nonfinite) return ctx_fail(c, BIE_ERR_NAN, "solve: non-finite residual");
  if (!converged)
    return ctx_fail(c, BIE_ERR_NOCONV, stagnated ? "solve: residual stagnated above rtol"
                                                  : "solve: rtol not reached within max_cycles");
  return BIE_OK;
}

bie_status solve_system(bie_ctx* c, const bie_solve_opts* o, double* x, const double* b,
                        bie_solve_info* info) {
  return (c->precision == BIE_FP64) ? run_solver<double>(c, o, x, b, info)
                                    : run_solver<float>(c, o, x, b, info);
}

bie_status solve_run(bie_ctx* c, const double* phit, double* omega, double* U, double* psi,
                     const bie_solve_opts* o, bie_solve_info* info) {
  double* b;
  BIE_GET(c, double, "kr_b", c->ld, b);
  bie_status s = rhs_run(c, phit, b);
  if (s != BIE_OK) return s;
  bie_status ss = (c->precision == BIE_FP64) ? run_solver<double>(c, o, omega, b, info)
                                             : run_solver<float>(c, o, omega, b, info);
  if (ss != BIE_OK && ss != BIE_ERR_NOCONV) return ss;
  s = velocity_run(c, omega, U, psi);
  if (s != BIE_OK) return s;
  return ss;
}
