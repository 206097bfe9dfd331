// Shared definitions of the GB300 boundary-integral library: error plumbing,
// double-float arithmetic, the context structure and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/bie.h"

#define BIE_MAXB 32                 // maximum number of boundaries
#define BIE_NPART 128               // row slices used by the vector kernels
#define BIE_PSTRIDE 256             // row stride of the partial-sum arrays (>= any producer grid)
#define BIE_FUSED_DOTS 64           // Arnoldi steps whose first CGS dots are fused into the GEMV
#define BIE_LD_ALIGN 64             // leading dimension padding (elements)

// ---------------------------------------------------------------------------
// double-float ("float-float") numbers.  A value is hi + lo with |lo| <= ulp(hi)/2.
// Built from the error-free transformations TwoSum (Knuth), Fast2Sum (Dekker)
// and the FMA-based TwoProd; the composite operations follow the double-double
// scheme of Hida, Li & Bailey ("Algorithms for quad-double precision floating
// point arithmetic", 2001) carried out in single precision, which gives about
// 48 significant bits on the FP32 pipes.  FP64 runs at 1/62 of the FP32 rate
// on this GPU, so every O(N^2) step that needs more than FP32 uses these.
// ---------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ dfl df_two_prod(float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  dfl s = df_two_sum(a.hi, b.hi);
  float e = s.lo + (a.lo + b.lo);
  return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  dfl p = df_two_prod(a.hi, b.hi);
  float e = fmaf(a.hi, b.lo, p.lo);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dfl df_mulf(dfl a, float b) {
  dfl p = df_two_prod(a.hi, b);
  float e = fmaf(a.lo, b, p.lo);
  return df_fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dfl df_sqr(dfl a) {
  dfl p = df_two_prod(a.hi, a.hi);
  float e = fmaf(2.0f * a.hi, a.lo, p.lo);
  return df_fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dfl df_addf(dfl a, float b) {
  dfl s = df_two_sum(a.hi, b);
  float e = s.lo + a.lo;
  return df_fast_two_sum(s.hi, e);
}
// Reciprocal by one Newton step (with its second-order term) from the
// hardware approximation: r0 ~ 1/b, e = 1 - b r0, 1/b = r0 (1 + e + e^2 + ...).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ dfl df_rcp(dfl b) {
  float r = rcp_approx(b.hi);
  float e = fmaf(-b.hi, r, 1.0f);  // exact for a faithful r
  e = fmaf(-b.lo, r, e);
  float re = r * e;
  float c = fmaf(re, e, re);       // r (e + e^2)
  return df_fast_two_sum(r, c);
}
__device__ __forceinline__ dfl df_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }
// third word of x beyond its double-float rounding: x - (hi + lo), as one float
__device__ __forceinline__ float df_residue(double x, dfl d) {
  return __double2float_rn((x - (double)d.hi) - (double)d.lo);
}
__device__ __forceinline__ dfl df_half(dfl a) { return {0.5f * a.hi, 0.5f * a.lo}; }

// ---------------------------------------------------------------------------
// generic real-number interface so the same kernel source serves FP64 and
// double-float
// ---------------------------------------------------------------------------
__device__ __forceinline__ double r_mul(double a, double b) { return a * b; }
__device__ __forceinline__ dfl r_mul(dfl a, dfl b) { return a * b; }
__device__ __forceinline__ double r_add(double a, double b) { return a + b; }
__device__ __forceinline__ dfl r_add(dfl a, dfl b) { return a + b; }
__device__ __forceinline__ double r_sub(double a, double b) { return a - b; }
__device__ __forceinline__ dfl r_sub(dfl a, dfl b) { return a - b; }
__device__ __forceinline__ double r_neg(double a) { return -a; }
__device__ __forceinline__ dfl r_neg(dfl a) { return -a; }
__device__ __forceinline__ double r_sqr(double a) { return a * a; }
__device__ __forceinline__ dfl r_sqr(dfl a) { return df_sqr(a); }
__device__ __forceinline__ double r_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ dfl r_rcp(dfl a) { return df_rcp(a); }
__device__ __forceinline__ double r_addf(double a, float b) { return a + (double)b; }
__device__ __forceinline__ dfl r_addf(dfl a, float b) { return df_addf(a, b); }
__device__ __forceinline__ double r_half(double a) { return 0.5 * a; }
__device__ __forceinline__ dfl r_half(dfl a) { return df_half(a); }
__device__ __forceinline__ float r_hi(double a) { return (float)a; }
__device__ __forceinline__ float r_hi(dfl a) { return a.hi; }
template <class R> __device__ __forceinline__ R r_from_double(double x);
template <> __device__ __forceinline__ double r_from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ dfl r_from_double<dfl>(double x) { return df_from_double(x); }
__device__ __forceinline__ double r_to_double(double a) { return a; }
__device__ __forceinline__ double r_to_double(dfl a) { return df_to_double(a); }

template <class R>
struct cx {
  R re, im;
};
template <class R>
__device__ __forceinline__ cx<R> c_mul(cx<R> a, cx<R> b) {
  return {r_sub(r_mul(a.re, b.re), r_mul(a.im, b.im)), r_add(r_mul(a.re, b.im), r_mul(a.im, b.re))};
}

// ---------------------------------------------------------------------------
// warp / block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ dfl warp_sum(dfl v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dfl t = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = v + t;
  }
  return v;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct SolveStatus {            // device-resident, mirrored to pinned host memory
  int inner_done;               // current GMRES cycle finished
  int outer_done;               // residual met rtol
  int nonfinite;                // non-finite value seen
  int iters;                    // Arnoldi steps in the current cycle
  double rnorm;                 // ||r|| at the start of the current cycle
  double resid_est;             // |g_{j+1}| (relative to ||r||)
  double bnorm;                 // ||b||
  double inner_tol;             // current cycle's relative tolerance
  double gpre;                  // g_j before the provisional rotation of column j
};

struct HostSlot {               // host-mapped copy of the flags, one per pipelined step
  int inner_done;
  int outer_done;
  int nonfinite;
  int iters;
  double rnorm;
  double resid_est;
};

#define BIE_NSLOTS 64

struct bie_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  // geometry
  int nb = 0;
  int N = 0;
  long long ld = 0;             // padded leading dimension (multiple of 64)
  int M[BIE_MAXB] = {0};
  int off[BIE_MAXB + 1] = {0};
  double2 zc[BIE_MAXB] = {};
  int fft_m1[BIE_MAXB] = {0};   // four-step DFT factor M1 of each boundary (M = M1 M2)
  bool have_geom = false;
  bool have_flow = false;
  double V1 = 0.0;
  double a[BIE_MAXB] = {0};

  // assembled storage
  int precision = -1;           // bie_precision of the stored matrix, -1 = none
  bool assembled = false;
  bool transposed = false;      // storage holds S^T (left by the last backward pass)
  bool asm_vs = false;          // this context holds a vortex-sheet solid system
  bool asm_alt = false;         // the next assembly forms the App. B operator (eq. A:alt)
  bool asm_noE = false;         // the next assembly leaves out the -E_k term
  double min_sep = 0.0;         // evolution stops when boundaries come closer (0 = off)
  bie_ctx* gt = nullptr;        // private context of the gamma_t system (eq. gam:t:final)
  int gt_version = -1;
  int gt_precision = -1;
  int variant = 0;              // assembled operator: 0 eq. AB:cor, 1 eq. A:alt (App. B)
  int geom_version = 0;         // bumped by every change of the nodes
  // bumped by bie_set_geometry only: the evolution stages move the free
  // surface and leave the bottom and the obstacles (blocks >= 1) as they are
  int solid_version = 0;
  // what the stored matrix holds: the solid_version it was assembled with and
  // a signature of the storage (precision, transpose, variant, sizes); when
  // both match, an assembly recomputes only the tile pairs touching the surface
  int asm_solid_version = -1;
  long long asm_sig = -1;
  int asm_count = 0;            // bumped by every assembly (the stored matrix changed)
  int oz_count = -1;            // asm_count of the exact-product slices of A held
  int ozv_count = -1;           // asm_count of the exact-product slices of the U-matrix held
  // vortex-sheet solid system of the current geometry (private sub-context)
  bie_ctx* vs = nullptr;
  int vs_version = -1;
  int vs_precision = -1;
  // host-mapped status mirror of the multi-right-hand-side solver
  void* ms_mirror_host = nullptr;
  int ms_mirror_n = 0;

  // host-mapped results of the geometry checks (one record per boundary)
  void* geom_host = nullptr;
  void* geom_dev = nullptr;
  // node counts the spectral tables (twiddles, cotangent tables) were built for
  int spec_M[BIE_MAXB] = {};
  int spec_nb = 0;

  // pinned status mirror, host-mapped step ring and its events
  SolveStatus* status_host = nullptr;
  HostSlot* slots_host = nullptr;
  HostSlot* slots_dev = nullptr;
  cudaEvent_t evs[BIE_NSLOTS] = {};

  // row partition (bie_set_partition): this context stores rows [row0, row1)
  // of the operator, part part_p of part_n; vectors stay whole
  int part_n = 1, part_p = 0;
  int row0 = 0, row1 = 0;
  long long part_R = 0;          // rows per part: the exchange segment length
  bie_exchange_fn exch = nullptr;
  void* exch_user = nullptr;
  void* exch_buf = nullptr;      // caller's staging buffer
  size_t exch_bytes = 0;

  // named device buffers
  std::vector<std::pair<std::string, DevBuf>> bufs;

  // profiling: event pairs around hot kernels, folded into `prof` on collect
  bool profiling = false;
  struct ProfRec {
    int kind;      // 0 inner gemv, 1 full gemv, 2 assemble, 3 velocity
    int ev;        // index of the start event in ev_pool (end = ev + 1)
    int tag;       // step index for inner products (-1 otherwise)
    bool valid;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRec> prof_recs;
  int ev_used = 0;
  bie_profile prof = {};
  long long launches = 0;
};

// profiling helpers (api.cu): prof_begin records a start event and returns the
// record index (or -1 when profiling is off); prof_end records the end event.
int prof_begin(bie_ctx* c, int kind, int tag);
void prof_end(bie_ctx* c, int rec);
void prof_invalidate_steps(bie_ctx* c, int from_step);
bie_status prof_collect(bie_ctx* c);

// Raise (never lower) a kernel's dynamic shared-memory limit on the current
// device.  The limit is a per-function attribute read when a launch is made;
// a CUDA graph replays launches recorded with their own sizes, so lowering it
// for a smaller problem would invalidate launches captured for a larger one.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);

// buffer management (api.cu)
void* ctx_buf(bie_ctx* c, const char* name, size_t bytes, bool* oom);
bie_status ctx_fail(bie_ctx* c, bie_status s, const std::string& msg);
bie_status ctx_cuda(bie_ctx* c, cudaError_t e, const char* where);

#define BIE_CUDA_TRY(ctx, call)                                  \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return ctx_cuda((ctx), _e, #call);    \
  } while (0)

#define BIE_LAUNCH_CHECK(ctx, where)                             \
  do {                                                           \
    (ctx)->launches += 1;                                        \
    cudaError_t _e = cudaGetLastError();                         \
    if (_e != cudaSuccess) return ctx_cuda((ctx), _e, where);    \
  } while (0)

#define BIE_GET(ctx, T, name, count, ptr)                                        \
  do {                                                                           \
    bool _oom = false;                                                           \
    ptr = (T*)ctx_buf((ctx), (name), sizeof(T) * (size_t)(count), &_oom);        \
    if (_oom) return ctx_fail((ctx), BIE_ERR_OOM, std::string("cudaMalloc failed: ") + (name)); \
  } while (0)

// per-boundary tables passed by value to kernels
struct Blocks {
  int nb;
  int N;
  int M[BIE_MAXB];
  int off[BIE_MAXB + 1];
};

inline Blocks make_blocks(const bie_ctx* c) {
  Blocks b;
  b.nb = c->nb;
  b.N = c->N;
  for (int k = 0; k < BIE_MAXB; ++k) b.M[k] = c->M[k];
  for (int k = 0; k <= BIE_MAXB; ++k) b.off[k] = c->off[k];
  return b;
}

// Right preconditioner of the inner solves, P = I - (3/2) sum_k e_k e_k^T / M_k
// over the obstacles k (e_k: ones on obstacle k's rows).  A constant density
// on an obstacle is annihilated by its Cauchy blocks (eq. Phij:w:const), so the
// -E_k term of the obstacle diagonal block makes A e_k = -e_k (eq. AB:cor):
// nb - 2 eigenvalues at -1, apart from the rest, which cluster at +-1/2.  A P
// maps e_k to e_k / 2 and leaves the rest of the spectrum as it is, so GMRES
// no longer spends iterations of every refinement cycle on those directions.
// For the transposed operator of the adjoint, e_k is a left eigenvector for -1
// instead, and the same P moves that eigenvalue to 1/2 as well (a rank-one
// change along a left eigenvector shifts only its eigenvalue).  The
// vortex-sheet solid system (eq. lin:sys2) has e_k as left eigenvectors for -1
// too, but its cluster sits at -1/2: there coef = 1/2 moves -1 to -1/2.  The product
// stages P x (x less 3/2 of its mean on each obstacle); the means come from
// block sums of x that the kernel producing x left as partial sums.
struct RightDefl {
  const double* part;      // row k: BIE_NPART partial sums of x over obstacle k (null: P = I)
  double* mean_out;        // means of x over the obstacles, written by CTA 0 (may be null)
  int nobs;                // obstacles
  int obs0;                // first obstacle row (N when there are none)
  int off[BIE_MAXB + 1];   // obstacle k: rows off[k] .. off[k+1] - 1
  float invM[BIE_MAXB];    // 1 / M of obstacle k
  float coef;              // P = I - coef sum_k e_k e_k^T / M_k (3/2, or 1/2: see below)
};

struct FlowParams {
  int nb;
  double V1;
  double a[BIE_MAXB];
  double2 zc[BIE_MAXB];
};

inline FlowParams make_flow(const bie_ctx* c) {
  FlowParams f;
  f.nb = c->nb;
  f.V1 = c->V1;
  for (int k = 0; k < BIE_MAXB; ++k) {
    f.a[k] = c->a[k];
    f.zc[k] = c->zc[k];
  }
  return f;
}

// internal entry points shared between translation units
bie_status asm_run(bie_ctx* c, int precision, int transpose);
bie_status solve_system(bie_ctx* c, const bie_solve_opts* o, double* x, const double* b,
                        bie_solve_info* info);
bie_status gemv_apply(bie_ctx* c, int which, const double* x_dev, double* y_dev);
bie_status sample_run(bie_ctx* c, int which, long n, const long long* rows, const long long* cols,
                      double* out);
bie_status velocity_run(bie_ctx* c, const double* omega, double* U, double* psi);
bie_status velocity_from_weights(bie_ctx* c, const float2* cw, const float2* hw0, double* U);
// omega'/M_l as double-float (xh, xl: [nvec][ld], zero padded) and H omega_0'
// (hw0: [nvec][M_0]) for nvec vectors omega ([nvec][N])
bie_status velocity_weights(bie_ctx* c, int nvec, const double* omega, float* xh, float* xl,
                            float2* hw0);
bie_status solve_run(bie_ctx* c, const double* phit, double* omega, double* U, double* psi,
                     const bie_solve_opts* opts, bie_solve_info* info);
bie_status rhs_run(bie_ctx* c, const double* phit, double* b);
bie_status rhs_run_many(bie_ctx* c, int nrhs, const double* phit, long long pstride, double* b,
                        long long bstride);
bie_status geometry_prep(bie_ctx* c);
bie_status geometry_refresh(bie_ctx* c);
bie_status psi_run(bie_ctx* c, const double* omega, double* psi);
bie_status separation_run(bie_ctx* c, double* ratio_min, int* node);
bie_status energy_run(bie_ctx* c, const double* phit, const double* omega, double tau, double g,
                      double* E_dev);

static inline long long round_up(long long x, long long a) { return (x + a - 1) / a * a; }

// rows of the stored operator held by this context (all N unless partitioned)
static inline int local_rows(const bie_ctx* c) { return c->row1 - c->row0; }
static inline bool partitioned(const bie_ctx* c) { return c->part_n > 1; }
// surface rows of the U-matrix held by this context (rows [row0, min(row1, M_0)))
static inline int local_vrows(const bie_ctx* c) {
  const int r1 = c->row1 < c->M[0] ? c->row1 : c->M[0];
  return r1 > c->row0 ? r1 - c->row0 : 0;
}
// partition arithmetic from N and (part_n, part_p) (api.cu)
void partition_update(bie_ctx* c);
// allgather of the local rows [row0, row1) of a whole vector (elem_bytes 4 or
// 8; rows past `limit` are not part of the vector) through the caller's
// exchange function: on return the vector is whole on every part (api.cu)
bie_status part_allgather(bie_ctx* c, void* vec, int elem_bytes, int limit);
// in-place sum of n doubles over the parts (api.cu)
bie_status part_allreduce(bie_ctx* c, double* vec, long long n);
