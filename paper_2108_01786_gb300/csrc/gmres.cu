// GMRES(m) with classical Gram-Schmidt applied twice (CGS2, the second pass
// delayed by one step so that each Arnoldi step takes one global reduction),
// FP64 Hessenberg / Givens / triangular solve, and iterative refinement.
//
// The paper solves eq. Awb with restarted GMRES to ||r|| <= 1e-15 ||b|| (Sec.
// 7.4) and gives no further detail; the choices here are: zero initial guess
// (or the caller's, e.g. the previous time step's),
// delayed CGS2, Givens rotations in FP64, convergence judged on the true
// residual computed with the full-accuracy operator.
//
// Refined schemes (BIE_*_IR): each cycle computes r = D(b - A omega) with the
// ~48-bit (hi + lo) operator (with its FP32 part alone while r is large, and
// near the end as an update from the last increment with a cheaper copy: see
// kResidDrift), runs one GMRES cycle on the low-precision operator for
// A d = r/||r|| to a relative tolerance, and updates omega += ||r|| d in FP64.  The plain scheme (BIE_FP64) is restarted GMRES in
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
                              const float* Vk, const float* Ck, int qk, int jdots, double* part1,
                              int* nparts, const RightDefl* defl);
bie_status gemv_full_partials_skip(bie_ctx* c, const double* x, double** ypart, int* npanel,
                                   const int* skip, int hi_only);
bie_status gemv_full_finish_skip(bie_ctx* c, const double* ypart, int npanel, const double* x,
                                 int rowflip, const double* b, double* outd, float* outf,
                                 double* part_norm, const int* skip, const double* Vk, int jdots,
                                 double* part1);

int gemv_num_ctas();

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
  double* part3[2];  // same layout, BIE_NPART valid partials: dots of z_j in part3[j & 1]
  double* hraw;      // last Hessenberg column before its correction and rotations (m+2)
  // right preconditioner P of the refined schemes (see RightDefl): obstacle
  // block sums of z_j follow alpha in part3[j & 1] (rows j+1 .. j+nobs); the
  // product of step j stores the means of z_j in zmean[j][k]
  int nobs;          // 0: P = I
  int obs0;
  int obs_off[BIE_MAXB + 1];
  float obs_invM[BIE_MAXB];
  float obs_coef;    // P = I - obs_coef sum_k e_k e_k^T / M_k
  double* zmean;     // (m+1) x BIE_MAXB
  // recycled subspace (see k_dcgs): q columns of C (orthonormal) and U with
  // T U = C; Bm column j (C-part of Hessenberg column j) at Bm + j BIE_RQMAX
  int q;
  void* Crv;         // BIE_RQMAX x ld
  void* Urv;         // BIE_RQMAX x ld
  double* Bm;        // m x BIE_RQMAX
  double* braw;      // C-part of the last column before its correction
  double* aC0;       // C-part of z_0: z_0 = C c_0 + nu v_0
  double* umean;     // BIE_RQMAX x BIE_MAXB: means of U's columns over the obstacles
  double* dlast;     // the last cycle's increment of omega (N; may be null)
  double* partn;     // NPART
  SolveStatus* st;
  HostSlot* slots;   // host-mapped ring
  int nslots;
  const unsigned char* pf;   // stored matrix that the next inner product streams
  long long pf_bytes;        // bytes of it to fetch into L2 per Arnoldi step (0: none)
  long long pf_stride;       // the product's CTAs read chunks of this many bytes,
  int pf_nchunks;            // pf_nchunks of them; each chunk's head is fetched
  long long pf_total;        // bytes of the stored matrix (no fetch beyond them)
};

// One thread per CTA asks L2 to fetch the heads of this CTA's share of the
// chunks (bytes / nchunks of each, a multiple of 16 bytes from a 16-byte
// aligned start).  The Arnoldi step is latency bound and leaves HBM idle; the
// inner product's CTAs each stream one chunk of rows from its head, so that
// much of its stream comes from L2.
__device__ __forceinline__ void l2_prefetch_chunks(const unsigned char* p, long long bytes,
                                                   long long stride, int nchunks, long long total) {
  const long long head = (bytes / nchunks) & ~15LL;
  for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long b0 = stride * ch;
    const long long b1 = (b0 + head < total ? b0 + head : total) & ~15LL;
    for (long long o = b0; o < b1; o += 65536) {
      const unsigned n = (unsigned)(b1 - o < 65536 ? b1 - o : 65536);
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + o), "r"(n) : "memory");
    }
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

// rd = D r (D: sign flip of the free-surface rows when rowflip)
__global__ void k_flip_copy(int N, const double* __restrict__ r, const int* __restrict__ blk,
                            int rowflip, double* __restrict__ rd) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < N) rd[m] = (rowflip && blk[m] == 0) ? -r[m] : r[m];
}

// the increment d in FP32 for the inner-storage product (zero past N)
__global__ void k_inc_to_f(int N, long long ld, const double* __restrict__ d, float* __restrict__ df) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) df[i] = i < N ? (float)d[i] : 0.f;
}

// r <- r - y (y = D A d from the inner storage) and the row slices' sums of r^2
__global__ void k_resid_sub(int N, const float* __restrict__ y, double* __restrict__ r,
                            double* __restrict__ partn) {
  __shared__ double red[32];
  int r0, r1;
  slice_of(N, r0, r1);
  double acc = 0.0;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
    const double v = r[m] - (double)y[m];
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

// Start of a cycle: ||r||, convergence test, z_0 = r/||r|| (in V_0 and Z_0) with
// its slice dots in part3[0] (rows 0..q-1: C_i^T z_0, row q: z_0^2, then the
// obstacle block sums), g = (1, 0, ...).
template <class VT>
__global__ void k_start(KrylovArgs K, const double* __restrict__ r, VT* __restrict__ V,
                        VT* __restrict__ Z, double rtol, double inner_tol, int first, int slot) {
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
    for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
      const VT z = (VT)(r[m] * inv);
      V[m] = z;
      Z[m] = z;
    }
    __syncthreads();   // the slice of z_0 is this CTA's
    const int q = K.q;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i <= q + K.nobs; i += nw) {
      double t = 0.0;
      if (i <= q) {   // C_i^T z_0, then z_0^2
        const VT* ci = i < q ? (const VT*)K.Crv + (size_t)i * K.ld : V;
        for (int m = r0 + lane; m < r1; m += 32) t += (double)ci[m] * (double)V[m];
      } else {        // z_0 summed over this slice's part of obstacle i - q - 1
        const int k = i - q - 1;
        const int a0 = max(r0, K.obs_off[k]), a1 = min(r1, K.obs_off[k + 1]);
        for (int m = a0 + lane; m < a1; m += 32) t += (double)V[m];
      }
      t = warp_sum(t);
      if (lane == 0) K.part3[0][(size_t)i * BIE_PSTRIDE + blockIdx.x] = t;
    }
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

// Recycled subspace (refined schemes): the cycles of one solve share the
// operator T, so the directions found by earlier cycles are kept as a pair
// T U = C with C orthonormal (GCRO-DR of Parks, de Sturler, Mackey, Johnson &
// Maiti, "Recycling Krylov subspaces for sequences of linear systems", 2006,
// keeping every earlier cycle's space rather than a few harmonic Ritz
// vectors).  Each Arnoldi step orthogonalises against [C, V] (index i < q: C_i,
// i >= q: V_{i-q}); the C-part of a column goes to B (T Z = C B + V H), the
// least-squares problem stays the one in H, and the correction is
// U (c_0 - B y) + Z y with c_0 the C-part of z_0.  After the cycle, C grows by
// the columns of V_{k+1} rotated by the cycle's Givens rotations and U by
// (Z - U B) R^-1, which keeps T U = C.
#define BIE_RQMAX 32   // recycled columns kept at most
#define BIE_RKMAX 16   // columns a cycle may add

template <class VT>
__device__ __forceinline__ const VT* qvec(const KrylovArgs& K, const VT* V, int i) {
  return i < K.q ? (const VT*)K.Crv + (size_t)i * K.ld : V + (size_t)(i - K.q) * K.ld;
}

// Dots of the new vector w with the basis Q_0..Q_{q+j} and with itself, for a
// context whose product is not fused with them (row-partitioned, or more than
// 64 dots): part1[i][c] = sum over slice c of Q_i[m] w[m] (i <= q+j),
// part1[q+j+1][c] = sum of w[m]^2
template <class VT>
__global__ void k_cgs1(KrylovArgs K, int j, const VT* __restrict__ V, const VT* __restrict__ w) {
  if (K.st->inner_done) return;
  int r0, r1;
  slice_of(K.N, r0, r1);
  const int nb = K.q + j;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i <= nb + 1; i += nw) {
    const VT* vi = i <= nb ? qvec(K, V, i) : w;
    double s = 0.0;
    for (int m = r0 + lane; m < r1; m += 32) s += (double)vi[m] * (double)w[m];
    s = warp_sum(s);
    if (lane == 0) K.part1[(size_t)i * BIE_PSTRIDE + blockIdx.x] = s;
  }
}

// Givens rotation that zeroes b against a: (c, s, r) with c a + s b = r
__device__ __forceinline__ void givens_of(double a, double b, double& c, double& s, double& r) {
  r = hypot(a, b);
  c = 1.0;
  s = 0.0;
  if (r > 0.0) {   // one FP64 division (a long dependent chain on this GPU), two products
    const double ir = 1.0 / r;
    c = a * ir;
    s = b * ir;
  }
}

// One Arnoldi step with a single global reduction: classical Gram-Schmidt
// twice, the second pass of each new vector delayed to the next step, where
// its dots join the reduction of that step's first pass (DCGS2 of
// Swirydowicz, Langou, Ananthan, Yang & Thomas, "Low synchronization
// Gram-Schmidt and GMRES algorithms", 2020), written in the flexible form.
// On entry V_0..V_{j-1} are orthonormal and V_j holds z_j, the previous step's
// projected vector divided by its norm estimate (orthogonal to one pass of
// rounding); the product w = A z_j has left
//   part1 rows 0..j+1:  s_i = V_i^T w (i < j), sigma = z_j^T w, omega = w^T w
// and the previous step (or the cycle start)
//   part3[j & 1] rows 0..j:  a_i = V_i^T z_j (i < j), alpha = z_j^T z_j.
// From these alone:
//   nu = sqrt(alpha - |a|^2),  v_j = (z_j - V a) / nu        second pass of z_j
//   h = (s, (sigma - a.s) / nu),  beta = sqrt(omega - |h|^2)
//   z_{j+1} = (w - V s - h_j v_j) / beta
// A z_j = V_{j+1} h + beta z_{j+1}; once z_{j+1} = nu' v_{j+1} + V_{j+1} a' is
// known, column j becomes h + beta a' with subdiagonal beta nu' (applied at
// the next step, or by k_update for the cycle's last column).  The relation
// A Z_k = V_{k+1} H_k with the stored vectors z (what A was applied to) makes
// the update omega += ||r|| Z y, y the least-squares solution in H (flexible
// GMRES), exact in exact arithmetic however far each z is from v.
// The Hessenberg column is kept unrotated in hraw until its correction; the
// rotation is recomputed then, and g_j before the provisional rotation is
// kept in st->gpre.
//
// The last warp of CTA 0 does the Hessenberg work (both columns, rotations,
// the convergence test) in shared memory while the other warps of every CTA
// update the vectors and form the next dots; it joins no barrier after the
// scalars are known, so its chain of dependent steps overlaps the vector work.
// Dynamic shared memory of k_dcgs, in doubles, for restart length m: the FP64
// scalars, then the coefficients converted to the basis type once per CTA.
__host__ __device__ inline size_t dcgs_fp64_doubles(int m) { return 6 * (size_t)m + 8 + 3 * BIE_RQMAX; }
static inline size_t dcgs_smem_doubles(int m) {
  return dcgs_fp64_doubles(m) + 2 * ((size_t)m + 2 + BIE_RQMAX);
}
template <class VT>
__global__ void __launch_bounds__(256)
    k_dcgs(KrylovArgs K, int j, VT* __restrict__ V, VT* __restrict__ Z,
           const VT* __restrict__ w, int slot) {
  if (K.st->inner_done) return;
  if (K.pf_bytes > 0 && threadIdx.x == 0)
    l2_prefetch_chunks(K.pf, K.pf_bytes, K.pf_stride, K.pf_nchunks, K.pf_total);
  extern __shared__ double sh[];   // dcgs_smem_doubles(m)
  const int mm = K.m, q = K.q, nb = q + j;   // nb: basis vectors before v_j
  double* s1 = sh;                            // s_0..s_{nb-1}, sigma at [nb], omega at [nb+1]
  double* s3 = sh + (BIE_RQMAX + mm + 2);     // a_0..a_{nb-1}, alpha at [nb]
  double* h_cs = s3 + (BIE_RQMAX + mm + 1);   // rotations 0..j-1, then j-1 recomputed
  double* h_sn = h_cs + mm;
  double* h_col = h_sn + mm;                  // a Hessenberg column, m + 2
  double* h_raw = h_col + (mm + 2);           // column j - 1 before correction, m + 2
  double* h_braw = h_raw + (mm + 2);          // its C-part, q
  VT* f1 = reinterpret_cast<VT*>(sh + dcgs_fp64_doubles(mm));   // (VT) s1, nb entries
  VT* f3 = f1 + (BIE_RQMAX + mm + 2);                           // (VT) s3, nb entries
  __shared__ double h_gpre;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const bool hwarp = blockIdx.x == 0 && warp == nw - 1;
  if (hwarp) {   // operands of the Hessenberg work, fetched while the partials reduce
    for (int i = lane; i < j; i += 32) {
      h_cs[i] = K.cs[i];
      h_sn[i] = K.sn[i];
    }
    for (int i = lane; i <= j; i += 32) h_raw[i] = K.hraw[i];
    for (int i = lane; i < q; i += 32) h_braw[i] = K.braw[i];
    if (lane == 0) h_gpre = K.st->gpre;
  }
  reduce_partials(K.part1, nb + 2, K.np1, s1);
  reduce_partials(K.part3[j & 1], nb + 1, BIE_NPART, s3);
  __syncthreads();
  __shared__ double s_nu, s_hj, s_beta;
  __shared__ VT s_inu, s_ib;
  if (threadIdx.x >= 32) {   // the vector update's coefficients, converted once per CTA
    for (int i = threadIdx.x - 32; i < nb; i += blockDim.x - 32) {
      f1[i] = (VT)s1[i];
      f3[i] = (VT)s3[i];
    }
  } else {
    double ta = 0.0, tas = 0.0, tss = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) {
      ta += s3[i] * s3[i];
      tas += s3[i] * s1[i];
      tss += s1[i] * s1[i];
    }
    ta = warp_sum(ta);
    tas = warp_sum(tas);
    tss = warp_sum(tss);
    if (threadIdx.x == 0) {
      const double nu = sqrt(fmax(s3[nb] - ta, 0.0));
      const double hj = (s1[nb] - tas) / nu;
      s_nu = nu;
      s_hj = hj;
      const double beta = sqrt(fmax(s1[nb + 1] - tss - hj * hj, 0.0));
      s_beta = beta;
      s_inu = (VT)(1.0 / nu);
      s_ib = (beta > 1e-300 && isfinite(beta)) ? (VT)(1.0 / beta) : (VT)0;
    }
  }
  __syncthreads();
  const double nu = s_nu, hj = s_hj, beta = s_beta;
  // z_j lies in span [C, V] (to rounding): column j - 1 is the cycle's last one
  const bool lost = !(nu > 1e-300) || !isfinite(nu) || !isfinite(hj);
  const bool brk = lost || !(beta > 1e-300) || !isfinite(beta);
  if (warp == nw - 1) {
    if (!hwarp) return;
    // Hessenberg columns j - 1 (final) and j (provisional), rotations, test
    SolveStatus* st = K.st;
    double gj = 0.0;   // g_j after the rotations of columns < j (lane 0)
    if (j > 0) {
      const double bprev = h_raw[j];
      for (int i = lane; i < j; i += 32) h_col[i] = h_raw[i] + bprev * s3[q + i];
      for (int i = lane; i < q; i += 32) K.Bm[(size_t)(j - 1) * BIE_RQMAX + i] = h_braw[i] + bprev * s3[i];
      if (lane == 0) h_col[j] = bprev * nu;
      __syncwarp();
      const double u = givens_apply_warp(h_col, h_cs, h_sn, j - 1);
      if (lane == 0) {
        double c, s, rr;
        givens_of(u, h_col[j], c, s, rr);
        h_cs[j - 1] = c;
        h_sn[j - 1] = s;
        h_col[j - 1] = rr;
        h_col[j] = 0.0;
        K.cs[j - 1] = c;
        K.sn[j - 1] = s;
        K.g[j - 1] = c * h_gpre;
        gj = -s * h_gpre;
      }
      __syncwarp();
      double* Hc = K.H + (size_t)(j - 1) * (mm + 1);
      for (int i = lane; i <= j; i += 32) Hc[i] = h_col[i];
      __syncwarp();
    } else {
      gj = nu;   // z_0 = C c_0 + nu v_0: the right-hand side in H is nu e_1
      for (int i = lane; i < q; i += 32) K.aC0[i] = s3[i];
    }
    HostSlot* hs = K.slots + (slot % K.nslots);
    if (lost) {
      if (lane == 0) {
        const double est = fabs(gj);
        K.g[j] = gj;
        st->iters = j;
        st->resid_est = est;
        if (!isfinite(est)) st->nonfinite = 1;
        st->inner_done = 1;
        hs->inner_done = 1;
        hs->outer_done = st->outer_done;
        hs->nonfinite = st->nonfinite;
        hs->iters = j;
        hs->rnorm = st->rnorm;
        hs->resid_est = est;
      }
      return;
    }
    for (int i = lane; i < j; i += 32) {
      h_col[i] = s1[q + i];
      K.hraw[i] = s1[q + i];
    }
    for (int i = lane; i < q; i += 32) K.braw[i] = s1[i];
    if (lane == 0) {
      h_col[j] = hj;
      K.hraw[j] = hj;
      K.hraw[j + 1] = beta;
    }
    __syncwarp();
    const double uj = givens_apply_warp(h_col, h_cs, h_sn, j);
    double c = 1.0, s = 0.0, rr = 0.0;
    if (lane == 0) {
      givens_of(uj, beta, c, s, rr);
      h_col[j] = rr;
      h_col[j + 1] = 0.0;
    }
    __syncwarp();
    double* Hj = K.H + (size_t)j * (mm + 1);
    for (int i = lane; i <= j + 1; i += 32) Hj[i] = h_col[i];
    if (lane != 0) return;
    K.cs[j] = c;
    K.sn[j] = s;
    st->gpre = gj;
    K.g[j + 1] = -s * gj;
    K.g[j] = c * gj;
    const double est = fabs(s * gj);
    st->iters = j + 1;
    st->resid_est = est;
    const bool nf = !isfinite(est) || !isfinite(rr);
    if (nf) st->nonfinite = 1;
    if (nf || brk || est <= st->inner_tol || j + 1 >= mm) st->inner_done = 1;
    hs->inner_done = st->inner_done;
    hs->outer_done = st->outer_done;
    hs->nonfinite = st->nonfinite;
    hs->iters = j + 1;
    hs->rnorm = st->rnorm;
    hs->resid_est = est;
    return;
  }
  if (lost) return;
  // the other warps: v_j and z_{j+1} over this CTA's slice, then the dots of z_{j+1}
  const int nt = blockDim.x - 32;
  const long long ld = K.ld;
  int r0, r1;
  slice_of(K.N, r0, r1);
  VT* vj = V + (size_t)j * ld;
  VT* vn = V + (size_t)(j + 1) * ld;
  VT* zn = Z + (size_t)(j + 1) * ld;
  const VT inu = s_inu, ib = brk ? (VT)0 : s_ib, vh = (VT)hj;
  for (int m = r0 + threadIdx.x; m < r1; m += nt) {
    VT t = vj[m], u = w[m];
    int i = 0;
    for (; i + 7 < nb; i += 8) {   // eight loads in flight per L2 round trip
      VT v[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) v[p] = qvec(K, (const VT*)V, i + p)[m];
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        t -= f3[i + p] * v[p];
        u -= f1[i + p] * v[p];
      }
    }
    for (; i < nb; ++i) {
      const VT v = qvec(K, (const VT*)V, i)[m];
      t -= f3[i] * v;
      u -= f1[i] * v;
    }
    const VT vt = t * inu;
    vj[m] = vt;
    if (!brk) {
      const VT zz = (u - vh * vt) * ib;
      vn[m] = zz;
      zn[m] = zz;
    }
  }
  // this CTA's slice of v_j and z_{j+1} is written by these warps only
  asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
  // a' = Q_i^T z_{j+1} (i <= nb, v_j included), alpha' = |z_{j+1}|^2 and the
  // obstacle block sums of z_{j+1} over the slice
  double* p3 = K.part3[(j + 1) & 1];
  const int nrow = nb + 2 + K.nobs;
  // products summed in the basis type in runs of eight, the runs in FP64
  auto slice_sum = [&](int i) -> double {   // this lane's share of row i
    double acc = 0.0;
    if (i <= nb + 1) {
      const VT* vi = qvec(K, (const VT*)V, i);
      VT run = 0;
      int c = 0;
      for (int m = r0 + lane; m < r1; m += 32) {
        run = fma(vi[m], vn[m], run);
        if (++c == 8) {
          acc += (double)run;
          run = 0;
          c = 0;
        }
      }
      acc += (double)run;
    } else {
      const int k = i - (nb + 2);
      const int a0 = max(r0, K.obs_off[k]), a1 = min(r1, K.obs_off[k + 1]);
      for (int m = a0 + lane; m < a1; m += 32) acc += (double)vn[m];
    }
    return acc;
  };
  for (int i = warp; i < nrow; i += 2 * (nw - 1)) {   // two rows per warp at a time
    const int i2 = i + (nw - 1);
    double acc = 0.0, acc2 = 0.0;
    if (!brk) {
      if (i2 <= nb + 1) {   // two basis rows: one pass over the slice
        const VT* vi = qvec(K, (const VT*)V, i);
        const VT* vi2 = qvec(K, (const VT*)V, i2);
        VT run = 0, run2 = 0;
        int c = 0;
        for (int m = r0 + lane; m < r1; m += 32) {
          const VT zv = vn[m];
          run = fma(vi[m], zv, run);
          run2 = fma(vi2[m], zv, run2);
          if (++c == 8) {
            acc += (double)run;
            acc2 += (double)run2;
            run = run2 = 0;
            c = 0;
          }
        }
        acc += (double)run;
        acc2 += (double)run2;
      } else {
        acc = slice_sum(i);
        if (i2 < nrow) acc2 = slice_sum(i2);
      }
    }
    acc = warp_sum(acc);
    acc2 = warp_sum(acc2);
    if (lane == 0) {
      p3[(size_t)i * BIE_PSTRIDE + blockIdx.x] = acc;
      if (i2 < nrow) p3[(size_t)i2 * BIE_PSTRIDE + blockIdx.x] = acc2;
    }
  }
}

// End of a cycle with k columns.  The last column k-1 takes the second pass of
// z_k (its dots are in part3[k & 1]: rows 0..q+k-1 against [C, V], row q+k: z_k^2)
// and its rotation is recomputed; R y = g (k x k upper triangular, FP64, one
// warp per CTA); omega += ||r|| P (Z y + U (c_0 - B y)).  With ext the cycle's
// space joins the recycled one: C gains the first k columns of V_{k+1} G^T (G
// the cycle's rotations, v_k the second pass of z_k) and U gains (Z - U B) R^-1,
// so that T U = C still holds; the means of the new U columns over the
// obstacles follow from those of Z and U.
// FP64 scalars, then their copies in the basis type for the row loop
__host__ __device__ inline size_t update_fp64_doubles(int m) {
  return 3 * (size_t)m + 2 + 3 * BIE_RQMAX + BIE_RKMAX * BIE_RKMAX + BIE_RQMAX * BIE_RKMAX;
}
static inline size_t update_smem_doubles(int m) {
  return update_fp64_doubles(m) + 4 * (size_t)m + 2 * BIE_RQMAX + 2;
}
template <class VT>
__global__ void k_update(KrylovArgs K, const VT* __restrict__ V, const VT* __restrict__ Z,
                         double* __restrict__ x, int ext) {
  extern __shared__ double y[];   // update_smem_doubles(m)
  const int k = K.st->iters;
  if (K.st->outer_done || k <= 0) return;
  const int m = K.m, q = K.q;
  double* hc = y + m;                          // column k-1, m + 1
  double* pa = hc + (m + 1);                   // dots of z_k, q + k + 1
  double* tq = pa + (BIE_RQMAX + m + 1);       // c_0 - B y, q
  double* bl = tq + BIE_RQMAX;                 // C-part of column k-1, q
  double* Ri = bl + BIE_RQMAX;                 // R^-1, BIE_RKMAX x BIE_RKMAX (row i, column c)
  double* Mq = Ri + BIE_RKMAX * BIE_RKMAX;     // -B R^-1, BIE_RQMAX x BIE_RKMAX
  __shared__ double s_nu, s_c, s_s;
  __shared__ double s_dm[BIE_MAXB];
  __shared__ double s_rinv[32];                       // 1 / R_ii (k <= 32), warp 0
  __shared__ double s_rinv1[BIE_RKMAX];                // the same for warp 1's R^-1
  __shared__ double s_R[BIE_RKMAX * BIE_RKMAX];        // R for R^-1 (row i, column c)
  reduce_partials(K.part3[k & 1], q + k + 1, BIE_NPART, pa);
  __syncthreads();
  const double* Hm = K.H;
  auto Rent = [&](int i, int c) -> double {    // R[i][c], i <= c < k
    return c == k - 1 ? hc[i] : Hm[(size_t)c * (m + 1) + i];
  };
  auto Bent = [&](int l, int i) -> double {    // B[l][i], l < q, i < k
    return i == k - 1 ? bl[l] : K.Bm[(size_t)i * BIE_RQMAX + l];
  };
  const int warp0 = threadIdx.x >> 5;
  if (warp0 == 0) {
    const int lane = threadIdx.x;
    double ta = 0.0;
    for (int i = lane; i < q + k; i += 32) ta += pa[i] * pa[i];
    ta = warp_sum(ta);
    const double nu = sqrt(fmax(pa[q + k] - ta, 0.0));
    const double bk = K.hraw[k];
    for (int i = lane; i < k; i += 32) hc[i] = K.hraw[i] + bk * pa[q + i];
    for (int l = lane; l < q; l += 32) bl[l] = K.braw[l] + bk * pa[l];
    __syncwarp();
    const double u = givens_apply_warp(hc, K.cs, K.sn, k - 1);
    double c, s, rr;
    givens_of(u, bk * nu, c, s, rr);
    if (lane == 0) {
      hc[k - 1] = rr;
      s_nu = nu;
      s_c = c;
      s_s = s;
    }
    __syncwarp();
    // warp 1 forms R^-1 and -B R^-1 beside this warp's solve for y once the
    // last column of R and the C-part of B are in place
    if (ext) asm volatile("bar.sync 2, 64;" ::: "memory");
    const double gl = c * K.st->gpre;
    __syncwarp();
    if (k <= 32) {
      // R y = g by columns with y_i in lane i: the diagonal's reciprocals in
      // parallel, then per column one broadcast and one FMA (column l - 1 of R
      // is loaded while column l is applied)
      double yv = 0.0, rv = 0.0;
      if (lane < k) {
        yv = lane == k - 1 ? gl : K.g[lane];
        rv = 1.0 / Rent(lane, lane);
        s_rinv[lane] = rv;
      }
      double Rc = lane < k - 1 ? Rent(lane, k - 1) : 0.0;
      for (int l = k - 1; l >= 0; --l) {
        const double Rn = (l >= 1 && lane < l - 1) ? Rent(lane, l - 1) : 0.0;
        if (lane == l) yv *= rv;
        const double yl = __shfl_sync(0xffffffffu, yv, l);
        if (lane < l) yv = fma(-Rc, yl, yv);
        Rc = Rn;
      }
      if (lane < k) y[lane] = yv;
      __syncwarp();
    } else {
      for (int i = k - 1; i >= 0; --i) {
        double t = 0.0;
        for (int l = i + 1 + lane; l < k; l += 32) t += Rent(i, l) * y[l];
        t = warp_sum(t);
        if (lane == 0) y[i] = ((i == k - 1 ? gl : K.g[i]) - t) / Rent(i, i);
        __syncwarp();
      }
    }
    for (int l = lane; l < q; l += 32) {
      double t = K.aC0[l];
      for (int i = 0; i < k; ++i) t -= Bent(l, i) * y[i];
      tq[l] = t;
    }
  } else if (warp0 == 1 && ext) {
    const int lane = threadIdx.x & 31;
    asm volatile("bar.sync 2, 64;" ::: "memory");
    if (lane < k) s_rinv1[lane] = 1.0 / Rent(lane, lane);
    // R^-1 by columns (lane c) from R staged in shared memory and the
    // diagonal's reciprocals (k <= BIE_RKMAX), then -B R^-1 and the new
    // columns' means
    for (int e = lane; e < k * k; e += 32) {
      const int cc = e / k, i = e - cc * k;   // consecutive lanes: one column
      s_R[i * BIE_RKMAX + cc] = i <= cc ? Rent(i, cc) : 0.0;
    }
    __syncwarp();
    if (lane < k) {
      const int cc = lane;
      for (int i = cc; i >= 0; --i) {
        double t = i == cc ? 1.0 : 0.0;
        for (int l = i + 1; l <= cc; ++l) t -= s_R[i * BIE_RKMAX + l] * Ri[l * BIE_RKMAX + cc];
        Ri[i * BIE_RKMAX + cc] = t * s_rinv1[i];
      }
      for (int i = cc + 1; i < k; ++i) Ri[i * BIE_RKMAX + cc] = 0.0;
    }
    __syncwarp();
    for (int e = lane; e < q * k; e += 32) {
      const int l = e / k, cc = e - l * k;
      double t = 0.0;
      for (int i = 0; i <= cc; ++i) t -= Bent(l, i) * Ri[i * BIE_RKMAX + cc];
      Mq[l * BIE_RKMAX + cc] = t;
    }
    __syncwarp();
    if (blockIdx.x == 0)
      for (int e = lane; e < K.nobs * k; e += 32) {
        const int o = e / k, cc = e - o * k;
        double t = 0.0;
        for (int i = 0; i <= cc; ++i) t += K.zmean[(size_t)i * BIE_MAXB + o] * Ri[i * BIE_RKMAX + cc];
        for (int l = 0; l < q; ++l) t += K.umean[(size_t)l * BIE_MAXB + o] * Mq[l * BIE_RKMAX + cc];
        K.umean[(size_t)(q + cc) * BIE_MAXB + o] = t;
      }
  }
  __syncthreads();
  __shared__ float RiF[BIE_RKMAX * BIE_RKMAX], MqF[BIE_RQMAX * BIE_RKMAX];
  if (ext) {   // single-precision copies for the extension's row loop
    for (int e = threadIdx.x; e < BIE_RKMAX * BIE_RKMAX; e += blockDim.x) RiF[e] = (float)Ri[e];
    for (int e = threadIdx.x; e < q * BIE_RKMAX; e += blockDim.x) MqF[e] = (float)Mq[e];
  }
  // the row loop's coefficients in the basis type, converted once per CTA
  VT* yv = reinterpret_cast<VT*>(y + update_fp64_doubles(m));   // y, k
  VT* tqv = yv + m;                                              // c_0 - B y, q
  VT* pav = tqv + BIE_RQMAX;                                     // dots of z_k, q + k
  VT* csv = pav + (BIE_RQMAX + m);                               // rotations, k
  VT* snv = csv + m;
  __shared__ VT s_inu;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    yv[i] = (VT)y[i];
    csv[i] = (VT)(i + 1 < k ? K.cs[i] : s_c);
    snv[i] = (VT)(i + 1 < k ? K.sn[i] : s_s);
  }
  for (int l = threadIdx.x; l < q; l += blockDim.x) tqv[l] = (VT)tq[l];
  if (ext)
    for (int i = threadIdx.x; i < q + k; i += blockDim.x) pav[i] = (VT)pa[i];
  if (threadIdx.x == 0) s_inu = s_nu > 1e-300 ? (VT)(1.0 / s_nu) : (VT)0;
  // P (Z y + U tq): obstacle rows lower by 3/2 of the combination's mean there
  if (K.nobs > 0 && threadIdx.x < K.nobs) {
    double t = 0.0;
    for (int i = 0; i < k; ++i) t += y[i] * K.zmean[(size_t)i * BIE_MAXB + threadIdx.x];
    for (int l = 0; l < q; ++l) t += tq[l] * K.umean[(size_t)l * BIE_MAXB + threadIdx.x];
    s_dm[threadIdx.x] = (double)K.obs_coef * t;
  }
  __syncthreads();
  const double scale = K.st->rnorm;
  const long long ld = K.ld;
  const VT* Cr = (const VT*)K.Crv;
  const VT* Ur = (const VT*)K.Urv;
  VT* Cw = (VT*)K.Crv;
  VT* Uw = (VT*)K.Urv;
  int r0, r1;
  slice_of(K.N, r0, r1);
  for (int mm = r0 + threadIdx.x; mm < r1; mm += blockDim.x) {
    // runs of eight terms in the basis type, the runs summed in FP64 (the
    // correction needs the inner tolerance's accuracy; x accumulates in FP64)
    // (each run's eight loads are issued before its products)
    double acc = 0.0;
    for (int i0 = 0; i0 < k; i0 += 8) {
      VT v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = i0 + u < k ? Z[(size_t)(i0 + u) * ld + mm] : (VT)0;
      VT run = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (i0 + u < k) run = fma(yv[i0 + u], v[u], run);
      acc += (double)run;
    }
    for (int l0 = 0; l0 < q; l0 += 8) {
      VT v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = l0 + u < q ? Ur[(size_t)(l0 + u) * ld + mm] : (VT)0;
      VT run = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (l0 + u < q) run = fma(tqv[l0 + u], v[u], run);
      acc += (double)run;
    }
    if (K.nobs > 0 && mm >= K.obs0) {
      int o = 0;
      while (o + 1 < K.nobs && mm >= K.obs_off[o + 1]) ++o;
      acc -= s_dm[o];
    }
    x[mm] += scale * acc;
    if (K.dlast) K.dlast[mm] = scale * acc;
    if (!ext) continue;
    // the extension in the vectors' own precision (the recycled pair has to
    // hold T U = C to that precision only): v_k = (z_k - C a'_C - V a'_V) / nu',
    // the rotations (C_{q+i}, i < k), and U_{q+c} = sum_i Z_i Ri[i][c] +
    // sum_l U_l Mq[l][c] with the k accumulators in registers
    VT vk = V[(size_t)k * ld + mm];
    for (int l = 0; l < q; ++l) vk -= pav[l] * Cr[(size_t)l * ld + mm];
    for (int i = 0; i < k; ++i) vk -= pav[q + i] * V[(size_t)i * ld + mm];
    vk *= s_inu;
    VT cur = V[mm];
    for (int i = 0; i < k; ++i) {
      const VT nxt = i + 1 < k ? V[(size_t)(i + 1) * ld + mm] : vk;
      const VT ci = csv[i], si = snv[i];
      Cw[(size_t)(q + i) * ld + mm] = ci * cur + si * nxt;
      cur = -si * cur + ci * nxt;
    }
    VT tu[BIE_RKMAX];
#pragma unroll
    for (int cc = 0; cc < BIE_RKMAX; ++cc) tu[cc] = (VT)0;
    for (int i = 0; i < k; ++i) {
      const VT zi = Z[(size_t)i * ld + mm];
#pragma unroll
      for (int cc = 0; cc < BIE_RKMAX; ++cc)
        if (cc >= i && cc < k) tu[cc] += (VT)RiF[i * BIE_RKMAX + cc] * zi;
    }
    for (int l = 0; l < q; ++l) {
      const VT ul = Ur[(size_t)l * ld + mm];
#pragma unroll
      for (int cc = 0; cc < BIE_RKMAX; ++cc)
        if (cc < k) tu[cc] += (VT)MqF[l * BIE_RKMAX + cc] * ul;
    }
#pragma unroll
    for (int cc = 0; cc < BIE_RKMAX; ++cc)
      if (cc < k) Uw[(size_t)(q + cc) * ld + mm] = tu[cc];
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
// Arnoldi steps the host enqueues ahead of the one whose status it waits for:
// one keeps the device busy (a step is ~90 us, the host's turn a few us) and
// leaves one launch pair to return at once after a cycle ends (two: 0.9% slower)
static const int kLookahead = 1;
// share of L2 filled with the stored matrix during each step's Gram-Schmidt kernels
static const double kL2PrefetchFrac = 0.25;
// Once the last residual r is small enough, and is the full-accuracy residual
// of omega (r_exact in run_solver), the next one is formed as r - D A_s d from
// the last increment d with a storage s cheaper than a direct hi + lo product
// of omega: A_s = A_hi (half the bytes) or the inner FP16 / BF16 storage (a
// quarter).  The storage holds the integral part K of A (the +-1/2 I is applied
// exactly), each entry rounded with unit roundoff eps_s; for independent
// roundings the error of A_s d is about eps_s / sqrt(3) max_l ||K e_l|| ||d||,
// with ||K e_l|| <= 0.18 on the 736- and 640-unknown systems (O(1/sqrt(N)))
// and ||d|| <= ||r|| / sigma_min(A) ~ 5 ||r|| there: about 0.5 eps_s ||r||.  A
// storage is taken when eps_s ||r|| <= kResidDrift ||b||: eps_hi = 2^-24
// (||r|| <= 1e-7 ||b||); the inner storage adds its own rounding (2^-11 FP16,
// 2^-8 BF16) to FP32 sums of ld / 32 terms per lane (FP16: ||r|| <= 1.1e-11
// ||b||).  Measured on 16383 unknowns: an updated and a direct residual of the
// third cycle differ by 3e-18 ||b||.  Only for rtol >= 1e-14: an updated
// residual does not see the rounding of omega itself (~1e-16 ||b||), so it
// must not decide convergence below that.
static const double kResidDrift = 6e-15;

template <class VT>
static bie_status enqueue_step(bie_ctx* c, KrylovArgs& K, int j, VT* V, VT* Z, VT* w,
                               int rowflip, const int* skip, size_t sh_h, int slot) {
  const bool ir = c->precision != BIE_FP64;
  const VT* vj = V + (size_t)j * c->ld;
  // the dots of w = A z_j with the basis [C, V_0..V_j] and with itself are
  // fused into the matrix-vector product (q + j + 2 <= 64 of them); on a
  // row-partitioned context the product covers the local rows only, so they
  // follow the allgather (k_cgs1)
  const bool part = partitioned(c);
  const bool fused = !part && (!ir || K.q + j + 1 < BIE_FUSED_DOTS);
  const int pr = prof_begin(c, 0, j);
  if (ir) {
    RightDefl df;
    memset(&df, 0, sizeof(df));
    df.obs0 = c->N;
    if (K.nobs > 0) {   // the product takes P z_j
      df.part = K.part3[j & 1] + (size_t)(K.q + j + 1) * BIE_PSTRIDE;
      df.mean_out = K.zmean + (size_t)j * BIE_MAXB;
      df.nobs = K.nobs;
      df.obs0 = K.obs0;
      for (int k = 0; k <= K.nobs; ++k) df.off[k] = K.obs_off[k];
      for (int k = 0; k < K.nobs; ++k) df.invM[k] = K.obs_invM[k];
      df.coef = K.obs_coef;
    }
    int np = 0;
    bie_status s = gemv_lowp_run_skip(c, (const float*)(const void*)vj, (float*)(void*)w, rowflip,
                                      skip, fused ? (const float*)(const void*)V : nullptr,
                                      (const float*)K.Crv, K.q, K.q + j,
                                      fused ? K.part1 : nullptr, &np, &df);
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
  k_dcgs<VT><<<BIE_NPART, 256, sh_h, c->stream>>>(K, j, V, Z, w, slot);
  BIE_LAUNCH_CHECK(c, "k_dcgs");
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
  VT *V, *Z, *w;
  double* r;
  BIE_GET(c, VT, ir ? "kr_V32" : "kr_V64", (size_t)(m + 1) * ld, V);
  BIE_GET(c, VT, ir ? "kr_Z32" : "kr_Z64", (size_t)(m + 1) * ld, Z);
  BIE_GET(c, VT, ir ? "kr_w32" : "kr_w64", ld, w);
  BIE_GET(c, double, "kr_r", ld, r);
  BIE_GET(c, double, "kr_H", (size_t)(m + 1) * m, K.H);
  BIE_GET(c, double, "kr_cs", m, K.cs);
  BIE_GET(c, double, "kr_sn", m, K.sn);
  BIE_GET(c, double, "kr_g", m + 1, K.g);
  BIE_GET(c, double, "kr_part1", (size_t)(m + 2 + BIE_RQMAX) * BIE_PSTRIDE, K.part1);
  BIE_GET(c, double, "kr_part3a", (size_t)(m + 2 + BIE_RQMAX + BIE_MAXB) * BIE_PSTRIDE, K.part3[0]);
  BIE_GET(c, double, "kr_part3b", (size_t)(m + 2 + BIE_RQMAX + BIE_MAXB) * BIE_PSTRIDE, K.part3[1]);
  BIE_GET(c, double, "kr_hraw", m + 2, K.hraw);
  BIE_GET(c, double, "kr_zmean", (size_t)(m + 1) * BIE_MAXB, K.zmean);
  // the refined schemes keep a recycled subspace across their cycles (starts
  // empty for every solve); the plain FP64 scheme runs one restarted GMRES
  const bool recycle = ir;
  K.q = 0;
  if (recycle) {
    VT *Cr, *Ur;
    BIE_GET(c, VT, "kr_C32", (size_t)BIE_RQMAX * ld, Cr);
    BIE_GET(c, VT, "kr_U32", (size_t)BIE_RQMAX * ld, Ur);
    K.Crv = Cr;
    K.Urv = Ur;
    BIE_GET(c, double, "kr_B", (size_t)m * BIE_RQMAX, K.Bm);
    BIE_GET(c, double, "kr_braw", BIE_RQMAX, K.braw);
    BIE_GET(c, double, "kr_aC0", BIE_RQMAX, K.aC0);
    BIE_GET(c, double, "kr_umean", (size_t)BIE_RQMAX * BIE_MAXB, K.umean);
    BIE_GET(c, double, "kr_dlast", ld, K.dlast);
  }
  // the refined schemes' inner solves take the right preconditioner P over
  // the obstacles: on the operator of eq. AB:cor or its transpose (the
  // adjoint) the obstacles are blocks 2 .. nb-1 and coef = 3/2; on the
  // vortex-sheet solid system (eq. lin:sys2; bottom = block 0) blocks
  // 1 .. nb-1 and coef = 1/2.  The plain FP64 scheme and the App. B and
  // gamma_t operators run without it.
  int ob = 0;
  K.obs_coef = 0.f;
  if (ir && c->variant == 0 && !c->asm_noE) {
    if (!c->asm_vs && c->nb > 2) {
      ob = 2;
      K.obs_coef = 1.5f;
    } else if (c->asm_vs && c->nb > 1) {
      ob = 1;
      K.obs_coef = 0.5f;
    }
  }
  K.nobs = ob > 0 ? c->nb - ob : 0;
  K.obs0 = K.nobs > 0 ? c->off[ob] : c->N;
  for (int k = 0; k < K.nobs; ++k) {
    K.obs_off[k] = c->off[ob + k];
    K.obs_invM[k] = (float)(1.0 / (double)c->M[ob + k]);
  }
  K.obs_off[K.nobs] = K.nobs > 0 ? c->off[c->nb] : c->N;
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
    // the product's CTA b streams the rows [b R, (b + 1) R), R = ceil(rows / CTAs)
    K.pf_nchunks = gemv_num_ctas();
    const long long R = (local_rows(c) + K.pf_nchunks - 1) / K.pf_nchunks;
    K.pf_stride = R * ld * (f32 ? 4 : 2);
    K.pf_total = (long long)abytes;
    if (K.pf_bytes / K.pf_nchunks > K.pf_stride) K.pf_bytes = K.pf_stride * K.pf_nchunks;
  }
  const int* skip = &K.st->inner_done;
  const size_t sh_h = sizeof(double) * dcgs_smem_doubles(m);
  const int rowflip = o->row_flip ? 1 : 0;
  double inner_tol = o->inner_tol;
  if (inner_tol <= 0.0) {   // with the recycled space a tighter cycle costs no more steps
    inner_tol = c->precision == BIE_FP64 ? 0.0 : c->precision == BIE_FP32_IR ? 1e-4 : 5e-4;
  }
  const bool x0 = o->x0 != 0;   // omega holds an initial guess
  if (!x0) BIE_CUDA_TRY(c, cudaMemsetAsync(x, 0, sizeof(double) * c->N, c->stream));
  BIE_CUDA_TRY(c, cudaMemsetAsync(w, 0, sizeof(VT) * ld, c->stream));
  int slot = 0, total_iters = 0, cycles = 0;
  bool converged = false, nonfinite = false, stagnated = false;
  double last_rn = 0.0, bnorm = 0.0, prev_rn = 0.0;
  int stall = 0, bnorm_slot = -1;
  bool have_d = false;   // dlast holds the last update's increment
  // r is the full-accuracy residual of omega (D b, a direct hi + lo product, or
  // updated from one); a residual of the FP32 part alone is not, and nothing
  // may be updated from it: its own error would stay in every later one
  bool r_exact = false;
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
      r_exact = true;
    } else if (K.dlast && have_d && r_exact && o->rtol >= 1e-14 && !partitioned(c) &&
               (c->precision == BIE_FP16_IR || c->precision == BIE_BF16_IR) &&
               ((c->precision == BIE_FP16_IR ? 0x1p-11 : 0x1p-8) + (double)(ld / 32) * 0x1p-24) *
                       last_rn <= kResidDrift * bnorm) {
      // r <- r - D A_16 d in the inner storage (the increment d of the last update)
      float *df, *yf;
      BIE_GET(c, float, "kr_df", ld, df);
      BIE_GET(c, float, "kr_yf", ld, yf);
      k_inc_to_f<<<(unsigned)((ld + 255) / 256), 256, 0, c->stream>>>(c->N, ld, K.dlast, df);
      BIE_LAUNCH_CHECK(c, "k_inc_to_f");
      const int pr = prof_begin(c, 0, -1);
      bie_status s = gemv_lowp_run_skip(c, df, yf, rowflip, nullptr, nullptr, nullptr, 0, 0, nullptr,
                                        nullptr, nullptr);
      if (s != BIE_OK) return s;
      prof_end(c, pr);
      k_resid_sub<<<BIE_NPART, 256, 0, c->stream>>>(c->N, yf, r, K.partn);
      BIE_LAUNCH_CHECK(c, "k_resid_sub");
    } else if (K.dlast && have_d && r_exact && o->rtol >= 1e-14 &&
               0x1p-24 * last_rn <= kResidDrift * bnorm) {
      // r <- r - D A_hi d (the increment d of the last update)
      double* rd;
      BIE_GET(c, double, "kr_rd", ld, rd);
      k_flip_copy<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->N, r, blk, rowflip, rd);
      BIE_LAUNCH_CHECK(c, "k_flip_copy");
      double* ypart = nullptr;
      int npanel = 0;
      const int pr = prof_begin(c, 4, -1);
      bie_status s = gemv_full_partials_skip(c, K.dlast, &ypart, &npanel, nullptr, 1);
      if (s != BIE_OK) return s;
      prof_end(c, pr);
      s = gemv_full_finish_skip(c, ypart, npanel, K.dlast, rowflip, rd, r, nullptr,
                                partitioned(c) ? nullptr : K.partn, nullptr, nullptr, 0, nullptr);
      if (s != BIE_OK) return s;
      if (partitioned(c)) {
        s = part_allgather(c, r, 8, c->N);
        if (s != BIE_OK) return s;
        k_norm_parts<<<BIE_NPART, 256, 0, c->stream>>>(c->N, r, K.partn);
        BIE_LAUNCH_CHECK(c, "k_norm_parts");
      }
    } else {
      double* ypart = nullptr;
      int npanel = 0;
      // while the last residual is above 1e-4 ||b||, the next one (about
      // inner_tol times smaller) only needs a few digits: FP32 part alone
      // (the residual of an initial guess is always taken in full)
      const int hi_only = (ir && cycle > 0 && last_rn > 1e-4 * bnorm) ? 1 : 0;
      r_exact = !hi_only;
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
    k_start<VT><<<BIE_NPART, 256, 0, c->stream>>>(K, r, V, Z, o->rtol, inner_tol, cycle == 0 && !x0,
                                                  start_slot);
    BIE_LAUNCH_CHECK(c, "k_start");
    BIE_CUDA_TRY(c, cudaEventRecord(c->evs[start_slot % BIE_NSLOTS], c->stream));
    const int step0 = slot;
    int enq = 0;
    // steps 0..L-1 go in before the start flags are read (they return at once
    // if the cycle is already converged)
    while (enq < m && enq < kLookahead) {
      bie_status s = enqueue_step<VT>(c, K, enq, V, Z, w, rowflip, skip, sh_h, step0 + enq);
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
      // stagnation: three refinement cycles in a row that do not bring the true
      // residual 10% below the smallest one seen (at the rounding floor it
      // fluctuates, and a 10% dip from one cycle to the next means nothing)
      if (cycle > 0 && !converged && !nonfinite) {
        stall = (last_rn > 0.9 * prev_rn) ? stall + 1 : 0;
        if (stall >= 3) stagnated = true;
      }
      prev_rn = cycle == 0 ? last_rn : std::min(prev_rn, last_rn);
    }
    int done_steps = 0;
    if (!nonfinite && !converged && !stagnated && cycle < o->max_cycles) {
      for (int j = 0; j < m; ++j) {
        while (enq < m && enq <= j + kLookahead) {
          bie_status s = enqueue_step<VT>(c, K, enq, V, Z, w, rowflip, skip, sh_h, step0 + enq);
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
    // the cycle's space joins the recycled one while it fits
    const int ext = (recycle && done_steps >= 1 && done_steps <= BIE_RKMAX &&
                     K.q + done_steps <= BIE_RQMAX) ? 1 : 0;
    k_update<VT><<<BIE_NPART, 256, sizeof(double) * update_smem_doubles(m), c->stream>>>(K, V, Z, x,
                                                                                       ext);
    BIE_LAUNCH_CHECK(c, "k_update");
    if (ext) K.q += done_steps;
    have_d = done_steps > 0;   // k_update leaves omega (and dlast) alone without a step
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
