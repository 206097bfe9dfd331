// Batched solve of many independent problems of uneven size.
//
// Each problem is the system of eq. lin:sys of its own geometry (Table 1, eq.
// Awb) solved by the GMRES-IR scheme of the single-problem solver: a cycle
// computes r = D(b - A omega) with the ~48-bit hi + lo operator, runs GMRES(m)
// with CGS2 on the low-precision operator to the cycle's relative tolerance,
// and updates omega in FP64.  The batch runs all problems' cycles in one
// cooperative (persistent) kernel, one CTA of 1024 threads per SM:
//
//   for each cycle:   RESID   r = D(b - A omega) rows, ||r||^2 per unit
//                     START   ||r||, convergence, v_0 = r/||r||
//                     for j < m (while some problem iterates):
//                        GEMV  w = D A v_j rows, first-pass dots V^T w per unit
//                        CGS2  h1 = sum of those; w' = w - V h1; V^T w', ||w'||^2
//                        CGS3  v_{j+1} = (w' - V h2)/beta; Hessenberg, Givens (leader)
//                     UPDATE  omega += ||r|| V y
//
// with a grid barrier between phases.  Problems advance in lock step by
// cycle; a problem whose cycle has converged skips the remaining steps at the
// cost of a flag test per unit.  Work in every phase is a list of units
// (row ranges of one problem) taken dynamically from a counter, so the
// active problems' rows spread over all SMs whatever their number:
//   GEMV units  a tuned number of bytes of stored matrix (default 1 MB: 32
//               rows at N = 12288, 256 at 1024; at least 32 rows),
//   vector units 1024 rows (one per thread).
// The GEMV unit size is chosen by timing the solver kernel for each candidate
// (256 KB .. 4 MB) on the first run of a set of problems (the autotuner).
// Every unit writes its partial sums to its own slot and every reduction adds
// a problem's slots in a fixed order, so results do not depend on the
// schedule.  The barrier spins on a generation counter with an iteration
// limit; a CTA that gives up sets the error flag and every CTA returns (the
// host reports BIE_ERR_TIMEOUT).
//
// Around the kernel the per-problem node tables, assembly, right-hand side
// and normal velocity run on eight forked streams, and the whole sequence is
// captured once into a CUDA graph that later runs replay.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "nvtx.cuh"
#include "gemv_dot.cuh"

#define BT_THREADS 1024
#define BT_VROWS 1024
#define BT_MAXM 63
#define BT_MAXLD 16384
#define BT_STREAMS 8
#define BT_RQ 32     // recycled columns kept at most per problem
#define BT_RK 16     // columns a cycle may add

struct BtProb {
  int N, M0;
  long long ld;
  int g0, ng;     // GEMV units (partial slots) [g0, g0 + ng)
  int v0, nv;     // vector units [v0, v0 + nv)
  const float* Ahi;
  const float* Alo;
  const void* A16;
  const float* wgt;
  const double* wgt64;
  const float* sgn;
  const int* blk;
  const double* b;
  double* x;
  double* r;
  double* dlast;  // the last update's increment of x (valid while BtStat::have_d)
  float* V;       // (m + 1) x ld basis
  float* w;       // ld
  double* H;      // (m + 1) x m, column j at H + j (m + 1)
  double* cs;
  double* sn;
  double* g;
  double* y;
  // right preconditioner P over the obstacles (see RightDefl); the GEMV unit
  // of slot g0 stores the means of v_j in mu[j][k]
  int nobs;
  int obs_off[BIE_MAXB + 1];
  double* mu;     // (m + 1) x BIE_MAXB
  // recycled subspace across the problem's cycles (GCRO-DR, as in the
  // single-problem solver): T U = C, C orthonormal, q = BtStat::qc[cycle & 1]
  float* Cr;      // BT_RQ x ld
  float* Ur;      // BT_RQ x ld
  double* Bm;     // m x BT_RQ: C-part of Hessenberg column j at Bm + j BT_RQ
  double* c0;     // C-part of the cycle's start vector r / ||r||
  double* umean;  // BT_RQ x BIE_MAXB: means of U's columns over the obstacles
};

struct BtStat {
  int active;      // still refining
  int inner;       // in the Arnoldi loop of the current cycle
  int iters;       // steps of the current cycle
  int total_iters;
  int cycles;
  int converged;
  int nonfinite;
  int have_d;      // the last update changed x by dlast
  double rnorm;
  double bnorm;
  double inner_tol;
  double resid_est;
  double rbytes;   // stored-matrix bytes read by the problem's residual products
  int qc[2];       // recycled columns in use: cycle c reads qc[c & 1]
  int rexact;      // r is the full-accuracy residual of x (see bt_resid_mode)
  int pad;
};

struct BtUnit {
  int p, r0, r1, slot;
};

struct BtArgs {
  int P, m, ngu, nvu, rowflip, max_cycles;
  double rtol, inner_tol;
  double eps16;    // unit roundoff of the FP16 / BF16 inner storage (0: FP32 storage)
  const BtProb* prob;
  const BtUnit* gunits;
  const BtUnit* vunits;
  BtStat* st;
  double* part1;   // [m + 1 + BT_RQ][ngu]
  double* part2;   // [m + 2 + BT_RQ][nvu]
  double* partn;   // [ngu]
  double* partc;   // [BT_RQ][ngu]: C_i^T r over each GEMV unit's rows
  unsigned* bar;   // [0] arrivals, [1] generation, [2..4] unit counters
  int* err;
  unsigned spin_limit;
};

// ---------------------------------------------------------------------------
// grid barrier with a bounded wait
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool bt_barrier(unsigned* bar, int* err, unsigned spin_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned it = 0;
      while (*gen == g0) {
        if (*(volatile int*)err) break;
        if (++it > spin_limit) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

// Thread 0 takes the next unit of the phase and tests its problem's flag
// (which: 0 none, 1 active, 2 inner); every thread gets the same answer:
// 0 no unit left, 1 skip, 2 work on *s_unit.
__device__ __forceinline__ int bt_take(unsigned* ctr, const BtUnit* units, int count,
                                       const BtStat* st, int which, BtUnit* s_unit, int* s_state) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const int u = (int)atomicAdd(ctr, 1u);
    int state = 0;
    if (u < count) {
      const BtUnit U = units[u];
      *s_unit = U;
      const int f = which == 0 ? 1 : (which == 1 ? __ldcg(&st[U.p].active) : __ldcg(&st[U.p].inner));
      state = f ? 2 : 1;
    }
    *s_state = state;
  }
  __syncthreads();
  return *s_state;
}

// out[i] = sum_{s < ns} part[i stride + s0 + s], i < cnt; 16 threads per row,
// fixed order.  Ends with __syncthreads.
__device__ __forceinline__ void bt_reduce(const double* part, int stride, int s0, int ns, int cnt,
                                          double* out, float* outf = nullptr) {
  const int q = threadIdx.x & 15;
  for (int base = 0; base < cnt; base += (int)(blockDim.x >> 4)) {
    const int i = base + (int)(threadIdx.x >> 4);
    double s = 0.0;
    if (i < cnt) {
      const double* row = part + (size_t)i * stride + s0;
      for (int c = q; c < ns; c += 16) s += __ldcg(row + c);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (i < cnt && q == 0) {
      out[i] = s;
      if (outf) outf[i] = (float)s;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double bt_block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = red[threadIdx.x];
    t = warp_sum(t);
  }
  return t;   // valid in thread 0
}

// ---------------------------------------------------------------------------
// phases, one unit at a time
// ---------------------------------------------------------------------------
// How the residual of a cycle is formed (the single-problem solver's rules):
// 0 r = D b (cycle 0); 1 direct hi + lo product of x; 2 the FP32 part alone
// (while the last residual is above 1e-4 ||b||); 3 r - D A_hi d and 4
// r - D A_16 d from the last increment d, once r is the full-accuracy residual
// of x and the storage's rounding times ||r|| stays below 6e-15 ||b|| (FP32 sums
// of ld / 32 terms per lane added to the FP16 / BF16 rounding), for rtol >= 1e-14.
__device__ __forceinline__ int bt_resid_mode(const BtArgs& a, const BtStat* S, int cycle, long long ld) {
  if (cycle == 0) return 0;
  const double rn = __ldcg(&S->rnorm), bn = __ldcg(&S->bnorm);
  if (__ldcg(&S->have_d) && __ldcg(&S->rexact) && a.rtol >= 1e-14) {
    if (a.eps16 > 0.0 && (a.eps16 + (double)(ld / 32) * 0x1p-24) * rn <= 6e-15 * bn) return 4;
    if (0x1p-24 * rn <= 6e-15 * bn) return 3;
  }
  return rn > 1e-4 * bn ? 2 : 1;
}

// r by bt_resid_mode over the unit's rows; partn[slot] = sum r^2 and the dots
// C_i^T r of the recycled columns
template <class TA>
__device__ void bt_resid(const BtArgs& a, const BtProb& P, const BtUnit& U, int cycle, int mode,
                         float* xh, float* xl, double* red) {
  double acc2 = 0.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool upd = mode >= 3;
  if (U.r0 == 0 && threadIdx.x == 0 && mode > 0) {   // the whole product, counted once
    const double per = mode == 1 ? 8.0 : (mode == 4 ? (double)sizeof(TA) : 4.0);
    a.st[U.p].rbytes += per * (double)P.N * (double)P.ld;
  }
  const double* src = upd ? P.dlast : P.x;   // the vector multiplied
  auto finish_row = [&](int m, double y) {   // y = (A src)_m less its diagonal term
    y += (double)P.sgn[m] * __ldcg(src + m);
    const bool flip = a.rowflip && P.blk[m] == 0;
    const double base = upd ? (flip ? -__ldcg(P.r + m) : __ldcg(P.r + m)) : P.b[m];
    double o = base - y;
    if (flip) o = -o;
    P.r[m] = o;
    acc2 += o * o;
  };
  if (mode == 0) {
    for (int m = U.r0 + (int)threadIdx.x; m < U.r1; m += blockDim.x) {
      double v = P.b[m];
      if (a.rowflip && P.blk[m] == 0) v = -v;
      P.r[m] = v;
      acc2 += v * v;
    }
  } else if (mode == 4) {   // the inner storage, FP32 sums (as the Arnoldi products)
    for (int c = threadIdx.x; c < P.ld; c += blockDim.x)
      xh[c] = (c < P.N) ? (float)__ldcg(src + c) * P.wgt[c] : 0.f;
    __syncthreads();
    const TA* A16 = reinterpret_cast<const TA*>(P.A16);
    constexpr int E = Dot16<TA>::E;
    const int nvec = (int)(P.ld / E);
    for (int m = U.r0 + warp; m < U.r1; m += 32) {
      const uint4* row = reinterpret_cast<const uint4*>(A16 + (size_t)m * P.ld);
      float acc = 0.f;
      int v = lane;
      for (; v + 32 * 3 < nvec; v += 32 * 4) {
        uint4 q4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q4[u] = __ldcs(row + v + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = Dot16<TA>::run(acc, q4[u], xh + (size_t)(v + 32 * u) * E);
      }
      for (; v < nvec; v += 32) acc = Dot16<TA>::run(acc, __ldcs(row + v), xh + (size_t)v * E);
      acc = warp_sum(acc);
      if (lane == 0) finish_row(m, (double)acc);
    }
  } else {   // double-float products with hi + lo, or with hi alone (modes 2, 3)
    const bool hi_only = mode != 1;
    for (int c = threadIdx.x; c < P.ld; c += blockDim.x) {
      const double v = (c < P.N) ? __ldcg(src + c) * P.wgt64[c] : 0.0;
      const dfl d = df_from_double(v);
      xh[c] = d.hi;
      xl[c] = d.lo;
    }
    __syncthreads();
    const int nvec = (int)(P.ld / 4);
    const float4* xh4 = reinterpret_cast<const float4*>(xh);
    const float4* xl4 = reinterpret_cast<const float4*>(xl);
    for (int m = U.r0 + warp; m < U.r1; m += 32) {
      const float4* rh = reinterpret_cast<const float4*>(P.Ahi + (size_t)m * P.ld);
      const float4* rl = reinterpret_cast<const float4*>(P.Alo + (size_t)m * P.ld);
      double acc = 0.0;
      int v = lane;
      for (; v + 32 * 3 < nvec; v += 32 * 4) {
        float4 ah[4], al[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ah[u] = __ldcs(rh + v + 32 * u);
          al[u] = hi_only ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldcs(rl + v + 32 * u);
        }
        dfl run = {0.f, 0.f};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 h = xh4[v + 32 * u], l = xl4[v + 32 * u];
          run = df_acc_prod(run, ah[u].x, al[u].x, h.x, l.x);
          run = df_acc_prod(run, ah[u].y, al[u].y, h.y, l.y);
          run = df_acc_prod(run, ah[u].z, al[u].z, h.z, l.z);
          run = df_acc_prod(run, ah[u].w, al[u].w, h.w, l.w);
        }
        acc += (double)run.hi + (double)run.lo;
      }
      for (; v < nvec; v += 32) {
        const float4 ah = __ldcs(rh + v);
        const float4 al = hi_only ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldcs(rl + v);
        const float4 h = xh4[v], l = xl4[v];
        dfl run = {0.f, 0.f};
        run = df_acc_prod(run, ah.x, al.x, h.x, l.x);
        run = df_acc_prod(run, ah.y, al.y, h.y, l.y);
        run = df_acc_prod(run, ah.z, al.z, h.z, l.z);
        run = df_acc_prod(run, ah.w, al.w, h.w, l.w);
        acc += (double)run.hi + (double)run.lo;
      }
      acc = warp_sum(acc);
      if (lane == 0) finish_row(m, acc);
    }
  }
  const double s = bt_block_sum(acc2, red);
  if (threadIdx.x == 0) a.partn[U.slot] = s;
  const int q = __ldcg(&a.st[U.p].qc[cycle & 1]);
  if (q > 0) {   // C_i^T r over the unit's rows (r written above by this CTA)
    __syncthreads();
    for (int i = warp; i < q; i += 32) {
      const float* ci = P.Cr + (size_t)i * P.ld;
      double t = 0.0;
      for (int m = U.r0 + lane; m < U.r1; m += 32) t += (double)ci[m] * __ldcg(P.r + m);
      t = warp_sum(t);
      if (lane == 0) a.partc[(size_t)i * a.ngu + U.slot] = t;
    }
  }
  __syncthreads();   // xh, xl, red reused by the next unit
}

// ||r|| and c_0 = C^T r / ||r|| from the problem's GEMV-unit partials;
// v_0 = (r / ||r|| - C c_0) / nu_0 with nu_0^2 = 1 - |c_0|^2 (the part of the
// start vector outside the recycled space); the leader updates the state
__device__ void bt_start(const BtArgs& a, const BtProb& P, const BtUnit& U, int p, int cycle,
                         double* sh) {
  BtStat* S = a.st + p;
  const int q = __ldcg(&S->qc[cycle & 1]);
  bt_reduce(a.partn, a.ngu, P.g0, P.ng, 1, sh);
  if (q > 0) bt_reduce(a.partc, a.ngu, P.g0, P.ng, q, sh + 1);
  const double rn = sqrt(sh[0]);
  __shared__ double s_nu0;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < q; ++i) t += (sh[1 + i] / rn) * (sh[1 + i] / rn);
    s_nu0 = sqrt(fmax(1.0 - t, 0.0));
  }
  __syncthreads();
  const double nu0 = s_nu0;
  const double bn = (cycle == 0) ? rn : __ldcg(&S->bnorm);
  const bool bad = !isfinite(rn);
  const bool conv = !bad && (rn <= a.rtol * bn || rn == 0.0);
  const bool done = bad || conv || cycle >= a.max_cycles;
  // r lies in the recycled space (to rounding): the correction is U c_0 alone
  const bool nokrylov = !done && !(nu0 > 1e-12);
  if (!done && !nokrylov) {
    const double inv = 1.0 / rn, inu = 1.0 / nu0;
    for (int m = U.r0 + (int)threadIdx.x; m < U.r1; m += blockDim.x) {
      double v = __ldcg(P.r + m) * inv;
      for (int i = 0; i < q; ++i) v -= (sh[1 + i] * inv) * (double)__ldcg(P.Cr + (size_t)i * P.ld + m);
      P.V[m] = (float)(v * inu);
    }
  }
  if (U.r0 == 0 && threadIdx.x == 0) {
    // the mode this cycle's residual took (from the state before this update)
    S->rexact = bt_resid_mode(a, S, cycle, P.ld) != 2 ? 1 : 0;
    if (cycle == 0) S->bnorm = rn;
    S->rnorm = rn;
    S->nonfinite = bad ? 1 : 0;
    S->converged = conv ? 1 : 0;
    S->active = done ? 0 : 1;
    S->inner = (done || nokrylov) ? 0 : 1;
    S->iters = 0;
    S->resid_est = 1.0;
    S->inner_tol = fmax(a.inner_tol, 0.5 * a.rtol * bn / fmax(rn, 1e-300));
    for (int i = 0; i < q; ++i) P.c0[i] = sh[1 + i] / rn;
    P.g[0] = nokrylov ? 0.0 : nu0;
    for (int i = 1; i <= a.m; ++i) P.g[i] = 0.0;
  }
  __syncthreads();
}

// basis vector i of the cycle: C_i (i < q), V_{i-q}
__device__ __forceinline__ const float* bt_q(const BtProb& P, int q, int i) {
  return i < q ? P.Cr + (size_t)i * P.ld : P.V + (size_t)(i - q) * P.ld;
}

// w = D (A P v_j); part1[i][slot] = sum over the unit's rows of Q_i w, i <= q + j
template <class TA>
__device__ void bt_gemv(const BtArgs& a, const BtProb& P, const BtUnit& U, int q, int j, float* xs,
                        double (*red)[65], double* red1) {
  const float* vj = P.V + (size_t)j * P.ld;
  {   // v_j / M_l staged as 16-byte vectors (ld is a multiple of 64), entries past N zero
    const float4* x4 = reinterpret_cast<const float4*>(vj);
    const float4* w4 = reinterpret_cast<const float4*>(P.wgt);
    float4* xs4 = reinterpret_cast<float4*>(xs);
#pragma unroll 4
    for (int c = threadIdx.x; c < (int)(P.ld >> 2); c += blockDim.x) {
      const float4 xa = __ldcg(x4 + c), wa = w4[c];
      const int e = 4 * c;
      float4 o;
      o.x = e < P.N ? xa.x * wa.x : 0.f;
      o.y = e + 1 < P.N ? xa.y * wa.y : 0.f;
      o.z = e + 2 < P.N ? xa.z * wa.z : 0.f;
      o.w = e + 3 < P.N ? xa.w * wa.w : 0.f;
      xs4[c] = o;
    }
  }
  __syncthreads();
  __shared__ float s_xc[BIE_MAXB];   // 3/2 v_j mean over obstacle k
  if (P.nobs > 0) {   // the staged x / M_k summed over obstacle k is its mean
    for (int k = 0; k < P.nobs; ++k) {
      double t = 0.0;
      for (int c = P.obs_off[k] + (int)threadIdx.x; c < P.obs_off[k + 1]; c += blockDim.x)
        t += (double)xs[c];
      t = bt_block_sum(t, red1);
      if (threadIdx.x == 0) {
        s_xc[k] = (float)(1.5 * t);
        if (U.slot == P.g0) P.mu[(size_t)j * BIE_MAXB + k] = t;
      }
    }
    __syncthreads();
  }
  const TA* A = reinterpret_cast<const TA*>(sizeof(TA) == 4 ? (const void*)P.Ahi : P.A16);
  constexpr int E = Dot16<TA>::E;
  const int nvec = (int)(P.ld / E);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double d0 = 0.0, d1 = 0.0;
  const int nd = q + j;   // dots with Q_0..Q_nd
  const float* vq0 = lane <= nd ? bt_q(P, q, lane) : nullptr;
  const float* vq1 = lane + 32 <= nd ? bt_q(P, q, lane + 32) : nullptr;
  for (int m = U.r0 + warp; m < U.r1; m += 32) {
    const uint4* row = reinterpret_cast<const uint4*>(A + (size_t)m * P.ld);
    float acc = 0.f;
    int v = lane;
    for (; v + 32 * 3 < nvec; v += 32 * 4) {
      uint4 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = __ldcs(row + v + 32 * u);
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = Dot16<TA>::run(acc, q[u], xs + (size_t)(v + 32 * u) * E);
    }
    for (; v < nvec; v += 32) acc = Dot16<TA>::run(acc, __ldcs(row + v), xs + (size_t)v * E);
    acc = warp_sum(acc);
    float r = fmaf(P.sgn[m], __ldcg(vj + m), acc);
    if (P.nobs > 0 && m >= P.obs_off[0]) {   // A P v = A v + 3/2 mu_k on obstacle k's rows
      int k = 0;
      while (k + 1 < P.nobs && m >= P.obs_off[k + 1]) ++k;
      r += s_xc[k];
    }
    if (a.rowflip && P.blk[m] == 0) r = -r;
    if (lane == 0) P.w[m] = r;
    if (vq0) d0 += (double)__ldcg(vq0 + m) * (double)r;
    if (vq1) d1 += (double)__ldcg(vq1 + m) * (double)r;
  }
  red[warp][lane] = d0;
  red[warp][lane + 32] = d1;
  __syncthreads();
  for (int i = warp; i <= nd; i += 32) {   // a warp per dot: a tree, not a chain of 32
    const double s = warp_sum(red[lane][i]);
    if (lane == 0) a.part1[(size_t)i * a.ngu + U.slot] = s;
  }
  __syncthreads();
}

// acc - sum_{i <= nd} h[i] Q_i[m], eight loads in flight per L2 round trip; h is the
// single-precision copy of the coefficients (one conversion per CTA, not per row)
__device__ __forceinline__ float bt_subtract(const BtProb& P, int q, int nd, const float* h,
                                             int m, float acc) {
  int i = 0;
  for (; i + 7 <= nd; i += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(bt_q(P, q, i + u) + m);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc -= h[i + u] * v[u];
  }
  for (; i <= nd; ++i) acc -= h[i] * __ldcg(bt_q(P, q, i) + m);
  return acc;
}

// h1 = sum part1; w' = w - Q h1 (rows); part2[i][slot] = Q_i . w' (i <= q + j),
// ||w'||^2 at q + j + 1 (Q = [C, V], see bt_q)
__device__ void bt_cgs2(const BtArgs& a, const BtProb& P, const BtUnit& U, int q, int j, double* sh) {
  const int nd = q + j;
  __shared__ float hf[BT_RQ + BT_MAXM + 2];
  bt_reduce(a.part1, a.ngu, P.g0, P.ng, nd + 1, sh, hf);
  const int m = U.r0 + (int)threadIdx.x;
  if (m < U.r1) P.w[m] = bt_subtract(P, q, nd, hf, m, __ldcg(P.w + m));
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= nd + 1; i += 32) {
    // each lane's 32 products summed in FP32 runs of eight, the runs in FP64
    double s = 0.0;
    float run = 0.f;
    int cnt = 0;
    const float* qi = i <= nd ? bt_q(P, q, i) : nullptr;
    for (int mm = U.r0 + lane; mm < U.r1; mm += 32) {
      const float wv = __ldcg(P.w + mm);
      run = fmaf(qi ? __ldcg(qi + mm) : wv, wv, run);
      if (++cnt == 8) {
        s += (double)run;
        run = 0.f;
        cnt = 0;
      }
    }
    s += (double)run;
    s = warp_sum(s);
    if (lane == 0) a.part2[(size_t)i * a.nvu + U.slot] = s;
  }
  __syncthreads();
}

// h2 = sum part2, beta = sqrt(||w'||^2 - ||h2||^2), v_{j+1} = (w' - Q h2)/beta;
// the leader unit (first rows) updates the Hessenberg column (the V-part of
// h1 + h2; its C-part is column j of B), applies the Givens rotations, tests
// the cycle and, when it ends, solves R y = g.  A cycle ends by q + j + 1 = 63
// at the latest, so the fused dots of the product cover the whole basis.
__device__ void bt_cgs3(const BtArgs& a, const BtProb& P, const BtUnit& U, int p, int q, int j,
                        double* sh, int* s_flag) {
  const bool leader = (U.r0 == 0);
  const int nd = q + j;
  __shared__ float hf[BT_RQ + BT_MAXM + 2];
  __shared__ double s_beta;
  __shared__ float s_inv;
  bt_reduce(a.part2, a.nvu, P.v0, P.nv, nd + 2, sh, hf);
  if (leader) bt_reduce(a.part1, a.ngu, P.g0, P.ng, nd + 1, sh + (nd + 2));
  if (threadIdx.x < 32) {   // beta once per CTA (FP64 is a narrow pipe here)
    double hh = 0.0;
    for (int i = threadIdx.x; i <= nd; i += 32) hh += sh[i] * sh[i];
    hh = warp_sum(hh);
    if (threadIdx.x == 0) {
      const double b = sqrt(fmax(sh[nd + 1] - hh, 0.0));
      s_beta = b;
      s_inv = (b > 1e-300 && isfinite(b)) ? (float)(1.0 / b) : 0.f;
    }
  }
  __syncthreads();
  const double beta = s_beta;
  const bool breakdown = !(beta > 1e-300) || !isfinite(beta);
  if (!breakdown) {
    const int m = U.r0 + (int)threadIdx.x;
    if (m < U.r1)
      P.V[(size_t)(j + 1) * P.ld + m] = bt_subtract(P, q, nd, hf, m, __ldcg(P.w + m)) * s_inv;
  }
  if (!leader) {
    __syncthreads();
    return;
  }
  BtStat* S = a.st + p;
  const int mm = a.m;
  const int mend = min(mm, 63 - q);
  if (threadIdx.x == 0) {
    double* Hj = P.H + (size_t)j * (mm + 1);
    for (int i = 0; i <= j; ++i) Hj[i] = sh[nd + 2 + q + i] + sh[q + i];
    for (int l = 0; l < q; ++l) P.Bm[(size_t)j * BT_RQ + l] = sh[nd + 2 + l] + sh[l];
    Hj[j + 1] = beta;
    for (int i = 0; i < j; ++i) {
      const double t = P.cs[i] * Hj[i] + P.sn[i] * Hj[i + 1];
      Hj[i + 1] = -P.sn[i] * Hj[i] + P.cs[i] * Hj[i + 1];
      Hj[i] = t;
    }
    const double rr = hypot(Hj[j], Hj[j + 1]);
    double c = 1.0, s = 0.0;
    if (rr > 0.0) {
      c = Hj[j] / rr;
      s = Hj[j + 1] / rr;
    }
    P.cs[j] = c;
    P.sn[j] = s;
    Hj[j] = rr;
    Hj[j + 1] = 0.0;
    P.g[j + 1] = -s * P.g[j];
    P.g[j] = c * P.g[j];
    const double est = fabs(P.g[j + 1]);
    S->iters = j + 1;
    S->resid_est = est;
    const bool nf = !isfinite(est) || !isfinite(rr);
    if (nf) {
      S->nonfinite = 1;
      S->active = 0;
    }
    const bool end = nf || breakdown || est <= S->inner_tol || j + 1 >= mend;
    if (end) S->inner = 0;
    *s_flag = (end && !nf) ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag && threadIdx.x < 32) {   // y = R^{-1} g, k = j + 1
    const int lane = threadIdx.x, k = j + 1;
    auto Rent = [&](int i, int c) -> double { return P.H[(size_t)c * (mm + 1) + i]; };
    if (k <= 32) {
      // by columns with y_i in lane i: the diagonal's reciprocals in parallel,
      // then per column one broadcast and one FMA
      double yv = 0.0, rv = 0.0;
      if (lane < k) {
        yv = P.g[lane];
        rv = 1.0 / Rent(lane, lane);
      }
      double Rc = lane < k - 1 ? Rent(lane, k - 1) : 0.0;
      for (int l = k - 1; l >= 0; --l) {
        const double Rn = (l >= 1 && lane < l - 1) ? Rent(lane, l - 1) : 0.0;
        if (lane == l) yv *= rv;
        const double yl = __shfl_sync(0xffffffffu, yv, l);
        if (lane < l) yv = fma(-Rc, yl, yv);
        Rc = Rn;
      }
      if (lane < k) P.y[lane] = yv;
    } else {
      for (int i = k - 1; i >= 0; --i) {
        double s = 0.0;
        for (int l = i + 1 + lane; l < k; l += 32) s += Rent(i, l) * P.y[l];
        s = warp_sum(s);
        if (lane == 0) P.y[i] = (P.g[i] - s) / Rent(i, i);
        __syncwarp();
      }
    }
  }
  __syncthreads();
}

// omega += ||r|| P (V y + U (c_0 - B y)) (rows); the leader counts the cycle.
// When the cycle's space fits, it joins the recycled one (as in the
// single-problem solver): C gains V_{k+1} G^T's first k columns (G the cycle's
// Givens rotations) and U gains (V_k - U B) R^-1, so that T U = C holds.
__device__ void bt_update(const BtArgs& a, const BtProb& P, const BtUnit& U, int p, int cycle,
                          double* sh) {
  BtStat* S = a.st + p;
  const int k = __ldcg(&S->iters);
  const int q = __ldcg(&S->qc[cycle & 1]);
  const bool act = __ldcg(&S->active) != 0;
  const int ext = (act && k >= 1 && k <= BT_RK && q + k <= BT_RQ) ? 1 : 0;
  const bool applied = act && !(k <= 0 && q == 0);   // else x (and dlast) stay as they are
  if (U.r0 == 0 && threadIdx.x == 0) {
    S->qc[(cycle + 1) & 1] = q + (ext ? k : 0);
    S->have_d = applied ? 1 : 0;
  }
  if (!applied) return;
  const int mm = a.m;
  double* y = sh;        // k
  double* tq = sh + k;   // c_0 - B y, q
  __shared__ double Ri[BT_RK * BT_RK];   // R^-1 (row i, column c)
  __shared__ double Mq[BT_RQ * BT_RK];   // -B R^-1
  __shared__ float RiF[BT_RK * BT_RK], MqF[BT_RQ * BT_RK];   // their single-precision copies
  __shared__ double s_dm[BIE_MAXB];      // 3/2 of the correction's mean over each obstacle
  // single-precision copies of y, c_0 - B y and the rotations for the row loops
  __shared__ float yf[BT_MAXM], tqf[BT_RQ], csf[BT_RK], snf[BT_RK];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    y[i] = __ldcg(P.y + i);
    yf[i] = (float)y[i];
    if (i < BT_RK) {
      csf[i] = (float)__ldcg(P.cs + i);
      snf[i] = (float)__ldcg(P.sn + i);
    }
  }
  __syncthreads();
  auto Bent = [&](int l, int i) -> double { return __ldcg(P.Bm + (size_t)i * BT_RQ + l); };
  auto Rent = [&](int i, int c) -> double { return __ldcg(P.H + (size_t)c * (mm + 1) + i); };
  if ((int)threadIdx.x < q) {
    const int l = threadIdx.x;
    double t = __ldcg(P.c0 + l);
    for (int i = 0; i < k; ++i) t -= Bent(l, i) * y[i];
    tq[l] = t;
    tqf[l] = (float)t;
  }
  if (ext && (threadIdx.x >> 5) == 1) {   // warp 1 (beside c_0 - B y on warp 0): R^-1 by columns
    const int c = threadIdx.x & 31;
    __shared__ double s_rinv[BT_RK];
    if (c < k) s_rinv[c] = 1.0 / Rent(c, c);   // the diagonal's reciprocals in parallel
    __syncwarp();
    if (c < k) {
      for (int i = 0; i < k; ++i) Ri[i * BT_RK + c] = 0.0;
      for (int i = c; i >= 0; --i) {
        double t = i == c ? 1.0 : 0.0;
        for (int l = i + 1; l <= c; ++l) t -= Rent(i, l) * Ri[l * BT_RK + c];
        Ri[i * BT_RK + c] = t * s_rinv[i];
      }
      for (int i = 0; i < k; ++i) RiF[i * BT_RK + c] = (float)Ri[i * BT_RK + c];
    }
  }
  __syncthreads();
  if (ext)
    for (int e = threadIdx.x; e < q * k; e += blockDim.x) {
      const int l = e / k, c = e - l * k;
      double t = 0.0;
      for (int i = 0; i <= c; ++i) t -= Bent(l, i) * Ri[i * BT_RK + c];
      Mq[l * BT_RK + c] = t;
      MqF[l * BT_RK + c] = (float)t;
    }
  if ((int)threadIdx.x < P.nobs) {
    double t = 0.0;
    for (int i = 0; i < k; ++i) t += y[i] * __ldcg(P.mu + (size_t)i * BIE_MAXB + threadIdx.x);
    for (int l = 0; l < q; ++l) t += tq[l] * __ldcg(P.umean + (size_t)l * BIE_MAXB + threadIdx.x);
    s_dm[threadIdx.x] = 1.5 * t;
  }
  __syncthreads();
  if (ext && U.r0 == 0)   // means of the new U columns over the obstacles
    for (int e = threadIdx.x; e < P.nobs * k; e += blockDim.x) {
      const int o = e / k, c = e - o * k;
      double t = 0.0;
      for (int i = 0; i <= c; ++i) t += __ldcg(P.mu + (size_t)i * BIE_MAXB + o) * Ri[i * BT_RK + c];
      for (int l = 0; l < q; ++l) t += __ldcg(P.umean + (size_t)l * BIE_MAXB + o) * Mq[l * BT_RK + c];
      P.umean[(size_t)(q + c) * BIE_MAXB + o] = t;
    }
  const double scale = __ldcg(&S->rnorm);
  const int m = U.r0 + (int)threadIdx.x;
  const long long ld = P.ld;
  if (m < U.r1) {
    // FP32 runs of eight terms, the runs summed in FP64 (the correction needs the
    // inner tolerance's accuracy; x itself accumulates in FP64)
    double acc = 0.0;
    for (int i0 = 0; i0 < k; i0 += 8) {
      float run = 0.f;
      for (int i = i0; i < min(i0 + 8, k); ++i) run = fmaf(yf[i], __ldcg(P.V + (size_t)i * ld + m), run);
      acc += (double)run;
    }
    for (int l0 = 0; l0 < q; l0 += 8) {
      float run = 0.f;
      for (int l = l0; l < min(l0 + 8, q); ++l) run = fmaf(tqf[l], __ldcg(P.Ur + (size_t)l * ld + m), run);
      acc += (double)run;
    }
    if (P.nobs > 0 && m >= P.obs_off[0]) {
      int o = 0;
      while (o + 1 < P.nobs && m >= P.obs_off[o + 1]) ++o;
      acc -= s_dm[o];
    }
    P.x[m] = __ldcg(P.x + m) + scale * acc;
    P.dlast[m] = scale * acc;
    if (ext) {   // in single precision, the recycled pair's own precision
      float cur = __ldcg(P.V + m);
      for (int i = 0; i < k; ++i) {
        const float ci = csf[i], si = snf[i];
        // v_k is not formed after a breakdown; its rotation then has s = 0
        const float nxt = (i + 1 < k || si != 0.f) ? __ldcg(P.V + (size_t)(i + 1) * ld + m) : 0.f;
        P.Cr[(size_t)(q + i) * ld + m] = ci * cur + si * nxt;
        cur = -si * cur + ci * nxt;
      }
      float tu[BT_RK];
#pragma unroll
      for (int c = 0; c < BT_RK; ++c) tu[c] = 0.f;
      for (int i = 0; i < k; ++i) {
        const float vi = __ldcg(P.V + (size_t)i * ld + m);
#pragma unroll
        for (int c = 0; c < BT_RK; ++c)
          if (c >= i && c < k) tu[c] += RiF[i * BT_RK + c] * vi;
      }
      for (int l = 0; l < q; ++l) {
        const float ul = __ldcg(P.Ur + (size_t)l * ld + m);
#pragma unroll
        for (int c = 0; c < BT_RK; ++c)
          if (c < k) tu[c] += MqF[l * BT_RK + c] * ul;
      }
#pragma unroll
      for (int c = 0; c < BT_RK; ++c)
        if (c < k) P.Ur[(size_t)(q + c) * ld + m] = tu[c];
    }
  }
  if (U.r0 == 0 && threadIdx.x == 0) {
    S->total_iters += k;
    S->cycles += 1;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <class TA>
__global__ void __launch_bounds__(BT_THREADS, 1) k_batch_gmres(BtArgs a, int maxld) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* xs = reinterpret_cast<float*>(smraw);
  float* xl = xs + maxld;
  double* sh = reinterpret_cast<double*>(xl + maxld);   // 2 (BT_MAXM + 3) doubles
  __shared__ double red[32][65];
  __shared__ double red1[32];
  __shared__ BtUnit s_unit;
  __shared__ int s_state, s_flag, s_any;
  unsigned* ctr = a.bar + 2;
  int t = 0;   // phase index
  auto begin_phase = [&]() {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr[(t + 1) % 3] = 0u;
  };
  auto end_phase = [&]() -> bool {
    ++t;
    return bt_barrier(a.bar, a.err, a.spin_limit);
  };
  auto any_of = [&](int which) -> bool {   // 0: active, 1: inner
    if (threadIdx.x == 0) {
      int any = 0;
      for (int p = 0; p < a.P && !any; ++p)
        any = which == 0 ? __ldcg(&a.st[p].active) : __ldcg(&a.st[p].inner);
      s_any = any;
    }
    __syncthreads();
    const bool r = s_any != 0;
    __syncthreads();
    return r;
  };
  for (int cycle = 0;; ++cycle) {
    begin_phase();
    for (;;) {   // RESID
      const int k = bt_take(ctr + (t % 3), a.gunits, a.ngu, a.st, 1, &s_unit, &s_state);
      if (k == 0) break;
      if (k == 1) continue;
      const BtUnit U = s_unit;
      const BtProb& P = a.prob[U.p];
      bt_resid<TA>(a, P, U, cycle, bt_resid_mode(a, a.st + U.p, cycle, P.ld), xs, xl, red1);
    }
    if (!end_phase()) return;
    begin_phase();
    for (;;) {   // START
      const int k = bt_take(ctr + (t % 3), a.vunits, a.nvu, a.st, 1, &s_unit, &s_state);
      if (k == 0) break;
      if (k == 1) continue;
      const BtUnit U = s_unit;
      bt_start(a, a.prob[U.p], U, U.p, cycle, sh);
    }
    if (!end_phase()) return;
    if (!any_of(0)) break;
    for (int j = 0; j < a.m; ++j) {
      begin_phase();
      for (;;) {   // GEMV
        const int k = bt_take(ctr + (t % 3), a.gunits, a.ngu, a.st, 2, &s_unit, &s_state);
        if (k == 0) break;
        if (k == 1) continue;
        const BtUnit U = s_unit;
        bt_gemv<TA>(a, a.prob[U.p], U, __ldcg(&a.st[U.p].qc[cycle & 1]), j, xs, red, red1);
      }
      if (!end_phase()) return;
      begin_phase();
      for (;;) {   // CGS2
        const int k = bt_take(ctr + (t % 3), a.vunits, a.nvu, a.st, 2, &s_unit, &s_state);
        if (k == 0) break;
        if (k == 1) continue;
        const BtUnit U = s_unit;
        bt_cgs2(a, a.prob[U.p], U, __ldcg(&a.st[U.p].qc[cycle & 1]), j, sh);
      }
      if (!end_phase()) return;
      begin_phase();
      for (;;) {   // CGS3
        // the leader may end the cycle while other units of the problem are
        // in this phase; they then skip v_{j+1}, which the update does not use
        const int k = bt_take(ctr + (t % 3), a.vunits, a.nvu, a.st, 2, &s_unit, &s_state);
        if (k == 0) break;
        if (k == 1) continue;
        const BtUnit U = s_unit;
        bt_cgs3(a, a.prob[U.p], U, U.p, __ldcg(&a.st[U.p].qc[cycle & 1]), j, sh, &s_flag);
      }
      if (!end_phase()) return;
      if (!any_of(1)) break;
    }
    begin_phase();
    for (;;) {   // UPDATE
      const int k = bt_take(ctr + (t % 3), a.vunits, a.nvu, a.st, 1, &s_unit, &s_state);
      if (k == 0) break;
      if (k == 1) continue;
      const BtUnit U = s_unit;
      bt_update(a, a.prob[U.p], U, U.p, cycle, sh);
    }
    if (!end_phase()) return;
  }
}

__global__ void k_batch_init(int P, BtStat* st, unsigned* bar, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) {
    BtStat s;
    memset(&s, 0, sizeof(s));
    s.active = 1;
    st[p] = s;
  }
  if (p < 5) bar[p] = 0u;
  if (p == 0) *err = 0;
}

// one CTA of every cooperative grid but `stall` passes the barriers; the
// stalled CTA returns at once, so the others' waits run out (test of the
// bounded wait; no CTA waits without a limit)
__global__ void __launch_bounds__(256) k_barrier_test(unsigned* bar, int* err, unsigned spin_limit,
                                                      int stall, int rounds, int* passed) {
  if ((int)blockIdx.x == stall) return;
  for (int r = 0; r < rounds; ++r) {
    if (!bt_barrier(bar, err, spin_limit)) return;
    if (threadIdx.x == 0) atomicAdd(passed, 1);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct bie_batch {
  int device = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t aux[BT_STREAMS] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[BT_STREAMS] = {};
  std::string err;
  std::vector<bie_ctx*> ctx;
  std::vector<int> set;
  // device tables and scratch
  std::vector<std::pair<std::string, DevBuf>> bufs;
  BtStat* st_host = nullptr;   // pinned
  int* err_host = nullptr;     // pinned
  int nsm = 0;
  // captured graph and what it was captured for
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;
  // autotuned GEMV unit size for the problem sizes in `tuned_for`
  long long unit_bytes = 0;
  std::vector<long long> tuned_for;
  float tune_ms[8] = {};
  double last_rbytes = 0.0;   // residual products' matrix bytes of the last run
};

static const long long kUnitCandidates[5] = {256 << 10, 512 << 10, 1 << 20, 2 << 20, 4 << 20};

static bie_status bt_fail(bie_batch* b, bie_status s, const std::string& m) {
  b->err = m;
  return s;
}
static bie_status bt_cuda(bie_batch* b, cudaError_t e, const char* where) {
  b->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  return BIE_ERR_CUDA;
}
#define BT_TRY(b, call)                                       \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return bt_cuda((b), _e, #call);    \
  } while (0)

static void* bt_buf(bie_batch* b, const char* name, size_t bytes, bool* oom) {
  *oom = false;
  if (bytes == 0) bytes = 16;
  for (auto& kv : b->bufs) {
    if (kv.first == name) {
      if (kv.second.bytes >= bytes) return kv.second.p;
      cudaFree(kv.second.p);
      kv.second.p = nullptr;
      kv.second.bytes = 0;
      if (cudaMalloc(&kv.second.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *oom = true;
        return nullptr;
      }
      kv.second.bytes = bytes;
      return kv.second.p;
    }
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *oom = true;
    return nullptr;
  }
  b->bufs.push_back({std::string(name), DevBuf{p, bytes}});
  return p;
}

static void bt_drop_graph(bie_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->key.clear();
}

struct BtPlan {
  std::vector<BtProb> probs;
  std::vector<BtUnit> gunits, vunits;
  int maxld = 0;
};

// per-problem pointers, units and the kernel arguments; allocates on first use
static bie_status bt_plan(bie_batch* b, int prec, int m, long long gbytes, const double* phit_all,
                          double* omega_all, double* U_all, BtPlan& pl, BtArgs& A,
                          std::vector<const void*>& key) {
  const int P = (int)b->ctx.size();
  pl.probs.assign(P, BtProb{});
  std::vector<int> order(P);
  for (int p = 0; p < P; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->ctx[x]->N > b->ctx[y]->N; });
  long long offN = 0, offM = 0;
  std::vector<long long> oN(P), oM(P);
  for (int p = 0; p < P; ++p) {
    oN[p] = offN;
    oM[p] = offM;
    offN += b->ctx[p]->N;
    offM += b->ctx[p]->M[0];
  }
  const size_t ebytes = (prec == BIE_FP32_IR) ? 4 : 2;
  for (int p : order) {
    bie_ctx* c = b->ctx[p];
    BtProb& Q = pl.probs[p];
    Q.N = c->N;
    Q.M0 = c->M[0];
    Q.ld = c->ld;
    pl.maxld = std::max(pl.maxld, (int)c->ld);
    int rows = (int)(gbytes / (long long)((size_t)c->ld * ebytes));
    rows = std::max(32, std::min(1024, rows / 32 * 32));
    Q.g0 = (int)pl.gunits.size();
    for (int r0 = 0; r0 < c->N; r0 += rows)
      pl.gunits.push_back(BtUnit{p, r0, std::min(c->N, r0 + rows), (int)pl.gunits.size()});
    Q.ng = (int)pl.gunits.size() - Q.g0;
    Q.v0 = (int)pl.vunits.size();
    for (int r0 = 0; r0 < c->N; r0 += BT_VROWS)
      pl.vunits.push_back(BtUnit{p, r0, std::min(c->N, r0 + BT_VROWS), (int)pl.vunits.size()});
    Q.nv = (int)pl.vunits.size() - Q.v0;
    const size_t NN = (size_t)c->N * (size_t)c->ld;
    bool oom = false, o = false;
    auto get = [&](const char* name, size_t bytes) {
      void* q = ctx_buf(c, name, bytes, &o);
      oom = oom || o;
      return q;
    };
    Q.Ahi = (const float*)get("A_hi", sizeof(float) * NN);
    Q.Alo = (const float*)get("A_lo", sizeof(float) * NN);
    Q.A16 = (prec != BIE_FP32_IR) ? get("A_16", 2 * NN) : nullptr;
    Q.wgt = (const float*)get("wgt", sizeof(float) * c->ld);
    Q.wgt64 = (const double*)get("wgt64", sizeof(double) * c->ld);
    Q.sgn = (const float*)get("sgn", sizeof(float) * c->ld);
    Q.blk = (const int*)get("blk", sizeof(int) * c->ld);
    Q.b = (const double*)get("bt_b", sizeof(double) * c->ld);
    Q.x = omega_all + oN[p];
    Q.r = (double*)get("bt_r", sizeof(double) * c->ld);
    Q.dlast = (double*)get("bt_dlast", sizeof(double) * c->ld);
    Q.V = (float*)get("bt_V", sizeof(float) * (size_t)(m + 1) * c->ld);
    Q.w = (float*)get("bt_w", sizeof(float) * c->ld);
    Q.H = (double*)get("bt_H", sizeof(double) * (size_t)(m + 1) * m);
    Q.cs = (double*)get("bt_cs", sizeof(double) * m);
    Q.sn = (double*)get("bt_sn", sizeof(double) * m);
    Q.g = (double*)get("bt_g", sizeof(double) * (m + 1));
    Q.y = (double*)get("bt_y", sizeof(double) * (m + 1));
    Q.mu = (double*)get("bt_mu", sizeof(double) * (size_t)(m + 1) * BIE_MAXB);
    Q.Cr = (float*)get("bt_C", sizeof(float) * (size_t)BT_RQ * c->ld);
    Q.Ur = (float*)get("bt_U", sizeof(float) * (size_t)BT_RQ * c->ld);
    Q.Bm = (double*)get("bt_B", sizeof(double) * (size_t)m * BT_RQ);
    Q.c0 = (double*)get("bt_c0", sizeof(double) * BT_RQ);
    Q.umean = (double*)get("bt_umean", sizeof(double) * (size_t)BT_RQ * BIE_MAXB);
    Q.nobs = c->nb > 2 ? c->nb - 2 : 0;
    for (int k = 0; k < Q.nobs; ++k) Q.obs_off[k] = c->off[2 + k];
    Q.obs_off[Q.nobs] = c->N;
    if (oom) return bt_fail(b, BIE_ERR_OOM, "bie_batch_run: problem buffers");
    key.push_back(c);
    // values baked into the captured kernels' arguments
    auto push_d = [&](double v) {
      const void* q;
      memcpy(&q, &v, sizeof(q));
      key.push_back(q);
    };
    key.push_back((const void*)(intptr_t)c->nb);
    for (int k = 0; k < c->nb; ++k) key.push_back((const void*)(intptr_t)c->M[k]);
    push_d(c->V1);
    for (int k = 0; k + 2 < c->nb; ++k) {
      push_d(c->a[k]);
      push_d(c->zc[k].x);
      push_d(c->zc[k].y);
    }
    for (const void* q : {(const void*)Q.Ahi, (const void*)Q.Alo, Q.A16, (const void*)Q.wgt,
                          (const void*)Q.b, (const void*)Q.r, (const void*)Q.V, (const void*)Q.w,
                          (const void*)Q.H, (const void*)Q.y, (const void*)Q.dlast})
      key.push_back(q);
  }
  // velocity and rhs pointers per problem enter the key through the packed arrays
  key.push_back(phit_all);
  key.push_back(omega_all);
  key.push_back(U_all);
  const int ngu = (int)pl.gunits.size(), nvu = (int)pl.vunits.size();
  bool oom = false, o = false;
  auto get = [&](const char* name, size_t bytes) {
    void* q = bt_buf(b, name, bytes, &o);
    oom = oom || o;
    return q;
  };
  memset(&A, 0, sizeof(A));
  A.P = P;
  A.m = m;
  A.ngu = ngu;
  A.nvu = nvu;
  A.prob = (const BtProb*)get("probs", sizeof(BtProb) * P);
  A.gunits = (const BtUnit*)get("gunits", sizeof(BtUnit) * ngu);
  A.vunits = (const BtUnit*)get("vunits", sizeof(BtUnit) * nvu);
  A.st = (BtStat*)get("stat", sizeof(BtStat) * P);
  A.part1 = (double*)get("part1", sizeof(double) * (size_t)(m + 1 + BT_RQ) * ngu);
  A.part2 = (double*)get("part2", sizeof(double) * (size_t)(m + 2 + BT_RQ) * nvu);
  A.partn = (double*)get("partn", sizeof(double) * ngu);
  A.partc = (double*)get("partc", sizeof(double) * (size_t)BT_RQ * ngu);
  A.bar = (unsigned*)get("bar", sizeof(unsigned) * 8);
  A.err = (int*)get("err", sizeof(int) * 4);
  if (oom) return bt_fail(b, BIE_ERR_OOM, "bie_batch_run: batch tables");
  for (const void* q : {(const void*)A.prob, (const void*)A.gunits, (const void*)A.vunits,
                        (const void*)A.st, (const void*)A.part1, (const void*)A.part2,
                        (const void*)A.partn, (const void*)A.partc, (const void*)A.bar})
    key.push_back(q);
  key.push_back((const void*)(intptr_t)prec);
  key.push_back((const void*)(intptr_t)m);
  key.push_back((const void*)(intptr_t)gbytes);
  return BIE_OK;
}

static bie_status bt_upload(bie_batch* b, const BtPlan& pl, const BtArgs& A) {
  BT_TRY(b, cudaMemcpyAsync((void*)A.prob, pl.probs.data(), sizeof(BtProb) * pl.probs.size(),
                            cudaMemcpyHostToDevice, b->stream));
  BT_TRY(b, cudaMemcpyAsync((void*)A.gunits, pl.gunits.data(), sizeof(BtUnit) * pl.gunits.size(),
                            cudaMemcpyHostToDevice, b->stream));
  BT_TRY(b, cudaMemcpyAsync((void*)A.vunits, pl.vunits.data(), sizeof(BtUnit) * pl.vunits.size(),
                            cudaMemcpyHostToDevice, b->stream));
  return BIE_OK;
}

// the whole batch on b->stream: fork, per-problem setup, solve, velocity, join
static bie_status bt_enqueue(bie_batch* b, int prec, const bie_solve_opts& o, const BtPlan& pl,
                             const BtArgs& A0, const double* phit_all, double* omega_all,
                             double* U_all, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr) {
  const int P = (int)b->ctx.size();
  BT_TRY(b, cudaEventRecord(b->ev_fork, b->stream));
  for (int k = 0; k < BT_STREAMS; ++k) BT_TRY(b, cudaStreamWaitEvent(b->aux[k], b->ev_fork, 0));
  long long offM = 0;
  for (int p = 0; p < P; ++p) {
    bie_ctx* c = b->ctx[p];
    c->stream = b->aux[p % BT_STREAMS];
    bie_status s = geometry_prep(c);
    // always in full: this sequence is captured once and replayed for new
    // geometries of the same sizes
    c->asm_sig = -1;
    if (s == BIE_OK) s = asm_run(c, prec, 0);
    double* bp = const_cast<double*>(pl.probs[p].b);
    if (s == BIE_OK) s = rhs_run(c, phit_all + offM, bp);
    if (s != BIE_OK) return bt_fail(b, s, "problem " + std::to_string(p) + ": " + c->err);
    c->precision = prec;
    c->assembled = true;
    c->transposed = false;
    offM += c->M[0];
  }
  for (int k = 0; k < BT_STREAMS; ++k) {
    BT_TRY(b, cudaEventRecord(b->ev_join[k], b->aux[k]));
    BT_TRY(b, cudaStreamWaitEvent(b->stream, b->ev_join[k], 0));
  }
  long long offN = 0;
  for (int p = 0; p < P; ++p) {   // omega = 0 (zero initial guess)
    BT_TRY(b, cudaMemsetAsync(omega_all + offN, 0, sizeof(double) * b->ctx[p]->N, b->stream));
    offN += b->ctx[p]->N;
  }
  k_batch_init<<<(P + 255) / 256 + 1, 256, 0, b->stream>>>(P, A0.st, A0.bar, A0.err);
  BT_TRY(b, cudaGetLastError());
  BtArgs A = A0;
  A.rowflip = o.row_flip ? 1 : 0;
  A.max_cycles = o.max_cycles;
  A.rtol = o.rtol;
  A.eps16 = prec == BIE_FP16_IR ? 0x1p-11 : (prec == BIE_BF16_IR ? 0x1p-8 : 0.0);
  double itol = o.inner_tol;
  if (itol <= 0.0) itol = prec == BIE_FP32_IR ? 1e-4 : 5e-4;   // as bie_solve (recycled space)
  A.inner_tol = itol;
  A.spin_limit = 1u << 22;
  int maxld = pl.maxld;
  const size_t smem = sizeof(float) * 2 * (size_t)maxld + sizeof(double) * 2 * (BT_MAXM + 3);
  void* args[] = {&A, &maxld};
  const void* fn = prec == BIE_FP32_IR ? (const void*)k_batch_gmres<float>
                   : prec == BIE_FP16_IR ? (const void*)k_batch_gmres<__half>
                                         : (const void*)k_batch_gmres<__nv_bfloat16>;
  BT_TRY(b, raise_smem_limit(fn, smem));
  int per_sm = 0;
  BT_TRY(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BT_THREADS, smem));
  if (per_sm < 1) return bt_fail(b, BIE_ERR_CUDA, "bie_batch_run: solver kernel does not fit an SM");
  if (ev0) BT_TRY(b, cudaEventRecord(ev0, b->stream));
  BT_TRY(b, cudaLaunchCooperativeKernel(fn, dim3(b->nsm), dim3(BT_THREADS), args, smem, b->stream));
  if (ev1) BT_TRY(b, cudaEventRecord(ev1, b->stream));
  // normal velocity of every problem
  BT_TRY(b, cudaEventRecord(b->ev_fork, b->stream));
  for (int k = 0; k < BT_STREAMS; ++k) BT_TRY(b, cudaStreamWaitEvent(b->aux[k], b->ev_fork, 0));
  offN = 0;
  long long offU = 0;
  for (int p = 0; p < P; ++p) {
    bie_ctx* c = b->ctx[p];
    bie_status s = velocity_run(c, omega_all + offN, U_all + offU, nullptr);
    if (s != BIE_OK) return bt_fail(b, s, "problem " + std::to_string(p) + ": " + c->err);
    offN += c->N;
    offU += c->M[0];
  }
  for (int k = 0; k < BT_STREAMS; ++k) {
    BT_TRY(b, cudaEventRecord(b->ev_join[k], b->aux[k]));
    BT_TRY(b, cudaStreamWaitEvent(b->stream, b->ev_join[k], 0));
  }
  BT_TRY(b, cudaMemcpyAsync(b->st_host, A0.st, sizeof(BtStat) * P, cudaMemcpyDeviceToHost, b->stream));
  BT_TRY(b, cudaMemcpyAsync(b->err_host, A0.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  return BIE_OK;
}

extern "C" {

bie_status bie_batch_create(bie_batch** out, int device, void* cuda_stream) {
  if (!out) return BIE_ERR_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  bie_batch* b = new bie_batch();
  b->device = device;
  b->user_stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  for (int k = 0; k < BT_STREAMS && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int k = 0; k < BT_STREAMS && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->err_host, sizeof(int) * 4, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    bie_batch_destroy(b);
    return BIE_ERR_CUDA;
  }
  *out = b;
  return BIE_OK;
}

void bie_batch_destroy(bie_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  bt_drop_graph(b);
  for (bie_ctx* c : b->ctx) {
    if (c) {
      c->stream = nullptr;   // the batch owns the streams
      bie_destroy(c);
    }
  }
  for (auto& kv : b->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  if (b->st_host) cudaFreeHost(b->st_host);
  if (b->err_host) cudaFreeHost(b->err_host);
  for (int k = 0; k < BT_STREAMS; ++k) {
    if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* bie_batch_last_error(const bie_batch* b) {
  if (!b) return "null batch";
  return b->err.c_str();
}

bie_status bie_batch_set_problem(bie_batch* b, int p, int nb, const int* M_host,
                                 const double* zeta_dev, const double* dzeta_dev,
                                 const double* d2zeta_dev, const double* zc_host, double V1,
                                 const double* a_host) {
  if (!b) return BIE_ERR_ARG;
  b->err.clear();
  if (p < 0 || p >= 4096) return bt_fail(b, BIE_ERR_ARG, "bie_batch_set_problem: bad index");
  cudaSetDevice(b->device);
  if ((int)b->ctx.size() <= p) {
    b->ctx.resize(p + 1, nullptr);
    b->set.resize(p + 1, 0);
    bt_drop_graph(b);
  }
  if (!b->ctx[p]) {
    bie_ctx* c = nullptr;
    bie_status s = bie_create(&c, b->device, b->aux[p % BT_STREAMS]);
    if (s != BIE_OK) return bt_fail(b, s, "bie_batch_set_problem: context");
    b->ctx[p] = c;
  }
  bie_ctx* c = b->ctx[p];
  c->stream = b->aux[p % BT_STREAMS];
  b->set[p] = 0;
  // the inputs may have been written on the caller's stream
  if (b->user_stream) BT_TRY(b, cudaStreamSynchronize(b->user_stream));
  const int oldN = c->N;
  bie_status s = bie_set_geometry(c, nb, M_host, zeta_dev, dzeta_dev, d2zeta_dev, zc_host);
  if (s == BIE_OK) s = bie_set_flow(c, V1, a_host);
  if (s != BIE_OK) return bt_fail(b, s, "problem " + std::to_string(p) + ": " + c->err);
  if (c->N > BT_MAXLD) return bt_fail(b, BIE_ERR_ARG, "bie_batch_set_problem: N > 16384");
  if (c->N != oldN) bt_drop_graph(b);
  b->set[p] = 1;
  return BIE_OK;
}

bie_status bie_batch_run(bie_batch* b, int nprob, const double* phit_all, double* omega_all,
                         double* U_all, int precision, const bie_solve_opts* opts,
                         bie_solve_info* infos) {
  BIE_NVTX("bie_batch_run");
  if (!b) return BIE_ERR_ARG;
  b->err.clear();
  if (nprob < 1 || nprob != (int)b->ctx.size())
    return bt_fail(b, BIE_ERR_ARG, "bie_batch_run: nprob must equal the number of problems set");
  for (int p = 0; p < nprob; ++p)
    if (!b->set[p]) return bt_fail(b, BIE_ERR_STATE, "bie_batch_run: problem " + std::to_string(p) + " not set");
  if (!phit_all || !omega_all || !U_all) return bt_fail(b, BIE_ERR_ARG, "bie_batch_run: null pointer");
  if (precision != BIE_FP32_IR && precision != BIE_FP16_IR && precision != BIE_BF16_IR)
    return bt_fail(b, BIE_ERR_ARG, "bie_batch_run: precision must be a refined scheme");
  bie_solve_opts o;
  bie_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > BT_MAXM || o.max_cycles < 1)
    return bt_fail(b, BIE_ERR_ARG, "bie_batch_run: bad options (restart <= 63)");
  cudaSetDevice(b->device);
  if (!b->st_host) BT_TRY(b, cudaHostAlloc((void**)&b->st_host, sizeof(BtStat) * 4096, cudaHostAllocDefault));
  // autotune the GEMV unit size once per set of problem sizes: time the
  // solver kernel for every candidate on these problems, keep the fastest
  std::vector<long long> sizes;
  for (bie_ctx* c : b->ctx) sizes.push_back(c->ld);
  sizes.push_back(precision);
  sizes.push_back(o.restart);
  bie_status s = BIE_OK;
  if (b->unit_bytes == 0 || sizes != b->tuned_for) {
    bt_drop_graph(b);
    if (b->user_stream) BT_TRY(b, cudaStreamSynchronize(b->user_stream));
    cudaEvent_t e0, e1;
    BT_TRY(b, cudaEventCreate(&e0));
    BT_TRY(b, cudaEventCreate(&e1));
    float best = 3.0e38f;
    long long best_bytes = kUnitCandidates[2];
    for (int ci = 0; ci < 5; ++ci) {
      BtPlan tp;
      BtArgs ta;
      std::vector<const void*> tk;
      s = bt_plan(b, precision, o.restart, kUnitCandidates[ci], phit_all, omega_all, U_all, tp, ta, tk);
      if (s == BIE_OK) s = bt_upload(b, tp, ta);
      if (s == BIE_OK) s = bt_enqueue(b, precision, o, tp, ta, phit_all, omega_all, U_all, e0, e1);
      cudaError_t ce = cudaStreamSynchronize(b->stream);
      if (s == BIE_OK && ce != cudaSuccess) s = bt_cuda(b, ce, "autotune");
      if (s != BIE_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      b->tune_ms[ci] = ms;
      if (*b->err_host) {
        s = bt_fail(b, BIE_ERR_TIMEOUT, "bie_batch_run: a grid barrier timed out");
        break;
      }
      if (ms < best) {
        best = ms;
        best_bytes = kUnitCandidates[ci];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != BIE_OK) return s;
    b->unit_bytes = best_bytes;
    b->tuned_for = sizes;
  }
  BtPlan pl;
  BtArgs A;
  std::vector<const void*> key;
  s = bt_plan(b, precision, o.restart, b->unit_bytes, phit_all, omega_all, U_all, pl, A, key);
  if (s != BIE_OK) return s;
  // options enter the graph by value
  const double kd[3] = {o.rtol, o.inner_tol, (double)o.max_cycles};
  for (double v : kd) {
    const void* q;
    memcpy(&q, &v, sizeof(q));
    key.push_back(q);
  }
  key.push_back((const void*)(intptr_t)o.row_flip);
  if (b->user_stream) {
    BT_TRY(b, cudaEventRecord(b->ev_fork, b->user_stream));
    BT_TRY(b, cudaStreamWaitEvent(b->stream, b->ev_fork, 0));
  }
  if (!b->exec || key != b->key) {
    bt_drop_graph(b);
    // the tables are constant for a given key: uploaded here, outside the graph
    s = bt_upload(b, pl, A);
    if (s != BIE_OK) return s;
    // one direct run allocates every buffer the sequence touches
    s = bt_enqueue(b, precision, o, pl, A, phit_all, omega_all, U_all);
    if (s != BIE_OK) return s;
    BT_TRY(b, cudaStreamSynchronize(b->stream));
    cudaGraph_t graph = nullptr;
    BT_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
    s = bt_enqueue(b, precision, o, pl, A, phit_all, omega_all, U_all);
    cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    if (s != BIE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (ce != cudaSuccess) return bt_cuda(b, ce, "cudaStreamEndCapture");
    ce = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      b->exec = nullptr;
      return bt_cuda(b, ce, "cudaGraphInstantiate");
    }
    b->key = key;
  }
  BT_TRY(b, cudaGraphLaunch(b->exec, b->stream));
  BT_TRY(b, cudaStreamSynchronize(b->stream));
  if (b->user_stream) {
    BT_TRY(b, cudaEventRecord(b->ev_fork, b->stream));
    BT_TRY(b, cudaStreamWaitEvent(b->user_stream, b->ev_fork, 0));
  }
  if (*b->err_host) return bt_fail(b, BIE_ERR_TIMEOUT, "bie_batch_run: a grid barrier timed out");
  bie_status worst = BIE_OK;
  b->last_rbytes = 0.0;
  for (int p = 0; p < nprob; ++p) {
    const BtStat& S = b->st_host[p];
    b->last_rbytes += S.rbytes;
    if (infos) {
      infos[p].iters = S.total_iters;
      infos[p].cycles = S.cycles;
      infos[p].converged = S.converged;
      infos[p].rel_resid = S.bnorm > 0 ? S.rnorm / S.bnorm : S.rnorm;
    }
    if (S.nonfinite) worst = BIE_ERR_NAN;
    else if (!S.converged && worst == BIE_OK) worst = BIE_ERR_NOCONV;
  }
  if (worst == BIE_ERR_NAN) return bt_fail(b, worst, "bie_batch_run: non-finite residual");
  if (worst == BIE_ERR_NOCONV) return bt_fail(b, worst, "bie_batch_run: some problem missed rtol");
  return BIE_OK;
}

bie_status bie_batch_resid_bytes(const bie_batch* b, double* bytes) {
  if (!b || !bytes) return BIE_ERR_ARG;
  *bytes = b->last_rbytes;
  return BIE_OK;
}

bie_status bie_batch_tuning(const bie_batch* b, long long* unit_bytes, float* candidate_ms) {
  if (!b || !unit_bytes) return BIE_ERR_ARG;
  *unit_bytes = b->unit_bytes;
  if (candidate_ms)
    for (int i = 0; i < 5; ++i) candidate_ms[i] = b->tune_ms[i];
  return BIE_OK;
}

bie_status bie_test_grid_barrier(int device, unsigned spin_limit, int stall, int* passed_out,
                                 int* err_out) {
  if (!passed_out || !err_out) return BIE_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  if (nsm < 2) return BIE_ERR_CUDA;
  unsigned* bar = nullptr;
  int *err = nullptr, *passed = nullptr;
  cudaError_t e = cudaMalloc(&bar, sizeof(unsigned) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&passed, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(bar, 0, sizeof(unsigned) * 8);
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(passed, 0, sizeof(int));
  if (stall >= nsm) stall = nsm - 1;
  int rounds = 3;
  void* args[] = {&bar, &err, &spin_limit, &stall, &rounds, &passed};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)k_barrier_test, dim3(nsm), dim3(256), args, 0, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(passed_out, passed, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(err_out, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  cudaFree(err);
  cudaFree(passed);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  return *err_out ? BIE_ERR_TIMEOUT : BIE_OK;
}

}  // extern "C"
