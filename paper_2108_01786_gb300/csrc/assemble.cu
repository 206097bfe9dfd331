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
#include <type_traits>

#include "common.cuh"
#include "df2.cuh"
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
  // per tile of ATILE nodes (k_tile_prep): boundary (-1 when the tile is
  // partial or spans two), node box, and the row data of the fast path packed
  // by row pairs (rp, rp + 16)
  const int* tile_blk;
  const float4* tile_box;
  const float4* tile_rows;   // [tile][16][5]
  // stored rows [row0, row1) (all N unless the context is row-partitioned):
  // row m of A and of the U-matrix is kept at (m - row0) ld; tile boundaries
  // fall on multiples of ATILE, so a tile is either stored or not
  int row0, row1;
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

// ---------------------------------------------------------------------------
// fast path: off-diagonal tile pairs whose rows lie on one boundary, whose
// columns lie on one boundary, and whose node pairs are all in the far field
// ---------------------------------------------------------------------------
// A tile's nodes sit in a box (centre and half-widths in x and y).  For
// Delta = zeta_l - zeta_m = a + i b, |e^{i Delta} - 1|^2 = (1 - e^{-b})^2 +
// 2 e^{-b} (1 - cos a), so |d| < 0.1 needs |b| < 0.106 and |a mod 2 pi| <
// 0.106: two tiles whose boxes are more than 0.11 apart in x (periodically)
// or in y have no near-field pair, and the separable form serves them all.
#define FAST_GAP 0.11f

// Per tile: the boundary it lies on (-1 if partial or spanning two), the box
// of its nodes (centre and half-width in x, then in y; half-widths rounded up
// against the FP32 rounding of the nodes) and its rows for the fast path,
// packed by row pairs (rp, rp + 16) so that a float4 load gives both lanes:
//   [0] Q.re hi (a, b), Q.re lo (a, b)   [1] Q.im hi, lo   [2] Q third words x, y
//   [3] zeta'.re hi, lo                  [4] zeta'.im hi, lo
// One warp per tile.
__global__ void k_tile_prep(AsmArgs a, int* __restrict__ tblk, float4* __restrict__ tbox,
                            float4* __restrict__ trows) {
  const int t = blockIdx.x, lane = threadIdx.x;
  const int t0 = t * ATILE;
  const int n = min(t0 + lane, a.N - 1);
  const float x0 = (float)a.z64[t0].x;
  const double2 z = a.z64[n];
  const float dx = (float)z.x - x0, y = (float)z.y;
  float xl = dx, xh = dx, yl = y, yh = y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    xl = fminf(xl, __shfl_xor_sync(0xffffffffu, xl, o));
    xh = fmaxf(xh, __shfl_xor_sync(0xffffffffu, xh, o));
    yl = fminf(yl, __shfl_xor_sync(0xffffffffu, yl, o));
    yh = fmaxf(yh, __shfl_xor_sync(0xffffffffu, yh, o));
  }
  const bool full = t0 + ATILE <= a.N;
  if (lane == 0) {
    const int b0 = a.blk[t0];
    tblk[t] = (full && a.blk[t0 + ATILE - 1] == b0) ? b0 : -1;
    tbox[t] = make_float4(x0 + 0.5f * (xl + xh), 0.5f * (xh - xl) + 1e-5f, 0.5f * (yl + yh),
                          0.5f * (yh - yl) + 1e-5f);
  }
  if (lane < 16 && full) {
    const int ma = t0 + lane, mb = ma + 16;
    const float4 qa = a.nQ[ma], qb = a.nQ[mb], ca = a.nPQc[ma], cb = a.nPQc[mb];
    const float4 za = a.nZp[ma], zb = a.nZp[mb];
    float4* r = trows + ((size_t)t * 16 + lane) * 5;
    r[0] = make_float4(qa.x, qb.x, qa.y, qb.y);
    r[1] = make_float4(qa.z, qb.z, qa.w, qb.w);
    r[2] = make_float4(ca.z, cb.z, ca.w, cb.w);
    r[3] = make_float4(za.x, zb.x, za.y, zb.y);
    r[4] = make_float4(za.z, zb.z, za.w, zb.w);
  }
}

// Which tile pairs take the fast path: tiles I < J that each lie inside one
// boundary (full tiles), boxes more than FAST_GAP apart, and the standard
// operator (not the vortex-sheet or App. B variants).
__device__ __forceinline__ bool fast_tile_pair(const AsmArgs& a, int I, int J, int& bI, int& bJ) {
  bI = a.tile_blk[I];
  bJ = a.tile_blk[J];
  if (I == J || bI < 0 || bJ < 0 || a.alt || a.vs) return false;
  const float4 u = a.tile_box[I], v = a.tile_box[J];
  float dcx = v.x - u.x;
  dcx -= 6.2831853f * rintf(dcx * 0.15915494f);
  const float gx = fabsf(dcx) - u.y - v.y;
  const float gy = fabsf(v.z - u.z) - u.w - v.w;
  return fmaxf(gx, gy) > FAST_GAP;
}

// stores of the fast path: base pointers of the tile pair, 32-bit offsets
struct FastOut {
  float *hi, *lo, *vhi, *vlo;
  void* h16;
};
template <int K16>
__device__ __forceinline__ void fast_store(const FastOut& o, int off, float hi, float lo) {
  o.hi[off] = hi;
  o.lo[off] = lo;
  if (K16 == 1) ((__half*)o.h16)[off] = __float2half_rn(hi);
  else if (K16 == 2) ((__nv_bfloat16*)o.h16)[off] = __float2bfloat16_rn(hi);
}

// Two node pairs per thread at once (rows rp and rp + 16 of the row tile,
// packed in the two lanes of the df2 arithmetic), with the entry formulas of
// the general kernel below specialised at compile time:
//   SM, SL   row / column tile on the free surface;
//   SAME     both tiles on the same obstacle (the -E_k term, -1 in storage units).
// G = 1/2 cot((zeta_l - zeta_m)/2) = i/2 + i/d, d = P_l Q_m - 1 (with the
// cross terms of the third words of P and Q), Re G = Im d/|d|^2,
// Im G = 1/2 + Re d/|d|^2; each stored value is one combined
// double-float a b + c d (+ constant) of zeta' and G.
template <int K16, bool SM, bool SL, bool SAME>
__device__ __forceinline__ void asm_fast(const AsmArgs& a, int I, int J, bool fwd, bool tr,
                                         dfl (*sAT)[ATILE + 1], dfl (*sVT)[ATILE + 1]) {
  const int m0 = I * ATILE, l0 = J * ATILE;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool wantV = (SM || SL) && !a.transpose;
  const int l = l0 + tx;
  const float4 pv = a.nP[l], pc4 = a.nPQc[l], zv = a.nZp[l];
  const df2 Pre = {f2(pv.x), f2(pv.y)}, Pim = {f2(pv.z), f2(pv.w)};
  const df2 nPim = d2_neg(Pim);
  const float2 Pcx = f2(pc4.x), Pcy = f2(pc4.y), nPcy = f2(-pc4.y), nPimh = f2(-pv.z);
  const df2 Zlr = {f2(zv.x), f2(zv.y)}, Zli = {f2(zv.z), f2(zv.w)};
  const df2 nZlr = d2_neg(Zlr), nZli = d2_neg(Zli);
  const int ld = (int)a.ld;
  // (m0, l0) block and its transpose (l0, m0) of the stored rows; offsets
  // inside a tile fit 32 bits
  const size_t bml = (size_t)(m0 - a.row0) * a.ld + l0, blm = (size_t)(l0 - a.row0) * a.ld + m0;
  FastOut o = {a.hi + bml, a.lo + bml, a.Vhi ? a.Vhi + bml : nullptr, a.Vlo ? a.Vlo + bml : nullptr,
               K16 == 0 ? nullptr : (void*)((char*)a.h16 + 2 * bml)};
  const float4* rows = a.tile_rows + (size_t)I * 16 * 5;
#pragma unroll 1
  for (int k = 0; k < 2; ++k) {
    const int rp = ty + 8 * k;
    const float4 r0 = rows[rp * 5 + 0], r1 = rows[rp * 5 + 1], r2 = rows[rp * 5 + 2],
                 r3 = rows[rp * 5 + 3], r4 = rows[rp * 5 + 4];
    const df2 Qre = {f2(r0.x, r0.y), f2(r0.z, r0.w)}, Qim = {f2(r1.x, r1.y), f2(r1.z, r1.w)};
    const float2 Qcx = f2(r2.x, r2.y), Qcy = f2(r2.z, r2.w);
    const df2 Zmr = {f2(r3.x, r3.y), f2(r3.z, r3.w)}, Zmi = {f2(r4.x, r4.y), f2(r4.z, r4.w)};
    // third-word cross terms of P Q
    float2 cr = p_mul(Pre.hi, Qcx);
    cr = p_fma(nPimh, Qcy, cr);
    cr = p_fma(Pcx, Qre.hi, cr);
    cr = p_fma(nPcy, Qim.hi, cr);
    float2 ci = p_mul(Pre.hi, Qcy);
    ci = p_fma(Pim.hi, Qcx, ci);
    ci = p_fma(Pcx, Qim.hi, ci);
    ci = p_fma(Pcy, Qre.hi, ci);
    const df2 dr = d2_dot2<true>(Pre, Qre, nPim, Qim, f2(-1.f), cr);   // Re d
    const df2 di = d2_dot2<false>(Pre, Qim, Pim, Qre, f2(0.f), ci);   // Im d
    const df2 n2 = d2_dot2<false>(dr, dr, di, di, f2(0.f), f2(0.f));
    const df2 inv = d2_rcp(n2);
    const df2 Gre = d2_mul(di, inv);
    const df2 Gim = d2_mul_addf(dr, inv, f2(0.5f));
    df2 Aml, Alm, Vml, Vlm;
    if (SM == SL) {   // Im{zeta_l' G}, -Im{zeta_m' G}
      Aml = d2_dot2<SAME>(Zlr, Gim, Zli, Gre, f2(-1.f), f2(0.f));
      Alm = d2_dot2<SAME>(d2_neg(Zmr), Gim, d2_neg(Zmi), Gre, f2(-1.f), f2(0.f));
      if (SM && wantV) {   // T + Re{zeta_m' G}, T' - Re{zeta_l' G}
        int ja = m0 + rp - l;              // (m - l) mod M_0 for lane a; lane b is 16 more
        ja += ja < 0 ? a.M0 : 0;
        int jb = ja + 16;
        jb -= jb >= a.M0 ? a.M0 : 0;
        const float2 ta = a.Ttab[ja], tb = a.Ttab[jb];
        const float2 ua = a.Ttab[a.M0 - ja], ub = a.Ttab[a.M0 - jb];   // (l - m) mod M_0
        Vml = d2_dot2<true>(Zmr, Gre, d2_neg(Zmi), Gim, f2(ta.x, tb.x), f2(ta.y, tb.y));
        Vlm = d2_dot2<true>(nZlr, Gre, Zli, Gim, f2(ua.x, ub.x), f2(ua.y, ub.y));
      }
    } else if (SM) {  // Re{zeta_l' G}, Re{zeta_m' G}; V_ml = -Im{zeta_m' G}
      Aml = d2_dot2<false>(Zlr, Gre, nZli, Gim, f2(0.f), f2(0.f));
      Alm = d2_dot2<false>(Zmr, Gre, d2_neg(Zmi), Gim, f2(0.f), f2(0.f));
      if (wantV) Vml = d2_dot2<false>(d2_neg(Zmr), Gim, d2_neg(Zmi), Gre, f2(0.f), f2(0.f));
    } else {          // -Re{zeta_l' G}, -Re{zeta_m' G}; V_lm = Im{zeta_l' G}
      Aml = d2_dot2<false>(nZlr, Gre, Zli, Gim, f2(0.f), f2(0.f));
      Alm = d2_dot2<false>(d2_neg(Zmr), Gre, Zmi, Gim, f2(0.f), f2(0.f));
      if (wantV) Vlm = d2_dot2<false>(Zlr, Gim, Zli, Gre, f2(0.f), f2(0.f));
    }
    if (a.transpose) {
      const df2 t = Aml;
      Aml = Alm;
      Alm = t;
    }
    const int oa = rp * ld + tx, ob = oa + 16 * ld;
    if (fwd) {
      fast_store<K16>(o, oa, Aml.hi.x, Aml.lo.x);
      fast_store<K16>(o, ob, Aml.hi.y, Aml.lo.y);
    }
    sAT[tx][rp] = dfl{Alm.hi.x, Alm.lo.x};
    sAT[tx][rp + 16] = dfl{Alm.hi.y, Alm.lo.y};
    if (SM && wantV && fwd) {
      o.vhi[oa] = Vml.hi.x;
      o.vlo[oa] = Vml.lo.x;
      o.vhi[ob] = Vml.hi.y;
      o.vlo[ob] = Vml.lo.y;
    }
    if (SL && wantV) {
      sVT[tx][rp] = dfl{Vlm.hi.x, Vlm.lo.x};
      sVT[tx][rp + 16] = dfl{Vlm.hi.y, Vlm.lo.y};
    }
  }
  __syncthreads();
  if (!tr) return;
  // transposed block: rows l0 + rl, columns m0 + tx
  FastOut t = {a.hi + blm, a.lo + blm, a.Vhi ? a.Vhi + blm : nullptr, a.Vlo ? a.Vlo + blm : nullptr,
               K16 == 0 ? nullptr : (void*)((char*)a.h16 + 2 * blm)};
#pragma unroll
  for (int k = 0; k < ATILE / 8; ++k) {
    const int rl = ty + 8 * k;
    const int off = rl * ld + tx;
    const dfl v = sAT[rl][tx];
    fast_store<K16>(t, off, v.hi, v.lo);
    if (SL && wantV) {
      const dfl w = sVT[rl][tx];
      t.vhi[off] = w.hi;
      t.vlo[off] = w.lo;
    }
  }
}

// One CTA per tile pair {(I,J), (J,I)}, I <= J.  Each unordered node pair
// (m, l) gives G once; A_ml = component of zeta_l' G, A_lm = component of
// -zeta_m' G (the kernel is odd), and on surface rows the U-matrix entries
//   V_rc = -Im{zeta_r' G_rc} (c off the surface),  T_{r-c} + Re{zeta_r' G_rc}
// (c on the surface; T the Hilbert-regularising term), V_rr = -Re{zeta''/(2 zeta')},
// so that s_alpha U_r = [eq. d:phi:mv] + sum_c V_rc omega_c'/M_c - 1/2 H omega_0'.
// Transposed entries go through shared memory for coalesced stores.
template <class R, int K16>
__global__ void __launch_bounds__(256, 4) k_assemble_pairs(AsmArgs a) {
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
  // rows of tile I (the (I,J) block) and of tile J (the transposed block) held here
  const bool fwd = I * ATILE >= a.row0 && I * ATILE < a.row1;
  const bool tr = J * ATILE >= a.row0 && J * ATILE < a.row1;
  if (!fwd && !tr) return;
  if constexpr (std::is_same<R, dfl>::value) {
    int bI, bJ;
    if (a.tile_blk && fast_tile_pair(a, I, J, bI, bJ)) {
      if (bI == 0 && bJ == 0) asm_fast<K16, true, true, false>(a, I, J, fwd, tr, sAT, sVT);
      else if (bI == 0) asm_fast<K16, true, false, false>(a, I, J, fwd, tr, sAT, sVT);
      else if (bJ == 0) asm_fast<K16, false, true, false>(a, I, J, fwd, tr, sAT, sVT);
      else if (bI == bJ && bI >= 2) asm_fast<K16, false, false, true>(a, I, J, fwd, tr, sAT, sVT);
      else asm_fast<K16, false, false, false>(a, I, J, fwd, tr, sAT, sVT);
      return;
    }
  }
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
    const size_t iml = (size_t)(m - a.row0) * a.ld + l;
    if (m == l) {
      R dv = sD[rm];
      if (bm >= 2 && a.alt) dv = r_add(dv, NodeLoad<R>::Ualt(a, bm, m));
      else if (bm >= 2 && !a.vs) dv = r_addf(dv, -1.0f);
      NodeLoad<R>::template storeA<K16>(a, iml, dv);   // diagonal tile: fwd holds
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
    if (fwd) NodeLoad<R>::template storeA<K16>(a, iml, Aml);
    sAT[tx][rm] = Alm;
    if ((sm || sl) && !a.transpose) {
      int tj = 0;
      if (sm && sl) {   // both on the surface: 0 <= m, l < M_0
        tj = m - l;
        if (tj < 0) tj += a.M0;
      }
      if (sm && fwd) {  // V_ml
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
  if (!tr) return;
  // transposed block: rows l0 + rl, columns m0 + cm
  const int cm = tx;
  const int mcol = m0 + cm;
#pragma unroll 1
  for (int k = 0; k < ATILE / 8; ++k) {
    const int rl = ty + 8 * k;
    const int lrow = l0 + rl;
    if (lrow >= a.N || mcol >= a.N) continue;
    if (diagTile && cm >= rl) continue;
    const size_t ilm = (size_t)(lrow - a.row0) * a.ld + mcol;
    NodeLoad<R>::template storeA<K16>(a, ilm, sAT[rl][cm]);
    if (lrow < a.M0 && !a.transpose) NodeLoad<R>::storeV(a, ilm, sVT[rl][cm]);
  }
}

// zero the padding columns [N, ld) of A (rows < N) and of V (rows < M0)
template <class R>
__global__ void k_zero_pad(AsmArgs a) {
  const int pad = (int)(a.ld - a.N);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pad <= 0 || t >= (long long)(a.row1 - a.row0) * pad) return;
  const int r = a.row0 + (int)(t / pad);
  const size_t idx = (size_t)(r - a.row0) * a.ld + a.N + (int)(t % pad);
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
  a.row0 = c->row0;
  a.row1 = c->row1;
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
  const bool keep_solids = !partitioned(c) && sig == c->asm_sig && c->asm_solid_version == c->solid_version;
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
  const size_t NN = (size_t)local_rows(c) * (size_t)c->ld;
  const size_t VN = (size_t)local_vrows(c) * (size_t)c->ld;
  // upper-triangular tile pairs in row-major order: the pairs with row tile
  // I < ceil(M_0 / ATILE) (every pair touching a surface node) come first
  const long long T = a.ntile, tS = std::min<long long>(T, (c->M[0] + ATILE - 1) / ATILE);
  const unsigned ntiles = (unsigned)(keep_solids ? tS * T - tS * (tS - 1) / 2 : T * (T + 1) / 2);
  const long long npad = (long long)local_rows(c) * (c->ld - c->N);
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
    if (!a.alt && !a.vs) {   // tile tables of the fast path
      int* tblk;
      float4 *tbox, *trows;
      BIE_GET(c, int, "tile_blk", a.ntile, tblk);
      BIE_GET(c, float4, "tile_box", a.ntile, tbox);
      BIE_GET(c, float4, "tile_rows", (size_t)a.ntile * 16 * 5, trows);
      k_tile_prep<<<a.ntile, 32, 0, c->stream>>>(a, tblk, tbox, trows);
      BIE_LAUNCH_CHECK(c, "k_tile_prep");
      a.tile_blk = tblk;
      a.tile_box = tbox;
      a.tile_rows = trows;
    }
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
