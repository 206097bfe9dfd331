// Row slices and fixed-order partial-sum reductions shared by the Krylov kernels.
#pragma once
#include "common.cuh"

__device__ __forceinline__ void slice_of(int N, int& r0, int& r1) {
  const int S = (N + gridDim.x - 1) / gridDim.x;
  r0 = blockIdx.x * S;
  r1 = min(N, r0 + S);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0
}

// out_smem[i] = sum of the first np (<= BIE_PSTRIDE) partials of row i
// (i < cnt).  One warp per row, two rows at a time: every lane issues the
// loads of both rows (at most eight each) back to back and adds each row in a
// fixed order, then a fixed shuffle tree: one L2 round trip per sixteen rows
// (deterministic order).
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int cnt, int np,
                                                double* __restrict__ out_smem) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < cnt; i += 2 * nw) {
    const int i2 = i + nw;
    const double* row = part + (size_t)i * BIE_PSTRIDE;
    const double* row2 = part + (size_t)i2 * BIE_PSTRIDE;
    double v[BIE_PSTRIDE / 32], v2[BIE_PSTRIDE / 32];
#pragma unroll
    for (int u = 0; u < BIE_PSTRIDE / 32; ++u) {
      const int c = lane + 32 * u;
      v[u] = c < np ? row[c] : 0.0;
      v2[u] = (c < np && i2 < cnt) ? row2[c] : 0.0;
    }
    double s = 0.0, s2 = 0.0;
#pragma unroll
    for (int u = 0; u < BIE_PSTRIDE / 32; ++u) {
      s += v[u];
      s2 += v2[u];
    }
    s = warp_sum(s);
    s2 = warp_sum(s2);
    if (lane == 0) {
      out_smem[i] = s;
      if (i2 < cnt) out_smem[i2] = s2;
    }
  }
}

// acc - sum_{i<=j} h[i] V_i[m], subtracting in the order i = 0, 1, ..., j; the
// loads of eight vectors are issued before their products so that one L2
// round trip serves eight terms (the loop is latency bound, not bandwidth bound)
template <class VT>
__device__ __forceinline__ VT subtract_basis(VT acc, const double* __restrict__ h,
                                             const VT* __restrict__ V, long long ld, int j,
                                             int m) {
  int i = 0;
  for (; i + 7 <= j; i += 8) {
    VT v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = V[(size_t)(i + u) * ld + m];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc -= (VT)h[i + u] * v[u];
  }
  for (; i <= j; ++i) acc -= (VT)h[i] * V[(size_t)i * ld + m];
  return acc;
}

// The previous Givens rotations 0..j-1 applied to a new Hessenberg column h
// (h[0..j], raw entries; h[j+1] = beta is not touched) by one warp.  Rotation i
// maps (u_i, h_{i+1}) to (c_i u_i + s_i h_{i+1}, -s_i u_i + c_i h_{i+1}) with u_0 = h_0:
// the second component is an affine map of u_i, so the sequential recurrence
// is a warp scan of affine maps (64 rotations per pass); the first component
// is written back as h[i].  Returns u_j (the entry at j after the rotations)
// in every lane.
__device__ __forceinline__ double givens_apply_warp(double* h, const double* __restrict__ cs,
                                                    const double* __restrict__ sn, int j) {
  const int lane = threadIdx.x & 31;
  double u = h[0];
  for (int base = 0; base < j; base += 64) {
    const int e0 = base + 2 * lane, e1 = e0 + 1;
    const bool v0 = e0 < j, v1 = e1 < j;
    const double c0 = v0 ? cs[e0] : 1.0, s0 = v0 ? sn[e0] : 0.0, h0 = v0 ? h[e0 + 1] : 0.0;
    const double c1 = v1 ? cs[e1] : 1.0, s1 = v1 ? sn[e1] : 0.0, h1 = v1 ? h[e1 + 1] : 0.0;
    // f_e(u) = A_e u + B_e, A_e = -s_e, B_e = c_e h_{e+1} (identity past j)
    const double A0 = v0 ? -s0 : 1.0, B0 = v0 ? c0 * h0 : 0.0;
    const double A1 = v1 ? -s1 : 1.0, B1 = v1 ? c1 * h1 : 0.0;
    double A = A1 * A0, B = fma(A1, B0, B1);   // f_e1 after f_e0
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {          // inclusive scan, later maps applied last
      const double Ap = __shfl_up_sync(0xffffffffu, A, d);
      const double Bp = __shfl_up_sync(0xffffffffu, B, d);
      if (lane >= d) {
        B = fma(A, Bp, B);
        A = A * Ap;
      }
    }
    double Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) {
      Ae = 1.0;
      Be = 0.0;
    }
    const double ue0 = fma(Ae, u, Be);           // u at e0
    const double ue1 = fma(A0, ue0, B0);         // u at e1
    const double ue2 = fma(A1, ue1, B1);         // u at e1 + 1
    const double last = __shfl_sync(0xffffffffu, ue2, 31);   // u at base + 64 (or j)
    __syncwarp();
    if (v0) h[e0] = fma(c0, ue0, s0 * h0);
    if (v1) h[e1] = fma(c1, ue1, s1 * h1);
    __syncwarp();
    u = last;
  }
  return u;
}
