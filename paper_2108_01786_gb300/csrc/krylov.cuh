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

// out_smem[i] = sum of the first np partials of row i (i < cnt).  Four
// threads per row, each summing a fixed quarter with independent loads, then
// two shuffles: one L2 round trip instead of one per row (deterministic order).
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int cnt, int np,
                                                double* __restrict__ out_smem) {
  const int q = threadIdx.x & 3;
  for (int base = 0; base < cnt; base += (int)(blockDim.x >> 2)) {
    const int i = base + (int)(threadIdx.x >> 2);
    double s = 0.0;
    if (i < cnt) {
      const double* row = part + (size_t)i * BIE_PSTRIDE;
      for (int c = q; c < np; c += 4) s += row[c];
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (i < cnt && q == 0) out_smem[i] = s;
  }
}

