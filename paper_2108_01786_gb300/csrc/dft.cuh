// Four-step FP64 DFT jobs shared by the normal-velocity and target kernels.
#pragma once
#include "common.cuh"

struct DftJob {
  int M, M1, M2;
  int off_in;    // input offset (real omega for mode 0, spectrum for modes 1/2)
  int off_out;   // output offset in the complex work array
  int off_tw;    // twiddle table offset (e^{-2 pi i j / M}, j < M)
  int mode;      // 0: real input; 1: conj(i k X); 2: conj(|k| X); 3: complex input;
                 // 4: conj(-i sgn(k) X) (Hilbert transform); 5: conj(-k^2 X)
                 // (second derivative); 6: conj(rho(k) X) (filter of eq. filter);
                 // 7: conj(X/(ik)), zero at k = 0 (zero-mean antiderivative)
  int start;     // first global element of this job
};
struct DftJobs {
  int n;
  int total;
  DftJob j[2 * BIE_MAXB + 2];
};


// Each output is summed by DFT_SPLIT lanes: launch dft_grid(outputs/256 blocks)
// blocks of 256 threads.
#define DFT_SPLIT 8
inline dim3 dft_grid(dim3 g) { return dim3(g.x * DFT_SPLIT, g.y, g.z); }

// The same jobs for gridDim.y independent vectors: vector y reads at
// y * in_stride and writes at y * out_stride (elements of the arrays passed).
__global__ void k_dft_a(DftJobs J, const double* __restrict__ xr, const double2* __restrict__ xc,
                        const double2* __restrict__ tw, double2* __restrict__ Y,
                        long long in_stride = 0, long long out_stride = 0);
__global__ void k_dft_b(DftJobs J, const double2* __restrict__ Y, const double2* __restrict__ tw,
                        double2* __restrict__ X, long long stride = 0);
