// Products of the stored low-precision matrix with several vectors at once
// (the multi-right-hand-side dense product) on the 5th-generation tensor cores.
//
// Y_r = A x_r for r < nrhs:  y_m = sum_l S_ml x_l / M_l + s_m x_m, with S the
// FP16 (or BF16) storage of eq. lin:sys.  The sum is a GEMM of S (N x N) with
// the columns x_r / M_l, one of the few dense contractions of the method: k
// right-hand sides make it k flops per stored byte, beyond the CUDA cores past
// k ~ 10 at HBM speed, within the tensor cores' reach to k ~ 64+.
//
// Kernel: CTA (row block of 128, K range) streams 128 x 64 tiles of S and
// NR x 64 tiles of the scaled columns with TMA (cp.async.bulk.tensor, 128-byte
// swizzle) into an S-stage shared-memory ring; one thread issues
// tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = NR, K = 16, FP32
// accumulators in tensor memory), committing each stage back to the producer
// through an mbarrier; at the end all four warps read their 32 rows from
// tensor memory (tcgen05.ld 32x32b) and store FP32 partial sums per K range.
// A finishing kernel adds the K ranges in a fixed order and applies the
// column scale, 1/M_l and s_m.  Waits are bounded; a CTA whose wait expires
// sets an error flag and returns after freeing its tensor memory.
//
// Each column is scaled by 1/max_l |x_l / M_l| before rounding to FP16/BF16,
// so any input stays in range; the product carries the storage's ~2^-11
// (FP16) or ~2^-8 (BF16) relative rounding, as the inner GMRES products do.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"

#define MM_KT 64
#define MM_SPIN (1u << 22)

__device__ __forceinline__ unsigned mm_sa(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of 1024 B
__device__ __forceinline__ uint64_t mm_desc_sw128(unsigned addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;               // leading byte offset (not used by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}
__device__ __forceinline__ bool mm_wait(unsigned long long* b, unsigned parity) {
  for (unsigned it = 0; it < MM_SPIN; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mm_sa(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <int NR, int STAGES, bool BF16>
__global__ void __launch_bounds__(128, 1)
    k_mm_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tX,
            float* __restrict__ Yp, int N, long long ld, int split, int* __restrict__ err) {
  constexpr int ABYTES = 128 * MM_KT * 2;
  constexpr int BBYTES = NR * MM_KT * 2;
  constexpr int SBYTES = ABYTES + (BBYTES + 1023) / 1024 * 1024;
  constexpr int TCOLS = NR < 32 ? 32 : NR;
  extern __shared__ __align__(1024) unsigned char mm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)mm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) unsigned long long full[STAGES], empty[STAGES], done;
  __shared__ unsigned tslot;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rb = blockIdx.x / split, ks = blockIdx.x % split;
  const int ntot = (int)(ld / MM_KT);
  const int t0 = (int)((long long)ntot * ks / split);
  const int nt = (int)((long long)ntot * (ks + 1) / split) - t0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     mm_sa(&tslot)),
                 "r"(TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mm_sa(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mm_sa(&empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mm_sa(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tslot;
  // instruction descriptor: FP32 accumulators, FP16 or BF16 operands, both
  // K-major, N = NR, M = 128
  const uint32_t fmt = BF16 ? 1u : 0u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NR >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  if (warp == 0 && lane == 0) {   // TMA producer
    for (int t = 0; t < nt; ++t) {
      const int s = t % STAGES;
      if (t >= STAGES && !mm_wait(&empty[s], (unsigned)((t / STAGES) - 1) & 1u)) {
        fail = 1;
        atomicExch(err, 1);
        break;
      }
      unsigned char* st = sm + (size_t)s * SBYTES;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mm_sa(&full[s])),
                   "r"(ABYTES + BBYTES)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
          "{%2, %3}], [%4];" ::"r"(mm_sa(st)),
          "l"(&tA), "r"((t0 + t) * MM_KT), "r"(rb * 128), "r"(mm_sa(&full[s]))
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
          "{%2, %3}], [%4];" ::"r"(mm_sa(st + ABYTES)),
          "l"(&tX), "r"((t0 + t) * MM_KT), "r"(0), "r"(mm_sa(&full[s]))
          : "memory");
    }
  } else if (warp == 1 && lane == 0) {   // MMA issuer
    for (int t = 0; t < nt; ++t) {
      const int s = t % STAGES;
      if (!mm_wait(&full[s], (unsigned)(t / STAGES) & 1u)) {
        fail = 1;
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned st = mm_sa(sm + (size_t)s * SBYTES);
      for (int kk = 0; kk < MM_KT / 16; ++kk) {
        const uint64_t ad = mm_desc_sw128(st + kk * 32);
        const uint64_t bd = mm_desc_sw128(st + ABYTES + kk * 32);
        const unsigned acc = (t > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              mm_sa(&empty[s]))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            mm_sa(&done))
        : "memory");
  }
  __syncwarp();
  bool ok = mm_wait(&done, 0u);
  if (!ok) atomicExch(err, 1);
  ok = __syncthreads_and(ok && !fail) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const unsigned ta = tmem + ((unsigned)(warp * 32) << 16);
    const int row = rb * 128 + warp * 32 + lane;
#pragma unroll
    for (int c = 0; c < NR; c += 8) {
      uint32_t v[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                     "=r"(v[6]), "=r"(v[7])
                   : "r"(ta + c)
                   : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < N) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          Yp[((size_t)ks * NR + c + j) * ld + row] = __uint_as_float(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                 : "memory");
}

// per column r: scale_r = max_l |x_rl / M_l| (one CTA per column)
__global__ void __launch_bounds__(256) k_mm_colmax(int N, const double* __restrict__ X,
                                                   const double* __restrict__ wgt64,
                                                   double* __restrict__ scale) {
  __shared__ double red[8];
  const int r = blockIdx.x;
  double m = 0.0;
  for (int l = threadIdx.x; l < N; l += blockDim.x) m = fmax(m, fabs(X[(size_t)r * N + l] * wgt64[l]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t = fmax(t, red[w]);
    scale[r] = t > 0.0 ? t : 1.0;
  }
}

// XT[r][l] = x_rl / (M_l scale_r) rounded to FP16/BF16; zero padding rows and columns
template <bool BF16>
__global__ void k_mm_prep(int N, long long ld, int nrhs, int NR, const double* __restrict__ X,
                          const double* __restrict__ wgt64, const double* __restrict__ scale,
                          void* __restrict__ XT) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)NR * ld) return;
  const int r = (int)(i / ld);
  const int l = (int)(i - (long long)r * ld);
  double v = 0.0;
  if (r < nrhs && l < N) v = X[(size_t)r * N + l] * wgt64[l] / scale[r];
  if (BF16) ((__nv_bfloat16*)XT)[i] = __float2bfloat16_rn((float)v);
  else ((__half*)XT)[i] = __float2half_rn((float)v);
}

// y_rm = scale_r sum_ks Yp[ks][r][m] + s_m x_rm  (fixed order over K ranges)
__global__ void k_mm_finish(int N, long long ld, int nrhs, int NR, int split,
                            const float* __restrict__ Yp, const double* __restrict__ X,
                            const float* __restrict__ sgn, const double* __restrict__ scale,
                            double* __restrict__ Y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nrhs * N) return;
  const int r = (int)(i / N);
  const int m = (int)(i - (long long)r * N);
  double s = 0.0;
  for (int k = 0; k < split; ++k) s += (double)Yp[((size_t)k * NR + r) * ld + m];
  Y[i] = scale[r] * s + (double)sgn[m] * X[i];
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

template <int NR, int STAGES, bool BF16>
static bie_status mm_launch(bie_ctx* c, const CUtensorMap& tA, const CUtensorMap& tX, float* Yp,
                            int split, int* err) {
  constexpr int SBYTES = 128 * MM_KT * 2 + (NR * MM_KT * 2 + 1023) / 1024 * 1024;
  const size_t smem = (size_t)STAGES * SBYTES + 1024;
  auto kern = k_mm_tc<NR, STAGES, BF16>;
  BIE_CUDA_TRY(c, raise_smem_limit((const void*)kern, smem));
  const int nrb = (c->N + 127) / 128;
  kern<<<nrb * split, 128, smem, c->stream>>>(tA, tX, Yp, c->N, c->ld, split, err);
  BIE_LAUNCH_CHECK(c, "k_mm_tc");
  return BIE_OK;
}

// Y (nrhs x N, FP64) = A X with the low-precision storage on the tensor cores
bie_status mm_run(bie_ctx* c, int nrhs, const double* X, double* Y) {
  if (c->precision != BIE_FP16_IR && c->precision != BIE_BF16_IR)
    return ctx_fail(c, BIE_ERR_STATE, "bie_matmat: needs FP16 or BF16 storage");
  if (nrhs < 1 || nrhs > 64) return ctx_fail(c, BIE_ERR_ARG, "bie_matmat: 1 <= nrhs <= 64");
  EncodeTiledFn enc = encode_fn();
  if (!enc) return ctx_fail(c, BIE_ERR_CUDA, "bie_matmat: cuTensorMapEncodeTiled unavailable");
  const bool bf = c->precision == BIE_BF16_IR;
  const int NR = nrhs <= 16 ? 16 : (nrhs <= 32 ? 32 : 64);
  const int N = c->N;
  const long long ld = c->ld;
  const int nrb = (N + 127) / 128;
  const int ntiles = (int)(ld / MM_KT);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  int split = (3 * nsm + nrb - 1) / nrb;
  split = std::max(1, std::min(split, std::max(1, ntiles / 8)));
  const size_t NN = (size_t)N * (size_t)ld;
  bool oom = false;
  void* A16 = ctx_buf(c, "A_16", 2 * NN, &oom);
  const double* wgt64 = (const double*)ctx_buf(c, "wgt64", sizeof(double) * ld, &oom);
  const float* sgn = (const float*)ctx_buf(c, "sgn", sizeof(float) * ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_matmat: buffers");
  void* XT;
  float* Yp;
  double* scale;
  int* err;
  BIE_GET(c, unsigned short, "mm_xt", (size_t)NR * ld, XT);
  BIE_GET(c, float, "mm_yp", (size_t)split * NR * ld, Yp);
  BIE_GET(c, double, "mm_scale", 64, scale);
  BIE_GET(c, int, "mm_err", 1, err);
  BIE_CUDA_TRY(c, cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  k_mm_colmax<<<nrhs, 256, 0, c->stream>>>(N, X, wgt64, scale);
  BIE_LAUNCH_CHECK(c, "k_mm_colmax");
  const unsigned gp = (unsigned)(((long long)NR * ld + 255) / 256);
  if (bf) k_mm_prep<true><<<gp, 256, 0, c->stream>>>(N, ld, nrhs, NR, X, wgt64, scale, XT);
  else k_mm_prep<false><<<gp, 256, 0, c->stream>>>(N, ld, nrhs, NR, X, wgt64, scale, XT);
  BIE_LAUNCH_CHECK(c, "k_mm_prep");
  // tensor maps: S (ld x N) and XT (ld x NR), boxes 64 x 128 and 64 x NR, 128-byte swizzle
  CUtensorMap tA, tX;
  const CUtensorMapDataType dt = bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t gdA[2] = {(cuuint64_t)ld, (cuuint64_t)N}, gsA[1] = {(cuuint64_t)ld * 2};
  const cuuint64_t gdX[2] = {(cuuint64_t)ld, (cuuint64_t)NR}, gsX[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t bA[2] = {MM_KT, 128}, bX[2] = {MM_KT, (cuuint32_t)NR}, es[2] = {1, 1};
  if (enc(&tA, dt, 2, A16, gdA, gsA, bA, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&tX, dt, 2, XT, gdX, gsX, bX, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return ctx_fail(c, BIE_ERR_CUDA, "bie_matmat: tensor map encoding failed");
  bie_status s;
  if (NR == 16) s = bf ? mm_launch<16, 6, true>(c, tA, tX, Yp, split, err) : mm_launch<16, 6, false>(c, tA, tX, Yp, split, err);
  else if (NR == 32) s = bf ? mm_launch<32, 6, true>(c, tA, tX, Yp, split, err) : mm_launch<32, 6, false>(c, tA, tX, Yp, split, err);
  else s = bf ? mm_launch<64, 5, true>(c, tA, tX, Yp, split, err) : mm_launch<64, 5, false>(c, tA, tX, Yp, split, err);
  if (s != BIE_OK) return s;
  const unsigned gf = (unsigned)(((long long)nrhs * N + 255) / 256);
  k_mm_finish<<<gf, 256, 0, c->stream>>>(N, ld, nrhs, NR, split, Yp, X, sgn, scale, Y);
  BIE_LAUNCH_CHECK(c, "k_mm_finish");
  int herr = 0;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) return ctx_fail(c, BIE_ERR_TIMEOUT, "bie_matmat: a pipeline wait timed out");
  return BIE_OK;
}

extern "C" bie_status bie_matmat(bie_ctx* c, int nrhs, const double* X_dev, double* Y_dev) {
  if (!c) return BIE_ERR_ARG;
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_matmat: not assembled");
  if (c->transposed)
    return ctx_fail(c, BIE_ERR_STATE, "bie_matmat: storage holds the adjoint operator; assemble again");
  if (!X_dev || !Y_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_matmat: null pointer");
  cudaSetDevice(c->device);
  return mm_run(c, nrhs, X_dev, Y_dev);
}
