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
#include "nvtx.cuh"

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

// One 128-row block rb of Y (NR columns, FP32) = A[rb rows, K tiles t0..t0+nt) X^T
// on the tensor cores: a TMA producer thread, an MMA issuer thread, the
// accumulator in TMEM, every wait bounded (a timed-out wait sets *err and the
// block skips its store).  tA / tX point at tensor maps in parameter space.
template <int NR, int STAGES, bool BF16>
__device__ __forceinline__ void mm_tile(const CUtensorMap* tA, const CUtensorMap* tX,
                                        float* __restrict__ Yp, int N, long long ld, int rb,
                                        int t0, int nt, int* __restrict__ err) {
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
          "l"(tA), "r"((t0 + t) * MM_KT), "r"(rb * 128), "r"(mm_sa(&full[s]))
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
          "{%2, %3}], [%4];" ::"r"(mm_sa(st + ABYTES)),
          "l"(tX), "r"((t0 + t) * MM_KT), "r"(0), "r"(mm_sa(&full[s]))
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
          Yp[(size_t)(c + j) * ld + row] = __uint_as_float(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS)
                 : "memory");
}

// Yp[ks][c][m] for split K ranges ks (grid: row blocks x split)
template <int NR, int STAGES, bool BF16>
__global__ void __launch_bounds__(128, 1)
    k_mm_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tX,
            float* __restrict__ Yp, int N, long long ld, int split, int* __restrict__ err) {
  const int rb = blockIdx.x / split, ks = blockIdx.x % split;
  const int ntot = (int)(ld / MM_KT);
  const int t0 = (int)((long long)ntot * ks / split);
  const int nt = (int)((long long)ntot * (ks + 1) / split) - t0;
  mm_tile<NR, STAGES, BF16>(&tA, &tX, Yp + (size_t)ks * NR * ld, N, ld, rb, t0, nt, err);
}

// Several products of the same width in one launch: item i multiplies the
// matrix of tensor map tA[lvl[i]] by the columns of tX[i] into Y[i] (whole K).
// Blocks run row block by row block with the items innermost, so items that
// share a matrix stream the same rows at the same time and share them in L2.
#define MM_GMAX 32
#define MM_GMATS 10
struct MmGroup {
  CUtensorMap tA[MM_GMATS];
  CUtensorMap tX[MM_GMAX];
  float* Y[MM_GMAX];
  int lvl[MM_GMAX];
  int n;
};
template <int NR, int STAGES>
__global__ void __launch_bounds__(128, 1)
    k_mm_tc_grp(const __grid_constant__ MmGroup G, int N, long long ld, int* __restrict__ err) {
  const int item = (int)blockIdx.x % G.n, rb = (int)blockIdx.x / G.n;
  mm_tile<NR, STAGES, false>(&G.tA[G.lvl[item]], &G.tX[item], G.Y[item], N, ld, rb, 0,
                             (int)(ld / MM_KT), err);
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
  BIE_NVTX("bie_matmat");
  if (!c) return BIE_ERR_ARG;
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_matmat: not available on a row-partitioned context");
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_matmat: not assembled");
  if (c->transposed)
    return ctx_fail(c, BIE_ERR_STATE, "bie_matmat: storage holds the adjoint operator; assemble again");
  if (!X_dev || !Y_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_matmat: null pointer");
  cudaSetDevice(c->device);
  return mm_run(c, nrhs, X_dev, Y_dev);
}

// ===========================================================================
// The full-accuracy (hi + lo, ~48-bit) operator on the tensor cores, by exact
// integer slices (an Ozaki-type splitting of both operands).
//
// Row m of the stored matrix is scaled by 2^-e_m (|A_ml| < 2^e_m) and cut into
// OZ_S slices of OZ_BITS bits: A_ml = 2^e_m sum_s a_s,ml 2^-5(s+1) + (below
// 2^-50 of the row scale), every a_s an integer with |a_0| <= 32, |a_s| <= 16,
// stored exactly in FP16.  Each column x_c (already divided by M_l) is cut the
// same way with its own scale 2^f_c.  A slice product sum_l a_s,ml x_t,cl is a
// sum of at most 16384 integers of size <= 2^10: exact in the FP32 tensor
// accumulators (< 2^24), so each of the GEMMs below is exact, and the FP64
// combination y = sum_{s+t<S} 2^(e_m + f_c - 5(s+t+2)) P_st carries only the
// truncation of the pairs s + t >= S (2^-5S of the row scale) and FP64
// rounding.  For ld > 16384 the K range is split so that every part stays exact.
// ===========================================================================
#define OZ_BITS 5
#define OZ_S 10
#define OZ_KMAX 16384   // K per exact accumulation: 16384 x 2^10 = 2^24
#define OZ_MIN_RHS 8    // below this many columns the double-float GEMV is faster

// e_m: max_l |A_ml| (1 + 2^-20) < 2^e_m, one warp per row
__global__ void k_oz_rowexp(int N, long long ld, const float* __restrict__ Ahi, int* __restrict__ e) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= N) return;
  const float4* row = reinterpret_cast<const float4*>(Ahi + (size_t)warp * ld);
  float mx = 0.f;
  for (long long v = lane; v < ld / 4; v += 32) {
    const float4 q = row[v];
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fmaxf(fabsf(q.z), fabsf(q.w))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    int k = 0;
    if (mx > 0.f) frexp((double)mx * (1.0 + 0x1p-20), &k);   // mx (1 + 2^-20) < 2^k
    e[warp] = k;
  }
}

// slices of the hi + lo storage: S[s][m][l], value a_s,ml (exact integers in FP16)
__global__ void k_oz_slice_A(int N, long long ld, const float* __restrict__ Ahi,
                             const float* __restrict__ Alo, const int* __restrict__ e,
                             __half* __restrict__ S) {
  const size_t total = (size_t)N * ld;
  const size_t plane = total;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / ld);
    const int em = e[m];
    float x, y;   // the entry scaled by 2^-e_m: x + y, |x + y| < 1
    if (em > -126 && em < 126) {
      const float sc = __int_as_float((127 - em) << 23);   // 2^-e_m exactly
      x = Ahi[i] * sc;
      y = Alo[i] * sc;
    } else {
      x = ldexpf(Ahi[i], -em);
      y = ldexpf(Alo[i], -em);
    }
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) {
      x *= (float)(1 << OZ_BITS);
      y *= (float)(1 << OZ_BITS);
      const float a = rintf(x);
      x -= a;                                        // exact
      const float t = x + y, bb = t - x;             // (x, y) <- two-sum (exact pair)
      y = (x - (t - bb)) + (y - bb);
      x = t;
      S[(size_t)s * plane + i] = __float2half_rn(a);   // |a| <= 32: exact
    }
  }
}

// f_c: max_l |x_cl / M_l| < 2^f_c (one CTA per column)
__global__ void __launch_bounds__(256) k_oz_colexp(int N, const double* __restrict__ X, long long xs,
                                                   const double* __restrict__ wgt64,
                                                   int* __restrict__ f) {
  __shared__ double red[8];
  const int r = blockIdx.x;
  double m = 0.0;
  for (int l = threadIdx.x; l < N; l += blockDim.x) m = fmax(m, fabs(X[(size_t)r * xs + l] * wgt64[l]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t = fmax(t, red[w]);
    int k = 0;
    if (t > 0.0) frexp(t * (1.0 + 0x1p-40), &k);
    f[r] = k;
  }
}

// XS[t nrhs + c][l] = slice t of x_cl / M_l (FP64 extraction, exact integers in FP16)
__global__ void k_oz_slice_x(int N, long long ld, int nrhs, int S, const double* __restrict__ X,
                             long long xs, const double* __restrict__ wgt64,
                             const int* __restrict__ f, __half* __restrict__ XS) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nrhs * ld) return;
  const int c = (int)(i / ld);
  const int l = (int)(i - (long long)c * ld);
  double v = (l < N) ? ldexp(X[(size_t)c * xs + l] * wgt64[l], -f[c]) : 0.0;
  for (int t = 0; t < S; ++t) {
    v *= (double)(1 << OZ_BITS);
    const double a = rint(v);
    v -= a;
    XS[((size_t)t * nrhs + c) * ld + l] = __float2half_rn((float)a);
  }
}

// y[c][m] = sum_{s+t<S} 2^(e_m + f_c - 5(s+t+2)) sum_k P[s][ks][t nrhs + c][m]
struct OzProducts {
  const float* P[OZ_S];   // slice s: [split][cols_s padded][ld]
  int ldP[OZ_S];          // column stride count per K part (padded columns)
};
__global__ void k_oz_combine(int N, long long ld, int nrhs, int S, int split, OzProducts pr,
                             const int* __restrict__ e, const int* __restrict__ f,
                             double* __restrict__ Y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nrhs * N) return;
  const int c = (int)(i / N);
  const int m = (int)(i - (long long)c * N);
  const int base = e[m] + f[c];
  double y = 0.0;
  // pairs with the same s + t share one scale: their integer sum is exact in FP64
  for (int L = S - 1; L >= 0; --L) {
    double p = 0.0;
    for (int s = 0; s <= L; ++s) {
      const int t = L - s;
      for (int k = 0; k < split; ++k)
        p += (double)pr.P[s][((size_t)k * pr.ldP[s] + (size_t)t * nrhs + c) * ld + m];
    }
    y += ldexp(p, base - OZ_BITS * (L + 2));
  }
  Y[(size_t)c * ld + m] = y;
}

static int oz_nr(int cols) {
  return cols <= 16 ? 16 : cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : 256;
}

__global__ void k_oz_fill(long long n, double* __restrict__ v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = 1.0;
}

// which = 0: the matrix A (N rows, "A_hi"/"A_lo"); which = 1: the surface
// U-matrix (M_0 rows, "V_hi"/"V_lo").  Slices are built once per assembly.
struct OzMat {
  const char *hi, *lo, *slices, *exps;
  int rows;
};
static OzMat oz_mat(const bie_ctx* c, int which) {
  return which == 0 ? OzMat{"A_hi", "A_lo", "oz_A", "oz_e", c->N}
                    : OzMat{"V_hi", "V_lo", "oz_V", "oz_ev", c->M[0]};
}

static bie_status oz_prepare(bie_ctx* c, int which) {
  int& held = which == 0 ? c->oz_count : c->ozv_count;
  if (held == c->asm_count) return BIE_OK;
  const OzMat mt = oz_mat(c, which);
  const long long ld = c->ld;
  const size_t NN = (size_t)mt.rows * ld;
  bool oom = false;
  const float* Ahi = (const float*)ctx_buf(c, mt.hi, sizeof(float) * NN, &oom);
  const float* Alo = (const float*)ctx_buf(c, mt.lo, sizeof(float) * NN, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "exact product: storage");
  int* e;
  __half* S;
  BIE_GET(c, int, mt.exps, mt.rows, e);
  BIE_GET(c, __half, mt.slices, (size_t)OZ_S * NN, S);
  k_oz_rowexp<<<(unsigned)((32LL * mt.rows + 255) / 256), 256, 0, c->stream>>>(mt.rows, ld, Ahi, e);
  BIE_LAUNCH_CHECK(c, "k_oz_rowexp");
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  k_oz_slice_A<<<8 * nsm, 256, 0, c->stream>>>(mt.rows, ld, Ahi, Alo, e, S);
  BIE_LAUNCH_CHECK(c, "k_oz_slice_A");
  held = c->asm_count;
  return BIE_OK;
}

// Y[c][m] (FP64, [nrhs][ld]) = sum_l B_ml x_cl w_l for the matrix `which`
// (w_l = 1/M_l when apply_w, else 1) with the hi + lo storage, using the first
// S slices of each operand (S = OZ_S for the full accuracy)
static bie_status oz_product(bie_ctx* c, int which, int nrhs, const double* X, long long xs,
                             int apply_w, int S, double* Y) {
  bie_status st = oz_prepare(c, which);
  if (st != BIE_OK) return st;
  const OzMat mt = oz_mat(c, which);
  const int N = c->N, R = mt.rows;
  const long long ld = c->ld;
  const size_t NN = (size_t)R * ld;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return ctx_fail(c, BIE_ERR_CUDA, "exact product: cuTensorMapEncodeTiled unavailable");
  bool oom = false;
  const double* wgt64 = (const double*)ctx_buf(c, "wgt64", sizeof(double) * ld, &oom);
  __half* SA = (__half*)ctx_buf(c, mt.slices, sizeof(__half) * (size_t)OZ_S * NN, &oom);
  const int* e = (const int*)ctx_buf(c, mt.exps, sizeof(int) * R, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "exact product: buffers");
  const int split = (int)((ld + OZ_KMAX - 1) / OZ_KMAX);
  if (split != 1) return ctx_fail(c, BIE_ERR_ARG, "exact product: more than 16384 unknowns per row");
  int *f, *err;
  __half* XS;
  double* ones = nullptr;
  BIE_GET(c, int, "oz_f", nrhs, f);
  BIE_GET(c, int, "oz_err", 1, err);
  BIE_GET(c, __half, "oz_X", (size_t)S * nrhs * ld, XS);
  if (!apply_w) {
    BIE_GET(c, double, "oz_ones", ld, ones);
    k_oz_fill<<<(unsigned)((ld + 255) / 256), 256, 0, c->stream>>>(ld, ones);
    BIE_LAUNCH_CHECK(c, "k_oz_fill");
  }
  const double* w = apply_w ? wgt64 : ones;
  BIE_CUDA_TRY(c, cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  k_oz_colexp<<<nrhs, 256, 0, c->stream>>>(N, X, xs, w, f);
  BIE_LAUNCH_CHECK(c, "k_oz_colexp");
  k_oz_slice_x<<<(unsigned)(((long long)nrhs * ld + 255) / 256), 256, 0, c->stream>>>(
      N, ld, nrhs, S, X, xs, w, f, XS);
  BIE_LAUNCH_CHECK(c, "k_oz_slice_x");
  OzProducts pr;
  memset(&pr, 0, sizeof(pr));
  const cuuint32_t es[2] = {1, 1};
  const char* names[OZ_S] = {"oz_P0", "oz_P1", "oz_P2", "oz_P3", "oz_P4",
                             "oz_P5", "oz_P6", "oz_P7", "oz_P8", "oz_P9"};
  // every (slice level s, chunk of <= 256 columns) product, launched in groups
  // of equal width: items of one level share the rows of A_s in L2
  static_assert(OZ_S <= MM_GMATS, "one tensor map per slice level");
  MmGroup grp[5];
  memset(grp, 0, sizeof(grp));
  auto slot_of = [](int NR) { return NR == 16 ? 0 : NR == 32 ? 1 : NR == 64 ? 2 : NR == 128 ? 3 : 4; };
  auto flush = [&](int g) -> bie_status {
    MmGroup& G = grp[g];
    if (G.n == 0) return BIE_OK;
    const int NR = 16 << g;
    const int STAGES = NR <= 32 ? 6 : NR <= 128 ? 5 : 4;
    const int SBYTES = 128 * MM_KT * 2 + (NR * MM_KT * 2 + 1023) / 1024 * 1024;
    const size_t smem = (size_t)STAGES * SBYTES + 1024;
    const unsigned grid = (unsigned)(((R + 127) / 128) * G.n);
    const void* kern = g == 0   ? (const void*)k_mm_tc_grp<16, 6>
                       : g == 1 ? (const void*)k_mm_tc_grp<32, 6>
                       : g == 2 ? (const void*)k_mm_tc_grp<64, 5>
                       : g == 3 ? (const void*)k_mm_tc_grp<128, 5>
                                : (const void*)k_mm_tc_grp<256, 4>;
    BIE_CUDA_TRY(c, raise_smem_limit(kern, smem));
    switch (g) {
      case 0: k_mm_tc_grp<16, 6><<<grid, 128, smem, c->stream>>>(G, R, ld, err); break;
      case 1: k_mm_tc_grp<32, 6><<<grid, 128, smem, c->stream>>>(G, R, ld, err); break;
      case 2: k_mm_tc_grp<64, 5><<<grid, 128, smem, c->stream>>>(G, R, ld, err); break;
      case 3: k_mm_tc_grp<128, 5><<<grid, 128, smem, c->stream>>>(G, R, ld, err); break;
      default: k_mm_tc_grp<256, 4><<<grid, 128, smem, c->stream>>>(G, R, ld, err); break;
    }
    BIE_LAUNCH_CHECK(c, "k_mm_tc_grp");
    G.n = 0;
    return BIE_OK;
  };
  for (int s = 0; s < S; ++s) {
    const int cols = (S - s) * nrhs;
    const int nchunk = (cols + 255) / 256;
    const int padded = (nchunk - 1) * 256 + oz_nr(cols - (nchunk - 1) * 256);
    float* P;
    BIE_GET(c, float, names[s], (size_t)padded * ld, P);
    pr.P[s] = P;
    pr.ldP[s] = padded;
    CUtensorMap tA;
    const cuuint64_t gdA[2] = {(cuuint64_t)ld, (cuuint64_t)R}, gsA[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t bA[2] = {MM_KT, 128};
    if (enc(&tA, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, SA + (size_t)s * NN, gdA, gsA, bA, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ctx_fail(c, BIE_ERR_CUDA, "exact product: tensor map (A)");
    for (int g = 0; g < 5; ++g) grp[g].tA[s] = tA;
    for (int q = 0; q < nchunk; ++q) {
      const int c0 = q * 256, cn = std::min(256, cols - c0), NR = oz_nr(cn);
      CUtensorMap tX;
      const cuuint64_t gdX[2] = {(cuuint64_t)ld, (cuuint64_t)cn}, gsX[1] = {(cuuint64_t)ld * 2};
      const cuuint32_t bX[2] = {MM_KT, (cuuint32_t)NR};
      if (enc(&tX, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, XS + (size_t)c0 * ld, gdX, gsX, bX, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return ctx_fail(c, BIE_ERR_CUDA, "exact product: tensor map (X)");
      const int g = slot_of(NR);
      MmGroup& G = grp[g];
      G.tX[G.n] = tX;
      G.Y[G.n] = P + (size_t)c0 * ld;
      G.lvl[G.n] = s;
      if (++G.n == MM_GMAX) {
        bie_status r = flush(g);
        if (r != BIE_OK) return r;
      }
    }
  }
  for (int g = 4; g >= 0; --g) {
    bie_status r = flush(g);
    if (r != BIE_OK) return r;
  }
  k_oz_combine<<<(unsigned)(((long long)nrhs * R + 255) / 256), 256, 0, c->stream>>>(
      R, ld, nrhs, S, 1, pr, e, f, Y);
  BIE_LAUNCH_CHECK(c, "k_oz_combine");
  int herr = 0;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) return ctx_fail(c, BIE_ERR_TIMEOUT, "exact product: a pipeline wait timed out");
  return BIE_OK;
}

// Y[r][m] = sum_l A_ml X_rl / M_l + s_m X_rm with the full-accuracy storage
__global__ void k_oz_finish(int N, long long ld, int nrhs, const double* __restrict__ P,
                            const double* __restrict__ X, const float* __restrict__ sgn,
                            double* __restrict__ Y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nrhs * N) return;
  const int r = (int)(i / N);
  const int m = (int)(i - (long long)r * N);
  Y[i] = P[(size_t)r * ld + m] + (double)sgn[m] * X[i];
}

extern "C" bie_status bie_matmat_full(bie_ctx* c, int nrhs, const double* X_dev, double* Y_dev) {
  if (!c) return BIE_ERR_ARG;
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_matmat_full: not available on a row-partitioned context");
  BIE_NVTX("bie_matmat_full");
  if (!c->assembled) return ctx_fail(c, BIE_ERR_STATE, "bie_matmat_full: not assembled");
  if (c->transposed)
    return ctx_fail(c, BIE_ERR_STATE, "bie_matmat_full: storage holds the adjoint operator; assemble again");
  if (c->precision == BIE_FP64)
    return ctx_fail(c, BIE_ERR_STATE, "bie_matmat_full: needs the hi + lo storage of a refined scheme");
  if (c->ld > OZ_KMAX)
    return ctx_fail(c, BIE_ERR_ARG, "bie_matmat_full: at most 16384 unknowns");
  if (nrhs < 1 || nrhs > 64) return ctx_fail(c, BIE_ERR_ARG, "bie_matmat_full: 1 <= nrhs <= 64");
  if (!X_dev || !Y_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_matmat_full: null pointer");
  cudaSetDevice(c->device);
  double* P;
  BIE_GET(c, double, "oz_Y", (size_t)nrhs * c->ld, P);
  bie_status s = oz_product(c, 0, nrhs, X_dev, c->N, 1, OZ_S, P);
  if (s != BIE_OK) return s;
  bool oom = false;
  const float* sgn = (const float*)ctx_buf(c, "sgn", sizeof(float) * c->ld, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_matmat_full: node buffers");
  k_oz_finish<<<(unsigned)(((long long)nrhs * c->N + 255) / 256), 256, 0, c->stream>>>(
      c->N, c->ld, nrhs, P, X_dev, sgn, Y_dev);
  BIE_LAUNCH_CHECK(c, "k_oz_finish");
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return BIE_OK;
}

// ===========================================================================
// Several right-hand sides on one matrix: independent GMRES-IR solves in lock
// step (the GMRES-IR of a single solve, for each column), every Arnoldi step one tensor-core product
// for all columns.
//
// Per cycle: residuals r_r = D(b_r - A omega_r) with the full-accuracy operator
// for all columns at once: the exact-slice tensor-core product above (a
// multi-vector double-float GEMV over the hi + lo storage past 16384 unknowns);
// per column ||r||, convergence, v_0; then Arnoldi steps j: the columns
// v_j / M_l (scaled by min M_k, rounded to the storage type) go through the
// tensor-core product, a finishing kernel forms w = D(A v_j) and the first
// Gram-Schmidt dots, and the CGS2 kernels of the single solver run per column
// (grid.y = column).  A column whose cycle has converged skips its kernels;
// the host stops enqueuing steps when every column has.  U of every column
// comes from one multi-vector pass over the surface U-matrix.
// ===========================================================================
#include "gemv_dot.cuh"
#include "krylov.cuh"

struct MStat {
  int inner_done, outer_done, nonfinite, iters;
  int total_iters, cycles, converged, have_d;   // have_d: the last update moved x by dlast
  double rnorm, bnorm, inner_tol, resid_est;
  int qc[2];         // recycled columns in use: cycle c reads qc[c & 1]
};

#define M_RQ 32      // recycled columns kept at most per column
#define M_RK 16      // columns a cycle may add

struct MArgs {
  int N;
  long long ld;
  int m;
  int nrhs;
  int rowflip;
  float* V;          // [nrhs][m+1][ld]
  float* w;          // [nrhs][ld]
  double* r;         // [nrhs][ld]
  const double* b;   // [nrhs][ld]
  double* x;         // [nrhs][N]
  double* dlast;     // [nrhs][N]: the last update's increment of x
  double* H;         // [nrhs][(m+1) m]
  double* cs;        // [nrhs][m]
  double* sn;        // [nrhs][m]
  double* g;         // [nrhs][m+1]
  double* part1;     // [nrhs][m+2][BIE_PSTRIDE]
  double* part2;     // [nrhs][m+2][BIE_PSTRIDE]
  double* partn;     // [nrhs][BIE_NPART]
  MStat* st;         // device
  MStat* mirror;     // host-mapped
  const int* blk;
  const float* sgn;
  const double* wgt64;
  // right preconditioner P over the obstacles (see RightDefl): block sums of
  // the current v_j per column in part3[rr][k][slice], their means in mu[rr][j][k]
  int nobs;
  int obs_off[BIE_MAXB + 1];
  double obs_invM[BIE_MAXB];
  double* part3;     // [nrhs][BIE_MAXB][BIE_PSTRIDE]
  double* mu;        // [nrhs][m+1][BIE_MAXB]
  // recycled subspace per column across its cycles (GCRO-DR, as in the
  // single-column solver, in the classical-CGS2 form T V_k = C B + V_{k+1} H):
  // T U = C, C orthonormal, q = st[rr].qc[cycle & 1]
  int cycle;
  int recycle;       // 0: cycles add nothing (q stays 0)
  float* Cr;         // [nrhs][M_RQ][ld]
  float* Ur;         // [nrhs][M_RQ][ld]
  double* Bm;        // [nrhs][m][M_RQ]: C-part of Hessenberg column j
  double* c0;        // [nrhs][M_RQ]: C-part of the cycle's start vector
  double* umean;     // [nrhs][M_RQ][BIE_MAXB]: means of U's columns over the obstacles
  double* partc;     // [nrhs][M_RQ][BIE_PSTRIDE]: C_i^T r over the slices
};

__device__ __forceinline__ int mq_of(const MArgs& a, int rr) { return a.st[rr].qc[a.cycle & 1]; }
__device__ __forceinline__ float* mC(const MArgs& a, int rr, int i) {
  return a.Cr + ((size_t)rr * M_RQ + i) * a.ld;
}
__device__ __forceinline__ float* mU(const MArgs& a, int rr, int i) {
  return a.Ur + ((size_t)rr * M_RQ + i) * a.ld;
}

// this CTA's slice sums of v over each obstacle, for the next product
__device__ __forceinline__ void m_obstacle_sums(const MArgs& a, int rr, const float* v, int r0,
                                                int r1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < a.nobs; k += nw) {
    const int a0 = max(r0, a.obs_off[k]), a1 = min(r1, a.obs_off[k + 1]);
    double t = 0.0;
    for (int m = a0 + lane; m < a1; m += 32) t += (double)v[m];
    t = warp_sum(t);
    if (lane == 0) a.part3[((size_t)rr * BIE_MAXB + k) * BIE_PSTRIDE + blockIdx.x] = t;
  }
}

__device__ __forceinline__ float* mV(const MArgs& a, int r, int i) {
  return a.V + ((size_t)r * (a.m + 1) + i) * a.ld;
}

// basis vector i of column rr's cycle: C_i (i < q), V_{i-q}
__device__ __forceinline__ const float* mQ(const MArgs& a, int rr, int q, int i) {
  return i < q ? mC(a, rr, i) : mV(a, rr, i - q);
}

__device__ __forceinline__ void m_mirror(const MArgs& a, int r) {
  a.mirror[r] = a.st[r];
  __threadfence_system();
}

// r = D b (cycle 0)
__global__ void k_m_init_resid(MArgs a) {
  __shared__ double red[32];
  const int rr = blockIdx.y;
  int r0, r1;
  slice_of(a.N, r0, r1);
  double acc = 0.0;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
    double v = a.b[(size_t)rr * a.ld + m];
    if (a.rowflip && a.blk[m] == 0) v = -v;
    a.r[(size_t)rr * a.ld + m] = v;
    acc += v * v;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) a.partn[(size_t)rr * BIE_NPART + blockIdx.x] = acc;
}

// r = D(b - (sum_p ypart + s x)) for columns still refining; upd: the product
// was of the last increments d instead, and r <- r - D(sum_p ypart + s d) (r
// unchanged for a column whose last update did not move it)
__global__ void k_m_resid_finish(MArgs a, const double* __restrict__ ypart, int npanel, int upd) {
  __shared__ double red[32];
  const int rr = blockIdx.y;
  if (a.st[rr].outer_done) return;
  const bool use_d = upd && a.st[rr].have_d;
  const double* src = upd ? a.dlast : a.x;
  int r0, r1;
  slice_of(a.N, r0, r1);
  double acc = 0.0;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
    const bool flip = a.rowflip && a.blk[m] == 0;
    double o;
    if (upd && !use_d) {
      o = a.r[(size_t)rr * a.ld + m];
    } else {
      double y = 0.0;
      for (int p = 0; p < npanel; ++p) y += ypart[((size_t)p * a.nrhs + rr) * a.ld + m];
      y += (double)a.sgn[m] * src[(size_t)rr * a.N + m];
      const double ro = a.r[(size_t)rr * a.ld + m];
      o = (upd ? (flip ? -ro : ro) : a.b[(size_t)rr * a.ld + m]) - y;
      if (flip) o = -o;
    }
    a.r[(size_t)rr * a.ld + m] = o;
    acc += o * o;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) a.partn[(size_t)rr * BIE_NPART + blockIdx.x] = acc;
  const int q = mq_of(a, rr);
  if (q > 0) {   // C_i^T r over this slice (r written above by this CTA)
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const double* rc = a.r + (size_t)rr * a.ld;
    for (int i = warp; i < q; i += nw) {
      const float* ci = mC(a, rr, i);
      double t = 0.0;
      for (int m = r0 + lane; m < r1; m += 32) t += (double)ci[m] * rc[m];
      t = warp_sum(t);
      if (lane == 0) a.partc[((size_t)rr * M_RQ + i) * BIE_PSTRIDE + blockIdx.x] = t;
    }
  }
}

// ||r||, c_0 = C^T r / ||r||, and v_0 = (r / ||r|| - C c_0) / nu_0 with
// nu_0^2 = 1 - |c_0|^2 (the part of the start vector outside the recycled space)
__global__ void k_m_start(MArgs a, double rtol, double inner_tol, int first, int max_reached) {
  __shared__ double tot, s_nu0;
  __shared__ double sc[M_RQ];
  const int rr = blockIdx.y;
  MStat* S = a.st + rr;
  if (S->outer_done) return;
  const int q = mq_of(a, rr);
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int t = threadIdx.x; t < (int)gridDim.x; t += 32) s += a.partn[(size_t)rr * BIE_NPART + t];
    s = warp_sum(s);
    if (threadIdx.x == 0) tot = s;
  }
  if (q > 0) reduce_partials(a.partc + (size_t)rr * M_RQ * BIE_PSTRIDE, q, gridDim.x, sc);
  __syncthreads();
  const double rn = sqrt(tot);
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < q; ++i) t += (sc[i] / rn) * (sc[i] / rn);
    s_nu0 = sqrt(fmax(1.0 - t, 0.0));
  }
  __syncthreads();
  const double nu0 = s_nu0;
  const double bn = first ? rn : S->bnorm;
  const bool bad = !isfinite(rn);
  const bool conv = !bad && (rn <= rtol * bn || rn == 0.0);
  const bool done = bad || conv || max_reached;
  // r lies in the recycled space (to rounding): the correction is U c_0 alone
  const bool nokrylov = !done && !(nu0 > 1e-12);
  if (!done && !nokrylov) {
    const double inv = 1.0 / rn, inu = 1.0 / nu0;
    int r0, r1;
    slice_of(a.N, r0, r1);
    float* v0 = mV(a, rr, 0);
    for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
      double v = a.r[(size_t)rr * a.ld + m] * inv;
      for (int i = 0; i < q; ++i) v -= (sc[i] * inv) * (double)mC(a, rr, i)[m];
      v0[m] = (float)(v * inu);
    }
    __syncthreads();
    m_obstacle_sums(a, rr, v0, r0, r1);
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (first) S->bnorm = rn;
    S->rnorm = rn;
    S->nonfinite = bad ? 1 : 0;
    S->outer_done = done ? 1 : 0;
    S->converged = conv ? 1 : 0;
    S->inner_done = (done || nokrylov) ? 1 : 0;
    S->iters = 0;
    S->resid_est = 1.0;
    S->inner_tol = fmax(inner_tol, 0.5 * rtol * bn / fmax(rn, 1e-300));
    double* g = a.g + (size_t)rr * (a.m + 1);
    g[0] = nokrylov ? 0.0 : nu0;
    for (int i = 1; i <= a.m; ++i) g[i] = 0.0;
    for (int i = 0; i < q; ++i) a.c0[(size_t)rr * M_RQ + i] = sc[i] / rn;
    m_mirror(a, rr);
  }
}

// XT[rr][l] = v_j^rr[l] / M_l * mmin in the storage type (zero for finished or padding columns)
template <bool BF16>
__global__ void k_m_prep(MArgs a, int j, int NR, double mmin, void* __restrict__ XT) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)NR * a.ld) return;
  const int rr = (int)(i / a.ld);
  const int l = (int)(i - (long long)rr * a.ld);
  float v = 0.f;
  if (rr < a.nrhs && l < a.N && !a.st[rr].inner_done)
    v = (float)((double)mV(a, rr, j)[l] * a.wgt64[l] * mmin);
  if (BF16) ((__nv_bfloat16*)XT)[i] = __float2bfloat16_rn(v);
  else ((__half*)XT)[i] = __float2half_rn(v);
}

// this lane's share of a . b over the slice: FP32 runs of eight, the runs in FP64
__device__ __forceinline__ double m_lane_dot(const float* va, const float* vb, int r0, int r1,
                                             int lane) {
  double s = 0.0;
  float run = 0.f;
  int c = 0;
  for (int m = r0 + lane; m < r1; m += 32) {
    run = fmaf(va[m], vb[m], run);
    if (++c == 8) {
      s += (double)run;
      run = 0.f;
      c = 0;
    }
  }
  return s + (double)run;
}

// w = D(s v_j + (1/mmin) sum_ks Yp) (+ 3/2 mu_k on obstacle k's rows: A P v_j
// with A 1_k = -1_k) and part1[i][slice] = V_i . w (i <= j)
__global__ void k_m_finish_dots(MArgs a, int j, const float* __restrict__ Yp, int split, int NR,
                                float inv_mmin) {
  const int rr = blockIdx.y;
  if (a.st[rr].inner_done) return;
  __shared__ float s_xc[BIE_MAXB];
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < a.nobs) {   // means of v_j over the obstacles, in a fixed order
      const double* prow = a.part3 + ((size_t)rr * BIE_MAXB + warp) * BIE_PSTRIDE;
      double t = 0.0;
      for (int q = lane; q < (int)gridDim.x; q += 32) t += prow[q];
      t = warp_sum(t);
      const double mu = t * a.obs_invM[warp];
      if (lane == 0) {
        s_xc[warp] = (float)(1.5 * mu);
        if (blockIdx.x == 0) a.mu[((size_t)rr * (a.m + 1) + j) * BIE_MAXB + warp] = mu;
      }
    }
    __syncthreads();
  }
  int r0, r1;
  slice_of(a.N, r0, r1);
  const float* vj = mV(a, rr, j);
  float* w = a.w + (size_t)rr * a.ld;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
    float y = 0.f;
    for (int k = 0; k < split; ++k) y += Yp[((size_t)k * NR + rr) * a.ld + m];
    float v = fmaf(a.sgn[m], vj[m], y * inv_mmin);
    if (a.nobs > 0 && m >= a.obs_off[0]) {
      int k = 0;
      while (k + 1 < a.nobs && m >= a.obs_off[k + 1]) ++k;
      v += s_xc[k];
    }
    if (a.rowflip && a.blk[m] == 0) v = -v;
    w[m] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int q = mq_of(a, rr);
  double* p1 = a.part1 + (size_t)rr * (a.m + 2 + M_RQ) * BIE_PSTRIDE;
  for (int i = warp; i <= q + j; i += nw) {
    double s = m_lane_dot(mQ(a, rr, q, i), w, r0, r1, lane);
    s = warp_sum(s);
    if (lane == 0) p1[(size_t)i * BIE_PSTRIDE + blockIdx.x] = s;
  }
}

// h1 = sum part1; w' = w - Q h1; part2 = Q^T w' and ||w'||^2 (Q = [C, V_0..V_j])
__global__ void k_m_cgs2(MArgs a, int j) {
  const int rr = blockIdx.y;
  if (a.st[rr].inner_done) return;
  extern __shared__ double msh[];
  const int q = mq_of(a, rr), nd = q + j;
  const double* p1 = a.part1 + (size_t)rr * (a.m + 2 + M_RQ) * BIE_PSTRIDE;
  double* p2 = a.part2 + (size_t)rr * (a.m + 2 + M_RQ) * BIE_PSTRIDE;
  __shared__ float hf[M_RQ + 66];   // h1 in single precision, converted once per CTA
  reduce_partials(p1, nd + 1, gridDim.x, msh);
  __syncthreads();
  for (int i = threadIdx.x; i <= nd; i += blockDim.x) hf[i] = (float)msh[i];
  __syncthreads();
  int r0, r1;
  slice_of(a.N, r0, r1);
  float* w = a.w + (size_t)rr * a.ld;
  for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
    float acc = w[m];
    for (int i = 0; i <= nd; ++i) acc -= hf[i] * mQ(a, rr, q, i)[m];
    w[m] = acc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i <= nd + 1; i += nw) {
    double s = m_lane_dot(i <= nd ? mQ(a, rr, q, i) : w, w, r0, r1, lane);
    s = warp_sum(s);
    if (lane == 0) p2[(size_t)i * BIE_PSTRIDE + blockIdx.x] = s;
  }
}

// h2 = sum part2, beta, v_{j+1} = (w' - Q h2) / beta; CTA 0: the V-part of
// h1 + h2 is Hessenberg column j, its C-part column j of B; rotations, test
__global__ void k_m_cgs3(MArgs a, int j) {
  const int rr = blockIdx.y;
  MStat* S = a.st + rr;
  if (S->inner_done) return;
  extern __shared__ double msh[];
  const int q = mq_of(a, rr), nd = q + j;
  const double* p1 = a.part1 + (size_t)rr * (a.m + 2 + M_RQ) * BIE_PSTRIDE;
  const double* p2 = a.part2 + (size_t)rr * (a.m + 2 + M_RQ) * BIE_PSTRIDE;
  reduce_partials(p2, nd + 2, gridDim.x, msh);
  if (blockIdx.x == 0) reduce_partials(p1, nd + 1, gridDim.x, msh + (nd + 2));
  __syncthreads();
  __shared__ double s_beta;   // sqrt(||w'||^2 - ||h2||^2), one warp's sum for the CTA
  __shared__ float hf[M_RQ + 66], s_inv;   // h2 and 1/beta in single precision
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i <= nd; i += 32) t += msh[i] * msh[i];
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      const double b = sqrt(fmax(msh[nd + 1] - t, 0.0));
      s_beta = b;
      s_inv = (b > 1e-300 && isfinite(b)) ? (float)(1.0 / b) : 0.f;
    }
  } else {
    for (int i = threadIdx.x - 32; i <= nd; i += blockDim.x - 32) hf[i] = (float)msh[i];
  }
  __syncthreads();
  const double beta = s_beta;
  const bool breakdown = !(beta > 1e-300) || !isfinite(beta);
  if (!breakdown) {
    const float inv = s_inv;
    int r0, r1;
    slice_of(a.N, r0, r1);
    const float* w = a.w + (size_t)rr * a.ld;
    float* vn = mV(a, rr, j + 1);
    for (int m = r0 + threadIdx.x; m < r1; m += blockDim.x) {
      float acc = w[m];
      for (int i = 0; i <= nd; ++i) acc -= hf[i] * mQ(a, rr, q, i)[m];
      vn[m] = acc * inv;
    }
    if (a.nobs > 0) {
      __syncthreads();   // the slice of v_{j+1} is this CTA's
      m_obstacle_sums(a, rr, vn, r0, r1);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {   // one warp: Hessenberg column and rotations
    const int m = a.m;
    double* H = a.H + (size_t)rr * (m + 1) * m;
    double* cs = a.cs + (size_t)rr * m;
    double* sn = a.sn + (size_t)rr * m;
    double* g = a.g + (size_t)rr * (m + 1);
    double* Hj = H + (size_t)j * (m + 1);
    for (int i = threadIdx.x; i <= j; i += 32) Hj[i] = msh[nd + 2 + q + i] + msh[q + i];
    for (int l = threadIdx.x; l < q; l += 32)
      a.Bm[((size_t)rr * m + j) * M_RQ + l] = msh[nd + 2 + l] + msh[l];
    __syncwarp();
    const double uj = givens_apply_warp(Hj, cs, sn, j);
    if (threadIdx.x != 0) return;
    Hj[j] = uj;
    Hj[j + 1] = beta;
    const double rr2 = hypot(Hj[j], Hj[j + 1]);
    double c = 1.0, s = 0.0;
    if (rr2 > 0.0) {
      c = Hj[j] / rr2;
      s = Hj[j + 1] / rr2;
    }
    cs[j] = c;
    sn[j] = s;
    Hj[j] = rr2;
    Hj[j + 1] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    const double est = fabs(g[j + 1]);
    S->iters = j + 1;
    S->resid_est = est;
    const bool nf = !isfinite(est) || !isfinite(rr2);
    if (nf) S->nonfinite = 1;
    if (nf || breakdown || est <= S->inner_tol || j + 1 >= m) S->inner_done = 1;
    m_mirror(a, rr);
  }
}

// omega += ||r|| P (V y + U (c_0 - B y)) with R y = g; when the cycle's space
// fits, it joins the column's recycled one (C gains V_{k+1} G^T's first k
// columns, U gains (V_k - U B) R^-1, so that T U = C holds)
__global__ void k_m_update(MArgs a) {
  extern __shared__ double y[];   // m + 1, then c_0 - B y (M_RQ)
  const int rr = blockIdx.y;
  MStat* S = a.st + rr;
  const int k = S->iters;
  const int q = mq_of(a, rr);
  const bool act = !S->outer_done && !S->nonfinite;
  const int ext = (a.recycle && act && k >= 1 && k <= M_RK && q + k <= M_RQ) ? 1 : 0;
  const bool applied = act && !(k <= 0 && q == 0);   // else x (and dlast) stay as they are
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->qc[(a.cycle + 1) & 1] = q + (ext ? k : 0);
    S->have_d = applied ? 1 : 0;
  }
  if (!applied) return;
  const int m = a.m;
  const double* H = a.H + (size_t)rr * (m + 1) * m;
  const double* g = a.g + (size_t)rr * (m + 1);
  const double* Bm = a.Bm + (size_t)rr * m * M_RQ;
  double* tq = y + (m + 1);
  __shared__ double Ri[M_RK * M_RK];   // R^-1 (row i, column c)
  __shared__ double Mq[M_RQ * M_RK];   // -B R^-1
  __shared__ float RiF[M_RK * M_RK], MqF[M_RQ * M_RK];   // their single-precision copies
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = k - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1 + lane; l < k; l += 32) s += H[(size_t)l * (m + 1) + i] * y[l];
      s = warp_sum(s);
      if (lane == 0) y[i] = (g[i] - s) / H[(size_t)i * (m + 1) + i];
      __syncwarp();
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < q) {
    const int l = threadIdx.x;
    double t = a.c0[(size_t)rr * M_RQ + l];
    for (int i = 0; i < k; ++i) t -= Bm[(size_t)i * M_RQ + l] * y[i];
    tq[l] = t;
  }
  if (ext && (int)threadIdx.x < k) {   // column c of R^-1
    const int c = threadIdx.x;
    for (int i = 0; i < k; ++i) Ri[i * M_RK + c] = 0.0;
    for (int i = c; i >= 0; --i) {
      double t = i == c ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; ++l) t -= H[(size_t)l * (m + 1) + i] * Ri[l * M_RK + c];
      Ri[i * M_RK + c] = t / H[(size_t)i * (m + 1) + i];
    }
    for (int i = 0; i < k; ++i) RiF[i * M_RK + c] = (float)Ri[i * M_RK + c];
  }
  __syncthreads();
  if (ext)
    for (int e = threadIdx.x; e < q * k; e += blockDim.x) {
      const int l = e / k, c = e - l * k;
      double t = 0.0;
      for (int i = 0; i <= c; ++i) t -= Bm[(size_t)i * M_RQ + l] * Ri[i * M_RK + c];
      Mq[l * M_RK + c] = t;
      MqF[l * M_RK + c] = (float)t;
    }
  __shared__ double s_dm[BIE_MAXB];   // 3/2 of the correction's mean over each obstacle
  const double* mu = a.mu + (size_t)rr * (m + 1) * BIE_MAXB;
  double* um = a.umean + (size_t)rr * M_RQ * BIE_MAXB;
  if ((int)threadIdx.x < a.nobs) {
    double t = 0.0;
    for (int i = 0; i < k; ++i) t += y[i] * mu[(size_t)i * BIE_MAXB + threadIdx.x];
    for (int l = 0; l < q; ++l) t += tq[l] * um[(size_t)l * BIE_MAXB + threadIdx.x];
    s_dm[threadIdx.x] = 1.5 * t;
  }
  __syncthreads();
  if (ext && blockIdx.x == 0)   // means of the new U columns over the obstacles
    for (int e = threadIdx.x; e < a.nobs * k; e += blockDim.x) {
      const int o = e / k, c = e - o * k;
      double t = 0.0;
      for (int i = 0; i <= c; ++i) t += mu[(size_t)i * BIE_MAXB + o] * Ri[i * M_RK + c];
      for (int l = 0; l < q; ++l) t += um[(size_t)l * BIE_MAXB + o] * Mq[l * M_RK + c];
      um[(size_t)(q + c) * BIE_MAXB + o] = t;
    }
  const double scale = S->rnorm;
  const double* cs = a.cs + (size_t)rr * m;
  const double* sn = a.sn + (size_t)rr * m;
  // the row loop's coefficients in single precision, converted once per CTA
  __shared__ float yf[64], tqf[M_RQ], csf[64], snf[64];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    yf[i] = (float)y[i];
    csf[i] = (float)cs[i];
    snf[i] = (float)sn[i];
  }
  for (int l = threadIdx.x; l < q; l += blockDim.x) tqf[l] = (float)tq[l];
  __syncthreads();
  int r0, r1;
  slice_of(a.N, r0, r1);
  for (int mm = r0 + threadIdx.x; mm < r1; mm += blockDim.x) {
    // FP32 runs of eight terms, the runs summed in FP64 (the correction needs the
    // inner tolerance's accuracy; x accumulates in FP64)
    double acc = 0.0;
    for (int i0 = 0; i0 < k; i0 += 8) {
      float run = 0.f;
      for (int i = i0; i < min(i0 + 8, k); ++i) run = fmaf(yf[i], mV(a, rr, i)[mm], run);
      acc += (double)run;
    }
    for (int l0 = 0; l0 < q; l0 += 8) {
      float run = 0.f;
      for (int l = l0; l < min(l0 + 8, q); ++l) run = fmaf(tqf[l], mU(a, rr, l)[mm], run);
      acc += (double)run;
    }
    if (a.nobs > 0 && mm >= a.obs_off[0]) {
      int o = 0;
      while (o + 1 < a.nobs && mm >= a.obs_off[o + 1]) ++o;
      acc -= s_dm[o];
    }
    a.x[(size_t)rr * a.N + mm] += scale * acc;
    a.dlast[(size_t)rr * a.N + mm] = scale * acc;
    if (!ext) continue;
    // in single precision, the recycled pair's own precision
    float cur = mV(a, rr, 0)[mm];
    for (int i = 0; i < k; ++i) {
      const float ci = csf[i], si = snf[i];
      // v_k is not formed after a breakdown; its rotation then has s = 0
      const float nxt = (i + 1 < k || si != 0.f) ? mV(a, rr, i + 1)[mm] : 0.f;
      mC(a, rr, q + i)[mm] = ci * cur + si * nxt;
      cur = -si * cur + ci * nxt;
    }
    float tu[M_RK];
#pragma unroll
    for (int c = 0; c < M_RK; ++c) tu[c] = 0.f;
    for (int i = 0; i < k; ++i) {
      const float vi = mV(a, rr, i)[mm];
#pragma unroll
      for (int c = 0; c < M_RK; ++c)
        if (c >= i && c < k) tu[c] += RiF[i * M_RK + c] * vi;
    }
    for (int l = 0; l < q; ++l) {
      const float ul = mU(a, rr, l)[mm];
#pragma unroll
      for (int c = 0; c < M_RK; ++c)
        if (c < k) tu[c] += MqF[l * M_RK + c] * ul;
    }
#pragma unroll
    for (int c = 0; c < M_RK; ++c)
      if (c < k) mU(a, rr, q + c)[mm] = tu[c];
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->total_iters += k;
    S->cycles += 1;
    m_mirror(a, rr);
  }
}

// x (FP64, [nrhs][xstride]) -> x / M_l as double-float hi/lo [nrhs][ld], zero padded
__global__ void k_m_xdf(int N, long long ld, int nrhs, long long xstride, const double* __restrict__ x,
                        const double* __restrict__ wgt64, float* __restrict__ xh,
                        float* __restrict__ xl) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nrhs * ld) return;
  const int rr = (int)(i / ld);
  const int l = (int)(i - (long long)rr * ld);
  const double v = (l < N) ? x[(size_t)rr * xstride + l] * wgt64[l] : 0.0;
  const dfl d = df_from_double(v);
  xh[i] = d.hi;
  xl[i] = d.lo;
}

// Several vectors against the hi + lo storage in double-float: ypart[p][c][m]
// = sum_{l in panel p} (hi + lo)_ml (xh + xl)_cl for c < nc (<= 8) of the
// columns starting at c0; the matrix is read once per 8 columns.  Each lane
// keeps, per column, the running sum S of the leading products hi*xh (with an
// exact two-sum per step) and an FP32 sum E of every lower-order term: the
// rounding error of each product, hi*xl, lo*xh and the two-sum errors (lo*xl
// is below the precision).  S + E carries about 48 bits; the lanes combine
// their (S, E) pairs in double-float and lane c converts column c to FP64.
__device__ __forceinline__ void se_acc(float& S, float& E, float a, float b, float h, float l) {
  const float p = a * h;
  E = fmaf(a, l, E);
  E = fmaf(b, h, E);
  E += fmaf(a, h, -p);
  const float s = S + p;
  const float bb = s - S;
  E += (S - (s - bb)) + (p - bb);
  S = s;
}

#define MH_THREADS 512
__global__ void __launch_bounds__(MH_THREADS, 2)
    k_gemv_hilo_multi(const float* __restrict__ Ahi, const float* __restrict__ Alo, long long ld,
                      int rows, int panel, int nc, int c0, int ntot,
                      const float* __restrict__ xh, const float* __restrict__ xl,
                      double* __restrict__ ypart, int hi_only) {
  extern __shared__ __align__(16) float mhs[];   // [8][panel] hi, then [8][panel] lo
  const long long p0 = (long long)blockIdx.y * panel;
  const int pw = (int)min((long long)panel, ld - p0);
  float* sh = mhs;
  float* sl = mhs + 8 * panel;
  for (int i = threadIdx.x; i < 8 * pw; i += blockDim.x) {
    const int c = i / pw, l = i - c * pw;
    const bool ok = c < nc;
    sh[c * panel + l] = ok ? xh[(size_t)(c0 + c) * ld + p0 + l] : 0.f;
    sl[c * panel + l] = ok ? xl[(size_t)(c0 + c) * ld + p0 + l] : 0.f;
  }
  __syncthreads();
  const int nvec = pw / 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int GW = (blockDim.x >> 5) * gridDim.x;
  for (int m = warp * gridDim.x + blockIdx.x; m < rows; m += GW) {
    const float4* rh = reinterpret_cast<const float4*>(Ahi + (size_t)m * ld + p0);
    const float4* rl = reinterpret_cast<const float4*>(Alo + (size_t)m * ld + p0);
    float S[8], E[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) S[c] = E[c] = 0.f;
    for (int v = lane; v < nvec; v += 64) {
      const bool two = v + 32 < nvec;
      const float4 a0 = __ldcs(rh + v);
      const float4 b0 = hi_only ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldcs(rl + v);
      float4 a1 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = a1;
      if (two) {
        a1 = __ldcs(rh + v + 32);
        if (!hi_only) b1 = __ldcs(rl + v + 32);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c >= nc) break;
        const float4 h0 = *reinterpret_cast<const float4*>(sh + c * panel + 4 * v);
        const float4 l0 = *reinterpret_cast<const float4*>(sl + c * panel + 4 * v);
        se_acc(S[c], E[c], a0.x, b0.x, h0.x, l0.x);
        se_acc(S[c], E[c], a0.y, b0.y, h0.y, l0.y);
        se_acc(S[c], E[c], a0.z, b0.z, h0.z, l0.z);
        se_acc(S[c], E[c], a0.w, b0.w, h0.w, l0.w);
        if (two) {
          const float4 h1 = *reinterpret_cast<const float4*>(sh + c * panel + 4 * (v + 32));
          const float4 l1 = *reinterpret_cast<const float4*>(sl + c * panel + 4 * (v + 32));
          se_acc(S[c], E[c], a1.x, b1.x, h1.x, l1.x);
          se_acc(S[c], E[c], a1.y, b1.y, h1.y, l1.y);
          se_acc(S[c], E[c], a1.z, b1.z, h1.z, l1.z);
          se_acc(S[c], E[c], a1.w, b1.w, h1.w, l1.w);
        }
      }
    }
    // butterfly over the warp in double-float; every lane ends with the totals
    float th = 0.f, tl = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c >= nc) break;
      dfl t = df_two_sum(S[c], E[c]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const dfl u = {__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)};
        t = t + u;
      }
      if (lane == c) {
        th = t.hi;
        tl = t.lo;
      }
    }
    if (lane < nc) ypart[((size_t)blockIdx.y * ntot + c0 + lane) * ld + m] = (double)th + (double)tl;
  }
}

// xd = xh + xl (the double-float weights as FP64, exact)
__global__ void k_m_dfsum(long long n, const float* __restrict__ xh, const float* __restrict__ xl,
                          double* __restrict__ xd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) xd[i] = (double)xh[i] + (double)xl[i];
}

// U_c = (eq. d:phi:mv + sum_p ypart[p][c] - 1/2 H omega_0') / s_alpha for every column
__global__ void k_m_u_finish(int M0, long long ld, int nrhs, int npanel, FlowParams F,
                             const double* __restrict__ ypart, const double2* __restrict__ z64,
                             const double2* __restrict__ dz64, const float2* __restrict__ hw0,
                             double* __restrict__ U) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int rr = blockIdx.y;
  if (m >= M0) return;
  double y = 0.0;
  for (int p = 0; p < npanel; ++p) y += ypart[((size_t)p * nrhs + rr) * ld + m];
  const double h = df_to_double(dfl{hw0[(size_t)rr * M0 + m].x, hw0[(size_t)rr * M0 + m].y});
  const double2 zp = dz64[m];
  double asum = 0.0;
  for (int j = 2; j < F.nb; ++j) asum += F.a[j - 2];
  double mv = -(F.V1 + 0.5 * asum) * zp.y;
  const double2 zm = z64[m];
  for (int j = 2; j < F.nb; ++j) {
    const double ux = zm.x - F.zc[j - 2].x, uy = zm.y - F.zc[j - 2].y;
    double s, c;
    sincos(ux, &s, &c);
    const double e = exp(-uy);
    const double qr = e * c - 1.0, qi = e * s;
    const double n2 = qr * qr + qi * qi;
    const double hr = qi / n2, hi = 0.5 + qr / n2;
    mv += F.a[j - 2] * (hr * zp.x - hi * zp.y);
  }
  U[(size_t)rr * M0 + m] = (mv + y - 0.5 * h) / hypot(zp.x, zp.y);
}

// hi + lo product of `rows` rows of (Ahi, Alo) with the columns of (xh, xl)
static bie_status hilo_multi(bie_ctx* c, const float* Ahi, const float* Alo, int rows, int nrhs,
                             const float* xh, const float* xl, double* ypart, int panel,
                             int hi_only) {
  const size_t smem = sizeof(float) * 16 * (size_t)panel;
  BIE_CUDA_TRY(c, raise_smem_limit((const void*)k_gemv_hilo_multi, smem));
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  const int npanel = (int)((c->ld + panel - 1) / panel);
  for (int c0 = 0; c0 < nrhs; c0 += 8) {
    const int nc = std::min(8, nrhs - c0);
    k_gemv_hilo_multi<<<dim3(nsm, npanel), MH_THREADS, smem, c->stream>>>(
        Ahi, Alo, c->ld, rows, panel, nc, c0, nrhs, xh, xl, ypart, hi_only);
    BIE_LAUNCH_CHECK(c, "k_gemv_hilo_multi");
  }
  return BIE_OK;
}

bie_status solve_multi_run(bie_ctx* c, int nrhs, int rhs_kind, const double* rhs, double* X,
                           double* U, const bie_solve_opts* o, bie_solve_info* infos) {
  const int N = c->N, M0 = c->M[0], m = o->restart;
  const long long ld = c->ld;
  const bool bf = c->precision == BIE_BF16_IR;
  const int NR = nrhs <= 16 ? 16 : (nrhs <= 32 ? 32 : 64);
  // 1024-column panels: 64 KB of vectors in shared memory, two CTAs per SM
  const int panel = (int)std::min<long long>(1024, ld);
  const int npanel = (int)((ld + panel - 1) / panel);
  const size_t NN = (size_t)N * (size_t)ld, VN = (size_t)M0 * (size_t)ld;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return ctx_fail(c, BIE_ERR_CUDA, "bie_solve_multi: cuTensorMapEncodeTiled unavailable");
  MArgs a;
  memset(&a, 0, sizeof(a));
  a.N = N;
  a.ld = ld;
  a.m = m;
  a.nrhs = nrhs;
  a.rowflip = o->row_flip ? 1 : 0;
  a.x = X;
  BIE_GET(c, double, "ms_dlast", (size_t)nrhs * N, a.dlast);
  double *bbuf, *ypart, *ypu;
  float *xh, *xl, *Yp;
  float2* hw0;
  void* XT;
  MStat* st;
  BIE_GET(c, float, "ms_V", (size_t)nrhs * (m + 1) * ld, a.V);
  BIE_GET(c, float, "ms_w", (size_t)nrhs * ld, a.w);
  BIE_GET(c, double, "ms_r", (size_t)nrhs * ld, a.r);
  BIE_GET(c, double, "ms_b", (size_t)nrhs * ld, bbuf);
  a.b = bbuf;
  BIE_GET(c, double, "ms_H", (size_t)nrhs * (m + 1) * m, a.H);
  BIE_GET(c, double, "ms_cs", (size_t)nrhs * m, a.cs);
  BIE_GET(c, double, "ms_sn", (size_t)nrhs * m, a.sn);
  BIE_GET(c, double, "ms_g", (size_t)nrhs * (m + 1), a.g);
  BIE_GET(c, double, "ms_part1", (size_t)nrhs * (m + 2 + M_RQ) * BIE_PSTRIDE, a.part1);
  BIE_GET(c, double, "ms_part2", (size_t)nrhs * (m + 2 + M_RQ) * BIE_PSTRIDE, a.part2);
  BIE_GET(c, float, "ms_C", (size_t)nrhs * M_RQ * ld, a.Cr);
  BIE_GET(c, float, "ms_U", (size_t)nrhs * M_RQ * ld, a.Ur);
  BIE_GET(c, double, "ms_B", (size_t)nrhs * m * M_RQ, a.Bm);
  BIE_GET(c, double, "ms_c0", (size_t)nrhs * M_RQ, a.c0);
  BIE_GET(c, double, "ms_umean", (size_t)nrhs * M_RQ * BIE_MAXB, a.umean);
  BIE_GET(c, double, "ms_partc", (size_t)nrhs * M_RQ * BIE_PSTRIDE, a.partc);
  BIE_GET(c, double, "ms_partn", (size_t)nrhs * BIE_NPART, a.partn);
  BIE_GET(c, MStat, "ms_stat", nrhs, st);
  a.st = st;
  BIE_GET(c, float, "ms_xh", (size_t)nrhs * ld, xh);
  BIE_GET(c, float, "ms_xl", (size_t)nrhs * ld, xl);
  BIE_GET(c, double, "ms_ypart", (size_t)npanel * nrhs * ld, ypart);
  BIE_GET(c, double, "ms_ypu", (size_t)npanel * nrhs * ld, ypu);
  BIE_GET(c, float2, "ms_hw0", (size_t)nrhs * M0, hw0);
  BIE_GET(c, unsigned short, "ms_xt", (size_t)NR * ld, XT);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  const int nrb = (N + 127) / 128;
  int split = (3 * nsm + nrb - 1) / nrb;
  split = std::max(1, std::min(split, std::max(1, (int)(ld / MM_KT) / 8)));
  BIE_GET(c, float, "ms_yp", (size_t)split * NR * ld, Yp);
  int* err;
  BIE_GET(c, int, "ms_err", 1, err);
  bool oom = false;
  a.blk = (const int*)ctx_buf(c, "blk", sizeof(int) * ld, &oom);
  a.sgn = (const float*)ctx_buf(c, "sgn", sizeof(float) * ld, &oom);
  a.wgt64 = (const double*)ctx_buf(c, "wgt64", sizeof(double) * ld, &oom);
  // the inner solves on the operator of eq. AB:cor take the right
  // preconditioner over the obstacles (blocks 2 .. nb-1)
  const bool std_op = !c->transposed && c->variant == 0 && !c->asm_noE && !c->asm_vs;
  a.nobs = (std_op && c->nb > 2) ? c->nb - 2 : 0;
  for (int k = 0; k < a.nobs; ++k) {
    a.obs_off[k] = c->off[2 + k];
    a.obs_invM[k] = 1.0 / (double)c->M[2 + k];
  }
  a.obs_off[a.nobs] = a.nobs > 0 ? c->off[c->nb] : N;
  a.part3 = (double*)ctx_buf(c, "ms_part3", sizeof(double) * (size_t)nrhs * BIE_MAXB * BIE_PSTRIDE, &oom);
  a.mu = (double*)ctx_buf(c, "ms_mu", sizeof(double) * (size_t)nrhs * (m + 1) * BIE_MAXB, &oom);
  const float* Ahi = (const float*)ctx_buf(c, "A_hi", sizeof(float) * NN, &oom);
  const float* Alo = (const float*)ctx_buf(c, "A_lo", sizeof(float) * NN, &oom);
  void* A16 = ctx_buf(c, "A_16", 2 * NN, &oom);
  const float* Vhi = (const float*)ctx_buf(c, "V_hi", sizeof(float) * VN, &oom);
  const float* Vlo = (const float*)ctx_buf(c, "V_lo", sizeof(float) * VN, &oom);
  const double2* z64 = (const double2*)ctx_buf(c, "zeta", sizeof(double2) * N, &oom);
  const double2* dz64 = (const double2*)ctx_buf(c, "dzeta", sizeof(double2) * N, &oom);
  if (oom) return ctx_fail(c, BIE_ERR_OOM, "bie_solve_multi: buffers");
  // host-mapped mirror of the statuses
  if (!c->ms_mirror_host || c->ms_mirror_n < nrhs) {
    if (c->ms_mirror_host) cudaFreeHost(c->ms_mirror_host);
    c->ms_mirror_host = nullptr;
    BIE_CUDA_TRY(c, cudaHostAlloc(&c->ms_mirror_host, sizeof(MStat) * 64, cudaHostAllocMapped));
    c->ms_mirror_n = 64;
  }
  MStat* mirror_h = (MStat*)c->ms_mirror_host;
  BIE_CUDA_TRY(c, cudaHostGetDevicePointer((void**)&a.mirror, c->ms_mirror_host, 0));
  // tensor maps of the storage and the scaled columns
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
    return ctx_fail(c, BIE_ERR_CUDA, "bie_solve_multi: tensor map encoding failed");
  int mmin = c->M[0];
  for (int k = 0; k < c->nb; ++k) mmin = std::min(mmin, c->M[k]);
  // right-hand sides (eq. Awb from phi~, or given), zero initial guesses, statuses
  if (rhs_kind == BIE_RHS_PHIT) {
    bie_status s = rhs_run_many(c, nrhs, rhs, M0, bbuf, ld);
    if (s != BIE_OK) return s;
  } else {
    BIE_CUDA_TRY(c, cudaMemcpy2DAsync(bbuf, sizeof(double) * ld, rhs, sizeof(double) * N,
                                      sizeof(double) * N, nrhs, cudaMemcpyDeviceToDevice,
                                      c->stream));
  }
  BIE_CUDA_TRY(c, cudaMemsetAsync(X, 0, sizeof(double) * (size_t)nrhs * N, c->stream));
  BIE_CUDA_TRY(c, cudaMemsetAsync(st, 0, sizeof(MStat) * nrhs, c->stream));
  BIE_CUDA_TRY(c, cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  double inner_tol = o->inner_tol;
  // Up to 16 columns the recycled space pays (26 -> 21 steps, 4 cycles instead of
  // 5); with more, the per-column Gram-Schmidt work over the extra basis vectors
  // costs more than the saved products (64 columns: 22.5 -> 25.1 ms), so the
  // cycles restart from nothing and keep the looser tolerances that suit that.
  a.recycle = nrhs <= 16 ? 1 : 0;
  if (inner_tol <= 0.0) inner_tol = a.recycle ? 5e-4 : (bf ? 1e-2 : 2e-3);
  // row slices per column: about 4 CTAs per SM over all columns, at most BIE_NPART
  const int npx = std::max(8, std::min(BIE_NPART, (4 * nsm + nrhs - 1) / nrhs));
  const dim3 gv(npx, nrhs);
  const size_t sh_h = sizeof(double) * (2 * (m + M_RQ) + 8);
  // two step events, released on every return path
  struct StepEvents {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~StepEvents() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    }
  } evs;
  cudaEvent_t* ev = evs.e;
  BIE_CUDA_TRY(c, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
  BIE_CUDA_TRY(c, cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));

  auto step = [&](int j) -> bie_status {
    const unsigned gp = (unsigned)(((long long)NR * ld + 255) / 256);
    if (bf) k_m_prep<true><<<gp, 256, 0, c->stream>>>(a, j, NR, (double)mmin, XT);
    else k_m_prep<false><<<gp, 256, 0, c->stream>>>(a, j, NR, (double)mmin, XT);
    BIE_LAUNCH_CHECK(c, "k_m_prep");
    bie_status s;
    if (NR == 16) s = bf ? mm_launch<16, 6, true>(c, tA, tX, Yp, split, err) : mm_launch<16, 6, false>(c, tA, tX, Yp, split, err);
    else if (NR == 32) s = bf ? mm_launch<32, 6, true>(c, tA, tX, Yp, split, err) : mm_launch<32, 6, false>(c, tA, tX, Yp, split, err);
    else s = bf ? mm_launch<64, 5, true>(c, tA, tX, Yp, split, err) : mm_launch<64, 5, false>(c, tA, tX, Yp, split, err);
    if (s != BIE_OK) return s;
    k_m_finish_dots<<<gv, 256, 0, c->stream>>>(a, j, Yp, split, NR, 1.0f / (float)mmin);
    BIE_LAUNCH_CHECK(c, "k_m_finish_dots");
    k_m_cgs2<<<gv, 256, sh_h, c->stream>>>(a, j);
    BIE_LAUNCH_CHECK(c, "k_m_cgs2");
    k_m_cgs3<<<gv, 256, sh_h, c->stream>>>(a, j);
    BIE_LAUNCH_CHECK(c, "k_m_cgs3");
    BIE_CUDA_TRY(c, cudaEventRecord(ev[j & 1], c->stream));
    return BIE_OK;
  };
  bie_status s = BIE_OK;
  bool r_exact = false;   // every refining column's r is the full-accuracy residual of its x
  for (int cycle = 0;; ++cycle) {
    a.cycle = cycle;   // the recycled-column counts alternate by cycle parity
    if (cycle == 0) {
      k_m_init_resid<<<gv, 256, 0, c->stream>>>(a);
      BIE_LAUNCH_CHECK(c, "k_m_init_resid");
      r_exact = true;
    } else {
      // On the exact-slice path, once every refining column's residual is the
      // full-accuracy one of its x and small, the next ones are updated from
      // the last increments d, r - D A d, with just enough slices of A and d
      // (S slices err by about 2^(1 - 5 S) of the row scale): S from the largest
      // ||r|| / ||b||, so that 2^(1 - 5 S) ||r|| <= 6e-15 ||b|| (the rule of the
      // single solver).  Otherwise a direct product of x: the FP32 part (or 7 of
      // the 10 slices) while every refining column's residual is above 1e-4
      // ||b||.  An updated residual does not see the rounding of x at each
      // update (the slices' updates came within 7e-16 ||b|| of the true
      // residual); the double-float multi-vector path keeps direct products
      // (its updates drifted by 1e-15 ||b||).
      const bool oz = ld <= OZ_KMAX && nrhs >= OZ_MIN_RHS;
      int hi_only = 1;
      double worst = 0.0;   // largest ||r|| / ||b|| of the refining columns
      for (int rr = 0; rr < nrhs; ++rr) {
        if (mirror_h[rr].outer_done) continue;
        if (!(mirror_h[rr].rnorm > 1e-4 * mirror_h[rr].bnorm)) hi_only = 0;
        const double bn = mirror_h[rr].bnorm;
        worst = std::max(worst, bn > 0.0 ? mirror_h[rr].rnorm / bn : 0.0);
      }
      int supd = 0;   // slices of the update product (0: no update)
      if (oz && r_exact && o->rtol >= 1e-14) {
        int sneed = 1;
        while (sneed < OZ_S && std::ldexp(2.0, -5 * sneed) * worst > 6e-15) ++sneed;
        if (std::ldexp(2.0, -5 * sneed) * worst <= 6e-15 && sneed < OZ_S) supd = sneed;
      }
      if (supd > 0) {
        s = oz_product(c, 0, nrhs, a.dlast, N, 1, supd, ypart);
        if (s != BIE_OK) break;
        k_m_resid_finish<<<gv, 256, 0, c->stream>>>(a, ypart, 1, 1);
      } else if (oz) {
        // exact slices on the tensor cores; fewer slices (35 bits) while the
        // residuals are still large, all ten (50 bits) near the end
        s = oz_product(c, 0, nrhs, X, N, 1, hi_only ? 7 : OZ_S, ypart);
        if (s != BIE_OK) break;
        k_m_resid_finish<<<gv, 256, 0, c->stream>>>(a, ypart, 1, 0);
        r_exact = !hi_only;
      } else {
        k_m_xdf<<<(unsigned)(((long long)nrhs * ld + 255) / 256), 256, 0, c->stream>>>(
            N, ld, nrhs, N, X, a.wgt64, xh, xl);
        BIE_LAUNCH_CHECK(c, "k_m_xdf");
        s = hilo_multi(c, Ahi, Alo, N, nrhs, xh, xl, ypart, panel, hi_only);
        if (s != BIE_OK) break;
        k_m_resid_finish<<<gv, 256, 0, c->stream>>>(a, ypart, npanel, 0);
        r_exact = !hi_only;
      }
      BIE_LAUNCH_CHECK(c, "k_m_resid_finish");
    }
    k_m_start<<<gv, 256, 0, c->stream>>>(a, o->rtol, inner_tol, cycle == 0 ? 1 : 0,
                                         cycle >= o->max_cycles ? 1 : 0);
    BIE_LAUNCH_CHECK(c, "k_m_start");
    BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    bool any = false;
    for (int rr = 0; rr < nrhs; ++rr) any = any || !mirror_h[rr].outer_done;
    if (!any) break;
    // Arnoldi steps, one step ahead of the host's convergence check
    s = step(0);
    if (s != BIE_OK) break;
    for (int j = 1; j < m; ++j) {
      s = step(j);
      if (s != BIE_OK) break;
      BIE_CUDA_TRY(c, cudaEventSynchronize(ev[(j - 1) & 1]));
      bool running = false;
      for (int rr = 0; rr < nrhs; ++rr) running = running || !mirror_h[rr].inner_done;
      if (!running) break;
    }
    if (s != BIE_OK) break;
    k_m_update<<<gv, 256, sizeof(double) * (m + 1 + M_RQ), c->stream>>>(a);
    BIE_LAUNCH_CHECK(c, "k_m_update");
  }
  if (s != BIE_OK) return s;
  // U of every column: DFT weights of all columns, one multi-vector pass over the U-matrix
  if (U) {
    s = velocity_weights(c, nrhs, X, xh, xl, hw0);
    if (s != BIE_OK) return s;
    int np = npanel;
    if (ld <= OZ_KMAX && nrhs >= OZ_MIN_RHS) {   // the U-matrix by exact slices
      double* xd;
      BIE_GET(c, double, "ms_xd", (size_t)nrhs * ld, xd);
      k_m_dfsum<<<(unsigned)(((long long)nrhs * ld + 255) / 256), 256, 0, c->stream>>>(
          (long long)nrhs * ld, xh, xl, xd);
      BIE_LAUNCH_CHECK(c, "k_m_dfsum");
      s = oz_product(c, 1, nrhs, xd, ld, 0, OZ_S, ypu);
      np = 1;
    } else {
      s = hilo_multi(c, Vhi, Vlo, M0, nrhs, xh, xl, ypu, panel, 0);
    }
    if (s != BIE_OK) return s;
    const FlowParams F = make_flow(c);
    k_m_u_finish<<<dim3((M0 + 255) / 256, nrhs), 256, 0, c->stream>>>(M0, ld, nrhs, np, F, ypu,
                                                                      z64, dz64, hw0, U);
    BIE_LAUNCH_CHECK(c, "k_m_u_finish");
  }
  int herr = 0;
  BIE_CUDA_TRY(c, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  BIE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) return ctx_fail(c, BIE_ERR_TIMEOUT, "bie_solve_multi: a pipeline wait timed out");
  bie_status worst = BIE_OK;
  for (int rr = 0; rr < nrhs; ++rr) {
    const MStat& S = mirror_h[rr];
    if (infos) {
      infos[rr].iters = S.total_iters;
      infos[rr].cycles = S.cycles;
      infos[rr].converged = S.converged;
      infos[rr].rel_resid = S.bnorm > 0 ? S.rnorm / S.bnorm : S.rnorm;
    }
    if (S.nonfinite) worst = BIE_ERR_NAN;
    else if (!S.converged && worst == BIE_OK) worst = BIE_ERR_NOCONV;
  }
  if (worst == BIE_ERR_NAN) return ctx_fail(c, worst, "bie_solve_multi: non-finite residual");
  if (worst == BIE_ERR_NOCONV) return ctx_fail(c, worst, "bie_solve_multi: a column missed rtol");
  return BIE_OK;
}

extern "C" bie_status bie_solve_multi(bie_ctx* c, int nrhs, int rhs_kind, const double* rhs_dev,
                                      double* omega_dev, double* U_dev, const bie_solve_opts* opts,
                                      bie_solve_info* infos) {
  BIE_NVTX("bie_solve_multi");
  if (!c) return BIE_ERR_ARG;
  if (c && c->part_n > 1)
    return ctx_fail(c, BIE_ERR_STATE, "bie_solve_multi: not available on a row-partitioned context");
  if (!c->assembled || !c->have_flow)
    return ctx_fail(c, BIE_ERR_STATE, "bie_solve_multi: assemble and set_flow first");
  if (c->transposed)
    return ctx_fail(c, BIE_ERR_STATE, "bie_solve_multi: storage holds the adjoint operator; assemble again");
  if (c->precision != BIE_FP16_IR && c->precision != BIE_BF16_IR)
    return ctx_fail(c, BIE_ERR_STATE, "bie_solve_multi: needs FP16 or BF16 storage");
  if (nrhs < 1 || nrhs > 64) return ctx_fail(c, BIE_ERR_ARG, "bie_solve_multi: 1 <= nrhs <= 64");
  if (rhs_kind != BIE_RHS_PHIT && rhs_kind != BIE_RHS_B)
    return ctx_fail(c, BIE_ERR_ARG, "bie_solve_multi: unknown rhs_kind");
  if (c->variant != 0 && (rhs_kind != BIE_RHS_B || U_dev))
    return ctx_fail(c, BIE_ERR_STATE,
                    "bie_solve_multi: the App. B operator takes raw right-hand sides and no U");
  if (!rhs_dev || !omega_dev) return ctx_fail(c, BIE_ERR_ARG, "bie_solve_multi: null pointer");
  bie_solve_opts o;
  bie_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.restart < 1 || o.restart > 63 || o.max_cycles < 1)
    return ctx_fail(c, BIE_ERR_ARG, "bie_solve_multi: bad options (restart <= 63)");
  cudaSetDevice(c->device);
  return solve_multi_run(c, nrhs, rhs_kind, rhs_dev, omega_dev, U_dev, &o, infos);
}
