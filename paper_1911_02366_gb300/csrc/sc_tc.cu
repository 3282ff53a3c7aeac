// TF32 tensor-core batched GEMM on sm_103a (tcgen05 + TMEM) for the element Schur
// products of the mixed arm: Y = A_ii^-1 A_ib,ee and S_ee -= A_bi,ee Y (Sec. 2.2,
// eq. StaticCondBlock; Sec. 3.2 "matrix-matrix multiplications").
//
// One CTA (one warpgroup, 128 threads) computes a 128 x BN tile of one batch entry:
//   * K is walked in chunks of 32; every thread stages its share of the A (128 x 32) and
//     B (BN x 32) chunks into shared memory in the K-major, no-swizzle core-matrix layout
//     (8 rows x 16 bytes per core matrix; K-adjacent core matrices 128 B apart, 8-row
//     groups 1024 B apart), zero-filling out-of-range rows and columns;
//   * one thread issues four tcgen05.mma.kind::tf32 (M = 128, N = BN, K = 8) into a TMEM
//     accumulator and commits them to an mbarrier; every wait is bounded and a time-out
//     raises an error status instead of spinning;
//   * the four warps read their 32 TMEM lanes (rows) with tcgen05.ld and write
//     C = alpha * acc + beta * C.
#include <cstdint>

#include "sc_internal.cuh"

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 32;
constexpr long long kWaitLimit = 1LL << 22;  // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (M/N-direction) byte offsets, fixed version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) of a (rows x 32) chunk in the core-matrix layout.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return static_cast<uint32_t>(((row >> 3) * 8 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

template <int BN>
__global__ void __launch_bounds__(128, 1) k_gemm_tf32(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                      long long sA, int lda, const float* __restrict__ B,
                                                      long long sB, int ldb, float beta, float* __restrict__ C,
                                                      long long sC, int ldc, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* As = smem;                     // TC_BM x TC_BK, 16 KB
  unsigned char* Bs = smem + TC_BM * TC_BK * 4; // BN x TC_BK
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_err;
  const int z = blockIdx.z;
  A += z * sA;
  B += z * sB;
  C += z * sC;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&tmem_base_s, BN);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_err = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = idesc_tf32(TC_BM, BN);
  uint32_t phase = 0;
  for (int k0 = 0; k0 < K; k0 += TC_BK) {
    for (int t = tid; t < TC_BM * TC_BK; t += 128) {
      const int r = t / TC_BK, kk = t % TC_BK;
      const int gr = m0 + r, gk = k0 + kk;
      const float v = (gr < M && gk < K) ? A[(long long)gr * lda + gk] : 0.0f;
      *reinterpret_cast<float*>(As + core_off(r, kk)) = v;
    }
    for (int t = tid; t < BN * TC_BK; t += 128) {
      const int kk = t / BN, n = t % BN;
      const int gk = k0 + kk, gn = n0 + n;
      const float v = (gk < K && gn < N) ? B[(long long)gk * ldb + gn] : 0.0f;
      *reinterpret_cast<float*>(Bs + core_off(n, kk)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint64_t ad = smem_desc(smem_u32(As) + kk * 256, 128, 1024);
        const uint64_t bd = smem_desc(smem_u32(Bs) + kk * 256, 128, 1024);
        mma_tf32(tmem, ad, bd, idesc, (k0 > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&mbar);
      long long it = 0;
      while (!mbar_try_wait(&mbar, phase)) {
        if (++it > kWaitLimit) { s_err = 1; break; }
      }
    }
    phase ^= 1u;
    __syncthreads();
    if (s_err) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_err) {
    const int row = m0 + warp * 32 + lane;
    for (int cc = 0; cc < BN; cc += 8) {
      float v[8];
      tmem_ld8(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(cc), v);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int col = n0 + cc + j;
          if (col < N) {
            float* cp = C + (long long)row * ldc + col;
            *cp = (beta == 0.0f) ? alpha * v[j] : fmaf(alpha, v[j], beta * *cp);
          }
        }
      }
    }
  }
  if (s_err && tid == 0) {
    // give the tensor-core work already issued a second bounded chance to finish
    // before its accumulator columns are released
    long long it = 0;
    while (!mbar_try_wait(&mbar, phase ^ 1u) && ++it < kWaitLimit) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
  if (s_err && tid == 0) atomicCAS(status, -1, 1 << 30);
}

constexpr int TC_BN = 256;
constexpr size_t kTcSmem = (size_t)TC_BM * TC_BK * 4 + (size_t)TC_BN * TC_BK * 4;

}  // namespace

namespace sc {

// C = alpha A B + beta C for `batch` row-major FP32 problems, TF32 tensor cores.
cudaError_t gemm_tf32(cudaStream_t stream, int M, int N, int K, float alpha, const float* A, long long sA, int lda,
                      const float* B, long long sB, int ldb, float beta, float* C, long long sC, int ldc, int batch,
                      int* status) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  // 1 CTA per SM at most: each holds TC_BN TMEM columns and ~96 KB of shared memory.
  const size_t smem = 96 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tf32<TC_BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  static_assert(kTcSmem <= 96 * 1024, "tile does not fit");
  dim3 grid((N + TC_BN - 1) / TC_BN, (M + TC_BM - 1) / TC_BM, batch);
  k_gemm_tf32<TC_BN><<<grid, 128, smem, stream>>>(M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc, status);
  return cudaGetLastError();
}

}  // namespace sc

extern "C" sc_status sc_gemm_tf32(int batch, int M, int N, int K, float alpha, const float* A, long long strideA,
                                  int lda, const float* B, long long strideB, int ldb, float beta, float* C,
                                  long long strideC, int ldc, void* cuda_stream) {
  if (!A || !B || !C || batch < 0 || M < 0 || N < 0 || K < 0 || lda < K || ldb < N || ldc < N) return SC_ERR_ARG;
  if (batch == 0 || M == 0 || N == 0) return SC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* status = nullptr;
  // The status word lives in a small pinned host allocation so that no device memory is
  // allocated per call.
  if (cudaHostAlloc(reinterpret_cast<void**>(&status), sizeof(int), cudaHostAllocMapped) != cudaSuccess)
    return SC_ERR_CUDA;
  *status = -1;
  int* dstatus = nullptr;
  cudaError_t e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&dstatus), status, 0);
  if (e == cudaSuccess)
    e = sc::gemm_tf32(st, M, N, K, alpha, A, strideA, lda, B, strideB, ldb, beta, C, strideC, ldc, batch, dstatus);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const int flag = *status;
  cudaFreeHost(status);
  if (e != cudaSuccess) return SC_ERR_CUDA;
  if (flag != -1) return SC_ERR_CUDA;
  return SC_OK;
}
