// TF32 tensor-core batched GEMM on sm_103a (tcgen05 + TMEM): the dense per-element
// products of the mixed arm, Y = A_ii^-1 A_ib,ee and S_ee -= A_bi,ee Y (Sec. 2.2,
// eq. StaticCondBlock; Sec. 3.2 "matrix-matrix multiplications"), and the trailing
// updates A22 -= L21 U12 of the blocked LU of S_ee.
//
// One CTA (one warpgroup, 128 threads) computes a 128 x BN tile of one batch entry:
//   * K is walked in chunks of 32.  Every thread loads its share of the next A (128 x 32)
//     and B (BN x 32) chunks into registers while the tensor cores work on the current
//     chunk, then stores them into the other of two shared-memory buffers in the K-major,
//     no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), transposing on
//     the way where the source has the tile rows contiguous, and zero-filling rows and
//     columns beyond the matrix;
//   * one thread issues four tcgen05.mma.kind::tf32 (M = 128, N = BN, K = 8) into a TMEM
//     accumulator and commits them to the buffer's mbarrier; every wait is bounded and a
//     time-out raises an error status instead of spinning;
//   * the four warps read their 32 TMEM lanes (rows) with tcgen05.ld and write
//     C = alpha * acc + beta * C.
#include <algorithm>
#include <cstdint>
#include <type_traits>

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

// Eight consecutive accumulator columns of this thread's TMEM lane, without the wait:
// the registers are valid only after tmem_wait_ld.
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t r[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
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

// Tile layout in shared memory (K-major, no swizzle): element (row, k) of a
// (rows x TC_BK) chunk sits in the 8 x 16-byte core matrix (row / 8, k / 4).  Core
// matrices adjacent in K are TC_LBO bytes apart and 8-row groups TC_SBO bytes apart; the
// 16-byte gap between K-neighbours (144 instead of 128) spreads the transposing stores
// below over twice as many banks.
constexpr int TC_LBO = 144;
constexpr int TC_SBO = (TC_BK / 4) * TC_LBO;  // 1152
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return static_cast<uint32_t>((row >> 3) * TC_SBO + (k >> 2) * TC_LBO + (row & 7) * 16 + (k & 3) * 4);
}

// Staging of one (R x TC_BK) operand chunk into registers and then shared memory.
//   MN = false: the source has K contiguous (element (r, k) at src[r * ld + k]); one
//       float4 holds 4 consecutive k of one row and lands as one 16-byte core row.
//   MN = true: the source has the tile rows contiguous (element (r, k) at
//       src[k * ld + r]); one float4 holds 4 consecutive rows of one k and is written as
//       4 scalars (a transpose on the way into shared memory).
// Slots are numbered so that each warp reads 64 contiguous bytes per source row and its
// shared-memory stores hit distinct banks (MN = false) or at most 2-way conflicts.
template <int R, bool MN>
struct Stager {
  static constexpr int kSlots = R * TC_BK / 4;
  static constexpr int kPer = (kSlots + 127) / 128;
  float4 v[kPer];
  __device__ __forceinline__ static void slot_rc(int t, int& r, int& k) {
    const int lane = t & 31, w = t >> 5;
    if (!MN) {
      r = (w >> 1) * 8 + (lane & 7);
      k = ((lane >> 3) + 4 * (w & 1)) * 4;
    } else {
      k = (lane & 7) + 8 * (w & 3);
      r = ((lane >> 3) + 4 * (w >> 2)) * 4;
    }
  }
  // rows: valid tile rows (rows beyond are zero); kv: valid k of this chunk.
  __device__ __forceinline__ void load(const float* __restrict__ src, int ld, int rows, int kv, bool vec, int tid) {
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int t = tid + 128 * s;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (t < kSlots) {
        int r, k;
        slot_rc(t, r, k);
        if (!MN) {
          if (r < rows) {
            const float* p = src + (long long)r * ld + k;
            if (vec && k + 3 < kv) {
              x = __ldg(reinterpret_cast<const float4*>(p));
            } else {
              if (k < kv) x.x = __ldg(p);
              if (k + 1 < kv) x.y = __ldg(p + 1);
              if (k + 2 < kv) x.z = __ldg(p + 2);
              if (k + 3 < kv) x.w = __ldg(p + 3);
            }
          }
        } else {
          if (k < kv) {
            const float* p = src + (long long)k * ld + r;
            if (vec && r + 3 < rows) {
              x = __ldg(reinterpret_cast<const float4*>(p));
            } else {
              if (r < rows) x.x = __ldg(p);
              if (r + 1 < rows) x.y = __ldg(p + 1);
              if (r + 2 < rows) x.z = __ldg(p + 2);
              if (r + 3 < rows) x.w = __ldg(p + 3);
            }
          }
        }
      }
      v[s] = x;
    }
  }
  __device__ __forceinline__ void store(unsigned char* tile, int tid) const {
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int t = tid + 128 * s;
      if (t < kSlots) {
        int r, k;
        slot_rc(t, r, k);
        if (!MN) {
          *reinterpret_cast<float4*>(tile + core_off(r, k)) = v[s];
        } else {
          *reinterpret_cast<float*>(tile + core_off(r + 0, k)) = v[s].x;
          *reinterpret_cast<float*>(tile + core_off(r + 1, k)) = v[s].y;
          *reinterpret_cast<float*>(tile + core_off(r + 2, k)) = v[s].z;
          *reinterpret_cast<float*>(tile + core_off(r + 3, k)) = v[s].w;
        }
      }
    }
  }
};

constexpr int TC_TMEM_COLS = 256;
// TMEM columns of a 128 x BN accumulator: a power of two of at least 32
constexpr uint32_t tmem_cols_for(int bn) { return bn <= 32 ? 32u : bn <= 64 ? 64u : bn <= 128 ? 128u : 256u; }
constexpr int TC_EG = 4;  // 8-column chunks per epilogue group
template <int BN>
constexpr size_t tc_stage_bytes() {
  return (size_t)(TC_BM / 8) * TC_SBO + (size_t)(BN / 8) * TC_SBO;
}

// flags: bit 0 A rows may be read as float4, bit 1 the same for B, bit 2 for C.
// TA: A is stored K x M (op(A) = A^T); TB: B is stored N x K (op(B) = B^T).
template <int BN, bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm_tf32(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                   long long sA, int lda, const float* __restrict__ B, long long sB,
                                                   int ldb, float beta, float* __restrict__ C, long long sC, int ldc,
                                                   int flags, int* __restrict__ status,
                                                   const float* const* __restrict__ Ap,
                                                   const float* const* __restrict__ Bp, float* const* __restrict__ Cp) {
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= TC_TMEM_COLS, "M = 128 needs N % 16 == 0 and N <= 256");
  constexpr uint32_t kTmemCols = tmem_cols_for(BN);
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr size_t kA = (size_t)(TC_BM / 8) * TC_SBO, kStage = tc_stage_bytes<BN>();
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int s_err;
  const int z = blockIdx.z;
  if (Ap) {  // per-entry block addresses (batched condensation of several systems)
    A = Ap[z];
    B = Bp[z];
    C = Cp[z];
  } else {
    A += z * sA;
    B += z * sB;
    C += z * sC;
  }
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool vecA = flags & 1, vecB = flags & 2, vecC = flags & 4;
  const float* Ab = TA ? A + m0 : A + (long long)m0 * lda;
  const float* Bb = TB ? B + (long long)n0 * ldb : B + n0;
  const int mrows = min(TC_BM, M - m0), nrows = min(BN, N - n0);
  if (warp == 0) tmem_alloc(&tmem_base_s, kTmemCols);
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_err = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = idesc_tf32(TC_BM, BN);
  const int nk = (K + TC_BK - 1) / TC_BK;
  Stager<TC_BM, TA> sa;
  Stager<BN, !TB> sb;
  {
    const int kv = min(TC_BK, K);
    sa.load(Ab, lda, mrows, kv, vecA, tid);
    sb.load(Bb, ldb, nrows, kv, vecB, tid);
  }
  int issued = 0;  // chunks whose MMAs were committed
  for (int kc = 0; kc < nk; ++kc) {
    const int buf = kc & 1;
    unsigned char* As = smem + buf * kStage;
    unsigned char* Bs = As + kA;
    if (kc >= 2) {
      // the MMAs of chunk kc - 2 read this buffer: wait for their commit
      if (tid == 0) {
        long long it = 0;
        while (!mbar_try_wait(&mbar[buf], ((kc - 2) >> 1) & 1)) {
          if (++it > kWaitLimit) { s_err = 1; break; }
        }
      }
      __syncthreads();
      if (s_err) break;
    }
    sa.store(As, tid);
    sb.store(Bs, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_BK / 8; ++kk) {
        const uint64_t ad = smem_desc(smem_u32(As) + kk * 2 * TC_LBO, TC_LBO, TC_SBO);
        const uint64_t bd = smem_desc(smem_u32(Bs) + kk * 2 * TC_LBO, TC_LBO, TC_SBO);
        mma_tf32(tmem, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&mbar[buf]);
    }
    issued = kc + 1;
    if (kc + 1 < nk) {
      const int k0 = (kc + 1) * TC_BK, kv = min(TC_BK, K - k0);
      sa.load(TA ? Ab + (long long)k0 * lda : Ab + k0, lda, mrows, kv, vecA, tid);
      sb.load(TB ? Bb + k0 : Bb + (long long)k0 * ldb, ldb, nrows, kv, vecB, tid);
    }
  }
  if (tid == 0 && !s_err) {
    // the last commit arrives after every MMA issued before it has completed
    const int last = issued - 1;
    long long it = 0;
    while (!mbar_try_wait(&mbar[last & 1], (last >> 1) & 1)) {
      if (++it > kWaitLimit) { s_err = 1; break; }
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_err) {
    const int row = warp * 32 + lane;
    float* crow = C + (long long)(m0 + row) * ldc + n0;
    // groups of TC_EG 8-column chunks: the C loads of a group are issued together, then
    // its TMEM loads with one wait, so that each thread has TC_EG x 32 bytes in flight
#pragma unroll 1
    for (int cg = 0; cg < BN; cg += 8 * TC_EG) {
      float4 cl[TC_EG][2];
#pragma unroll
      for (int g = 0; g < TC_EG; ++g) {
        const int cc = cg + 8 * g;
        cl[g][0] = cl[g][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (beta != 0.0f && vecC && row < mrows && cc + 8 <= nrows) {
          cl[g][0] = *reinterpret_cast<const float4*>(crow + cc);
          cl[g][1] = *reinterpret_cast<const float4*>(crow + cc + 4);
        }
      }
      uint32_t r[TC_EG][8];
#pragma unroll
      for (int g = 0; g < TC_EG; ++g)
        tmem_ld8_async(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(cg + 8 * g), r[g]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int g = 0; g < TC_EG; ++g)
#pragma unroll
        for (int i = 0; i < 8; ++i) asm volatile("" : "+r"(r[g][i]));  // no use moves above the wait
#pragma unroll
      for (int g = 0; g < TC_EG; ++g) {
        const int cc = cg + 8 * g;
        if (row >= mrows || cc >= nrows) continue;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[g][i]);
        if (vecC && cc + 8 <= nrows) {
          float4 lo = cl[g][0], hi = cl[g][1];
          lo.x = fmaf(alpha, v[0], beta * lo.x);
          lo.y = fmaf(alpha, v[1], beta * lo.y);
          lo.z = fmaf(alpha, v[2], beta * lo.z);
          lo.w = fmaf(alpha, v[3], beta * lo.w);
          hi.x = fmaf(alpha, v[4], beta * hi.x);
          hi.y = fmaf(alpha, v[5], beta * hi.y);
          hi.z = fmaf(alpha, v[6], beta * hi.z);
          hi.w = fmaf(alpha, v[7], beta * hi.w);
          *reinterpret_cast<float4*>(crow + cc) = lo;
          *reinterpret_cast<float4*>(crow + cc + 4) = hi;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if (cc + j < nrows) {
              float* cp = crow + cc + j;
              *cp = (beta == 0.0f) ? alpha * v[j] : fmaf(alpha, v[j], beta * *cp);
            }
          }
        }
      }
    }
  }
  if (s_err && tid == 0) {
    // give the tensor-core work already committed a bounded chance to finish before its
    // accumulator columns are released
    for (int c = (issued >= 2 ? issued - 2 : 0); c < issued; ++c) {
      long long it = 0;
      while (!mbar_try_wait(&mbar[c & 1], (c >> 1) & 1) && ++it < kWaitLimit) {
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
  if (s_err && tid == 0) atomicCAS(status, -1, SC_TC_TIMEOUT);
}

template <int BN, bool TA, bool TB>
cudaError_t launch_tf32(cudaStream_t stream, int M, int N, int K, float alpha, const float* A, long long sA, int lda,
                        const float* B, long long sB, int ldb, float beta, float* C, long long sC, int ldc, int batch,
                        int flags, int* status, const float* const* Ap = nullptr, const float* const* Bp = nullptr,
                        float* const* Cp = nullptr) {
  constexpr size_t smem2 = 2 * tc_stage_bytes<BN>();
  static_assert(2 * (smem2 + 1024) <= 228 * 1024, "two CTAs per SM must fit");
  // K within one 32-wide chunk (the LU trailing updates): one staging buffer.  The request
  // is padded so that no more CTAs share an SM than its 512 TMEM columns hold, and none
  // waits in tcgen05.alloc.
  constexpr int kMaxCtas = 512 / (int)tmem_cols_for(BN);
  constexpr size_t kSmemSM = 228 * 1024, kMinSmem = kSmemSM / (kMaxCtas + 1) - 1024 + 16;
  const size_t smem = std::max(K <= TC_BK ? tc_stage_bytes<BN>() : smem2, kMinSmem);
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tf32<BN, TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((N + BN - 1) / BN, (M + TC_BM - 1) / TC_BM, batch);
  k_gemm_tf32<BN, TA, TB><<<grid, 128, smem, stream>>>(M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc, flags,
                                                       status, Ap, Bp, Cp);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_tf32_t(cudaStream_t stream, int M, int N, int K, float alpha, const float* A, long long sA,
                          int lda, bool ta, const float* B, long long sB, int ldb, bool tb, float beta, float* C,
                          long long sC, int ldc, int batch, int flags, int* status) {
  if (!ta && !tb)
    return launch_tf32<BN, false, false>(stream, M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc, batch,
                                         flags, status);
  if (!ta && tb)
    return launch_tf32<BN, false, true>(stream, M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc, batch,
                                        flags, status);
  if (ta && !tb)
    return launch_tf32<BN, true, false>(stream, M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc, batch,
                                        flags, status);
  return launch_tf32<BN, true, true>(stream, M, N, K, alpha, A, sA, lda, B, sB, ldb, beta, C, sC, ldc, batch, flags,
                                     status);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

namespace sc {

// C = alpha op(A) op(B) + beta C for `batch` row-major FP32 problems on the TF32 tensor
// cores.  op(A) is M x K (A stored M x K, or K x M when ta); op(B) is K x N (B stored
// K x N, or N x K when tb).
cudaError_t gemm_tf32(cudaStream_t stream, int M, int N, int K, float alpha, const float* A, long long sA, int lda,
                      bool ta, const float* B, long long sB, int ldb, bool tb, float beta, float* C, long long sC,
                      int ldc, int batch, int* status) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  // float4 access needs 16-byte aligned rows in every batch entry
  const bool vA = aligned16(A) && lda % 4 == 0 && sA % 4 == 0;
  const bool vB = aligned16(B) && ldb % 4 == 0 && sB % 4 == 0;
  const bool vC = aligned16(C) && ldc % 4 == 0 && sC % 4 == 0;
  const int flags = (vA ? 1 : 0) | (vB ? 2 : 0) | (vC ? 4 : 0);
  if (N <= 64)
    return launch_tf32_t<64>(stream, M, N, K, alpha, A, sA, lda, ta, B, sB, ldb, tb, beta, C, sC, ldc, batch, flags,
                             status);
  if (K <= TC_BK)  // rank-32 updates: 128-wide tiles, one staging buffer, four CTAs per SM
    return launch_tf32_t<128>(stream, M, N, K, alpha, A, sA, lda, ta, B, sB, ldb, tb, beta, C, sC, ldc, batch, flags,
                              status);
  if (N <= 144)
    return launch_tf32_t<144>(stream, M, N, K, alpha, A, sA, lda, ta, B, sB, ldb, tb, beta, C, sC, ldc, batch, flags,
                              status);
  return launch_tf32_t<256>(stream, M, N, K, alpha, A, sA, lda, ta, B, sB, ldb, tb, beta, C, sC, ldc, batch, flags,
                            status);
}

// Pointer-table form: entry z multiplies Ap[z], Bp[z] into Cp[z] (row-major, the given
// leading dimensions; rows are read as float4 when the leading dimensions are multiples
// of 4, which holds for every condensation block), N-tile width bn in {64, 144, 256}.
cudaError_t gemm_tf32_ptrs(cudaStream_t stream, int M, int N, int K, float alpha, const float* const* Ap, int lda,
                           bool ta, const float* const* Bp, int ldb, bool tb, float beta, float* const* Cp, int ldc,
                           int batch, int bn, int* status) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  const int flags = (lda % 4 == 0 ? 1 : 0) | (ldb % 4 == 0 ? 2 : 0) | (ldc % 4 == 0 ? 4 : 0);
  const float* A0 = nullptr;
  const float* B0 = nullptr;
  float* C0 = nullptr;
  auto go = [&](auto bnc) -> cudaError_t {
    constexpr int BNC = decltype(bnc)::value;
    if (!ta && !tb)
      return launch_tf32<BNC, false, false>(stream, M, N, K, alpha, A0, 0, lda, B0, 0, ldb, beta, C0, 0, ldc, batch,
                                            flags, status, Ap, Bp, Cp);
    if (!ta && tb)
      return launch_tf32<BNC, false, true>(stream, M, N, K, alpha, A0, 0, lda, B0, 0, ldb, beta, C0, 0, ldc, batch,
                                           flags, status, Ap, Bp, Cp);
    if (ta && !tb)
      return launch_tf32<BNC, true, false>(stream, M, N, K, alpha, A0, 0, lda, B0, 0, ldb, beta, C0, 0, ldc, batch,
                                           flags, status, Ap, Bp, Cp);
    return launch_tf32<BNC, true, true>(stream, M, N, K, alpha, A0, 0, lda, B0, 0, ldb, beta, C0, 0, ldc, batch, flags,
                                        status, Ap, Bp, Cp);
  };
  if (bn == 64) return go(std::integral_constant<int, 64>{});
  if (bn == 144) return go(std::integral_constant<int, 144>{});
  return go(std::integral_constant<int, 256>{});
}

}  // namespace sc

extern "C" sc_status sc_gemm_tf32(int batch, int M, int N, int K, float alpha, const float* A, long long strideA,
                                  int lda, int transA, const float* B, long long strideB, int ldb, int transB,
                                  float beta, float* C, long long strideC, int ldc, void* cuda_stream) {
  if (!A || !B || !C || batch < 0 || M < 0 || N < 0 || K < 0) return SC_ERR_ARG;
  if (lda < (transA ? M : K) || ldb < (transB ? K : N) || ldc < N) return SC_ERR_ARG;
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
    e = sc::gemm_tf32(st, M, N, K, alpha, A, strideA, lda, transA != 0, B, strideB, ldb, transB != 0, beta, C,
                      strideC, ldc, batch, dstatus);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const int flag = *status;
  cudaFreeHost(status);
  if (e != cudaSuccess) return SC_ERR_CUDA;
  if (flag != -1) return SC_ERR_CUDA;
  return SC_OK;
}
