// Batched dense linear algebra on the element blocks of the condensation
// (Sec. 3.2, "Analysis and Implementation": dense A_ii blocks inverted element by
// element, Schur products by matrix-matrix multiplication).
//
//   k_gj_inv    A_ii^-1 by Gauss-Jordan elimination with partial pivoting, one block
//               per CTA held in shared memory.
//   k_gemm      C = alpha A B + beta C for a batch of row-major blocks (SIMT, 64x64
//               tiles, 4x4 register micro-tiles).
//   k_lu        right-looking blocked LU with partial pivoting of a batch of blocks
//               in global memory (32-column panels factorised in shared memory).
//   k_solve_prep  partitioned inverses of the LU factors in the solve layout (below).
//   k_lu_solve    z = (P^T L U)^-1 v for every element, one warp per element, one lane
//                 per row of each 32-row block.
#include <cuda_fp16.h>

#include <type_traits>

#include "sc_internal.cuh"

namespace {

template <class T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// Warp argmax of |v| (ties: smallest index).
__device__ __forceinline__ void warp_argmax(double& v, int& idx) {
  for (int off = 16; off > 0; off >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, v, off);
    int oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
}

// A_ii^-1 of one block by one CTA (shared memory: n (n+1) + n values and n pivots).
template <class T>
__device__ void gj_inv_body(int n, const T* __restrict__ Ae, int lda, T* __restrict__ Oe, int ldo,
                            int* __restrict__ status, int e) {
  extern __shared__ unsigned char smem_raw[];
  const int ld = n + 1;
  T* M = reinterpret_cast<T*>(smem_raw);
  T* colk = M + (size_t)n * ld;
  int* piv = reinterpret_cast<int*>(colk + n);
  __shared__ int s_p;
  __shared__ int s_bad;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t % n;
    M[i * ld + j] = Ae[(long long)i * lda + j];
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0; int bi = k;
      for (int i = k + threadIdx.x; i < n; i += 32) {
        const double v = (double)tabs(M[i * ld + k]);
        if (v > best) { best = v; bi = i; }
      }
      warp_argmax(best, bi);
      if (threadIdx.x == 0) {
        s_p = bi;
        piv[k] = bi;
        if (!(best > 0.0)) s_bad = 1;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        T t = M[k * ld + j]; M[k * ld + j] = M[p * ld + j]; M[p * ld + j] = t;
      }
    __syncthreads();
    const T pinv = s_bad ? T(0) : T(1) / M[k * ld + k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = M[i * ld + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) M[k * ld + j] = (j == k) ? pinv : M[k * ld + j] * pinv;
    __syncthreads();
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int i = t / n, j = t % n;
      if (i == k) continue;
      const T f = colk[i];
      if (j == k) M[i * ld + j] = -f * pinv;
      else M[i * ld + j] -= f * M[k * ld + j];
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T t = M[i * ld + k]; M[i * ld + k] = M[i * ld + p]; M[i * ld + p] = t;
      }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) Oe[(long long)(t / n) * ldo + (t % n)] = M[(t / n) * ld + (t % n)];
  if (threadIdx.x == 0 && s_bad) atomicCAS(status, -1, e);
  __syncthreads();
}

// A_ii^-1 of one FP32 block of order n <= 136 by one CTA of 256 threads with the block held
// in registers: thread (warp w, lane l) owns rows w + 8 r (r < 17) and columns l + 32 c
// (c < 5).  Partial pivoting is implicit: step k takes as pivot row p_k the unused row with
// the largest |M[., k]| and eliminates in place without moving rows, which is Gauss-Jordan
// on B = P A (row k of B = row p_k of A) with B^-1 left in physical row p_k.  Since
// A^-1 = B^-1 P, the result is A^-1[i][p_k] = M[p_i][k], applied while staging the output.
// The rows are equilibrated first (D A with d_i = 1 / max_j |a_ij|, then A^-1 = (D A)^-1 D):
// the Jacobian's rows span three orders of magnitude, and unscaled FP32 Gauss-Jordan loses
// about two digits against an LU-based inverse on these blocks.
constexpr int GJR_R = 17, GJR_C = 5, GJR_N = 8 * GJR_R, GJR_LDS = GJR_N + 1;
static_assert(GJR_N == sc::kGjRegRows, "register Gauss-Jordan bound");
// dynamic shared memory the one-CTA Gauss-Jordan may take (227 KB less its static part)
constexpr size_t kGjSmemMax = 227 * 1024 - 64;

__device__ void gj_inv_reg_body(int n, const float* __restrict__ Ae, int lda, float* __restrict__ Oe, int ldo,
                                int* __restrict__ status, int e) {
  extern __shared__ unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);  // [GJR_N][GJR_LDS] output staging
  __shared__ float colk[2][GJR_N];                // column k of the current matrix
  __shared__ float rowk[32 * GJR_C];              // pivot row before scaling
  __shared__ int pk[GJR_N], invp[GJR_N];          // step -> pivot row, pivot row -> step
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  __shared__ float dsc[GJR_N];                    // row equilibration: d_i = 1 / max_j |a_ij|
  float M[GJR_R][GJR_C];
#pragma unroll
  for (int r = 0; r < GJR_R; ++r) {
    float mx = 0.f;
#pragma unroll
    for (int c = 0; c < GJR_C; ++c) {
      const int i = ty + 8 * r, j = tx + 32 * c;
      M[r][c] = (i < n && j < n) ? Ae[(long long)i * lda + j] : 0.f;
      mx = fmaxf(mx, fabsf(M[r][c]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const float d = mx > 0.f ? 1.f / mx : 1.f;
#pragma unroll
    for (int c = 0; c < GJR_C; ++c) M[r][c] *= d;
    if (tx == 0) dsc[ty + 8 * r] = d;
  }
  if (tx == 0) {
#pragma unroll
    for (int r = 0; r < GJR_R; ++r) colk[0][ty + 8 * r] = M[r][0];
  }
  unsigned used = 0;  // bit t: row tx + 32 t is a pivot row already, or padding
#pragma unroll
  for (int t = 0; t < GJR_C; ++t)
    if (tx + 32 * t >= n) used |= 1u << t;
  bool bad = false;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const float* ck = colk[k & 1];
    // pivot search, repeated by every warp on the same data: key = (|v| bits + 1, -row),
    // so NaN ranks above every number and ties go to the smallest row
    unsigned long long key = 0ull;
#pragma unroll
    for (int t = 0; t < GJR_C; ++t) {
      const int i = tx + 32 * t;
      if (!((used >> t) & 1u)) {
        const unsigned long long kv = ((unsigned long long)(__float_as_uint(fabsf(ck[i])) + 1u) << 32) |
                                      (unsigned)(0x7fffffff - i);
        key = kv > key ? kv : key;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, off);
      key = o > key ? o : key;
    }
    const int p = 0x7fffffff - (int)(unsigned)(key & 0xffffffffull);
    const float piv = ck[p];
    const bool ok = fabsf(piv) > 0.f;
    bad |= !ok;
    const float pinv = ok ? 1.f / piv : 0.f;
    if (tx == (p & 31)) used |= 1u << (p >> 5);
    if (threadIdx.x == 0) { pk[k] = p; invp[p] = k; }
    if (ty == (p & 7)) {
      const int pr = p >> 3;
#pragma unroll
      for (int r = 0; r < GJR_R; ++r)
        if (r == pr) {
#pragma unroll
          for (int c = 0; c < GJR_C; ++c) rowk[tx + 32 * c] = M[r][c];
        }
    }
    __syncthreads();
    float rk[GJR_C];
#pragma unroll
    for (int c = 0; c < GJR_C; ++c) rk[c] = rowk[tx + 32 * c];
    const int k1 = k + 1, nx = k1 & 31, nc = k1 >> 5;
    float* cn = colk[k1 & 1];
#pragma unroll
    for (int r = 0; r < GJR_R; ++r) {
      const int i = ty + 8 * r;
      const float f = ck[i] * pinv;
      const bool isp = i == p;
#pragma unroll
      for (int c = 0; c < GJR_C; ++c) {
        const bool isk = tx + 32 * c == k;
        const float m = M[r][c];
        const float v = isp ? (isk ? pinv : m * pinv) : (isk ? -f : fmaf(-f, rk[c], m));
        M[r][c] = v;
        if (c == nc && tx == nx) cn[i] = v;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < GJR_R; ++r)
#pragma unroll
    for (int c = 0; c < GJR_C; ++c) {
      const int i = ty + 8 * r, j = tx + 32 * c;
      if (i < n && j < n) S[invp[i] * GJR_LDS + pk[j]] = M[r][c];
    }
  __syncthreads();
  for (int i = ty; i < n; i += 8)
    for (int j = tx; j < n; j += 32) Oe[(long long)i * ldo + j] = S[i * GJR_LDS + j] * dsc[j];
  if (threadIdx.x == 0 && bad) atomicCAS(status, -1, e);
}

__global__ void __launch_bounds__(256, 2) k_gj_inv_reg(int n, const float* __restrict__ A, long long strideA,
                                                       int lda, float* __restrict__ Ainv, long long strideO,
                                                       int ldo, int* __restrict__ status) {
  const int e = blockIdx.x;
  gj_inv_reg_body(n, A + (long long)e * strideA, lda, Ainv + (long long)e * strideO, ldo, status, e);
}

template <class T>
__global__ void k_gj_inv(int n, const T* __restrict__ A, long long strideA, int lda,
                         T* __restrict__ Ainv, long long strideO, int ldo, int* __restrict__ status) {
  const int e = blockIdx.x;
  gj_inv_body<T>(n, A + (long long)e * strideA, lda, Ainv + (long long)e * strideO, ldo, status, e);
}

// ---- grouped kernels of the batched condensation: one CTA per CondItem ----------------
__global__ void __launch_bounds__(256, 2) k_gj_inv_reg_grouped(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.x];
  gj_inv_reg_body(it.ni, it.Aown, it.lda, it.Ainv, it.ldi, it.status, it.e);
}

__global__ void k_copy_bb_grouped(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.x];
  const float* src = it.Aown + (size_t)it.ni * it.lda + it.cb0;
  for (int t = threadIdx.x; t < it.nb * it.nb; t += blockDim.x) {
    const int i = t / it.nb, j = t % it.nb;
    it.See[(size_t)i * it.lds + j] = src[(size_t)i * it.lda + j];
  }
}

// C = alpha * A * B + beta * C, all row-major, one batch entry per blockIdx.z.
template <class T>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, T alpha,
                                              const T* __restrict__ A, long long sA, int lda,
                                              const T* __restrict__ B, long long sB, int ldb, T beta,
                                              T* __restrict__ C, long long sC, int ldc) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  const int z = blockIdx.z;
  A += (long long)z * sA; B += (long long)z * sB; C += (long long)z * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += 256) {
      const int r = t / BK, c = t % BK;
      const int gr = m0 + r, gc = k0 + c;
      As[c][r] = (gr < M && gc < K) ? A[(long long)gr * lda + gc] : T(0);
    }
    for (int t = threadIdx.x; t < BK * BN; t += 256) {
      const int r = t / BN, c = t % BN;
      const int gr = k0 + r, gc = n0 + c;
      Bs[r][c] = (gr < K && gc < N) ? B[(long long)gr * ldb + gc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = m0 + ty + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = n0 + tx + 16 * j;
      if (gc >= N) continue;
      T* cp = C + (long long)gr * ldc + gc;
      *cp = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *cp;
    }
  }
}

// Copy a sub-block (rows x cols) of a batch of row-major matrices.
template <class T>
__global__ void k_copy_block(int rows, int cols, const T* __restrict__ src, long long sS, int lds,
                             T* __restrict__ dst, long long sD, int ldd) {
  const int z = blockIdx.y;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rows * cols; t += gridDim.x * blockDim.x) {
    const int i = t / cols, j = t % cols;
    dst[(long long)z * sD + (long long)i * ldd + j] = src[(long long)z * sS + (long long)i * lds + j];
  }
}

constexpr int PW = 32;  // LU panel width

// One panel step of the right-looking LU with partial pivoting (rows first index of the
// largest |a|): factor columns k0 .. k0+bw-1 of rows k0 .. n-1 in shared memory, apply
// the panel's row interchanges to the columns outside it, and form U12 = L11^-1 A12.
// P: shared panel buffer [n][PW+1].  Returns with all threads synchronised.
template <class T>
__device__ void lu_panel(int n, int k0, T* __restrict__ Mx, int lda, int* __restrict__ piv, T* P, int* s_p,
                         int* s_bad) {
  constexpr int pld = PW + 1;
  const int bw = min(PW, n - k0), rows = n - k0;
  for (int t = threadIdx.x; t < rows * bw; t += blockDim.x) {
    const int i = t / bw, c = t % bw;
    P[i * pld + c] = Mx[(long long)(k0 + i) * lda + k0 + c];
  }
  __syncthreads();
  for (int c = 0; c < bw; ++c) {
    if (threadIdx.x < 32) {
      double best = -1.0; int bi = c;
      for (int i = c + threadIdx.x; i < rows; i += 32) {
        const double v = (double)tabs(P[i * pld + c]);
        if (v > best) { best = v; bi = i; }
      }
      warp_argmax(best, bi);
      if (threadIdx.x == 0) {
        *s_p = bi;
        piv[k0 + c] = k0 + bi;
        if (!(best > 0.0)) *s_bad = 1;
      }
    }
    __syncthreads();
    const int pr = *s_p;
    if (pr != c)
      for (int j = threadIdx.x; j < bw; j += blockDim.x) {
        T t = P[c * pld + j]; P[c * pld + j] = P[pr * pld + j]; P[pr * pld + j] = t;
      }
    __syncthreads();
    const T d = P[c * pld + c];
    const T dinv = (d == T(0)) ? T(0) : T(1) / d;
    for (int i = c + 1 + threadIdx.x; i < rows; i += blockDim.x) P[i * pld + c] *= dinv;
    __syncthreads();
    const int w = bw - c - 1;
    if (w > 0)
      for (int t = threadIdx.x; t < (rows - c - 1) * w; t += blockDim.x) {
        const int i = c + 1 + t / w, j = c + 1 + t % w;
        P[i * pld + j] -= P[i * pld + c] * P[c * pld + j];
      }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < rows * bw; t += blockDim.x) {
    const int i = t / bw, c = t % bw;
    Mx[(long long)(k0 + i) * lda + k0 + c] = P[i * pld + c];
  }
  // row interchanges of this panel applied to the columns outside it
  for (int c = 0; c < bw; ++c) {
    const int r1 = k0 + c, r2 = piv[k0 + c];
    if (r2 != r1)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (j >= k0 && j < k0 + bw) continue;
        T t = Mx[(long long)r1 * lda + j]; Mx[(long long)r1 * lda + j] = Mx[(long long)r2 * lda + j];
        Mx[(long long)r2 * lda + j] = t;
      }
    __syncthreads();
  }
  if (n - k0 - bw > 0) {
    // U12 = L11^-1 A12, one column per thread
    for (int j = k0 + bw + threadIdx.x; j < n; j += blockDim.x) {
      T col[PW];
      for (int c = 0; c < bw; ++c) col[c] = Mx[(long long)(k0 + c) * lda + j];
      for (int c = 0; c < bw; ++c)
        for (int i = c + 1; i < bw; ++i) col[i] -= P[i * pld + c] * col[c];
      for (int c = 0; c < bw; ++c) Mx[(long long)(k0 + c) * lda + j] = col[c];
    }
  }
  __syncthreads();
}

// Whole LU of one element block per CTA: panel steps with the trailing update
// A22 -= L21 U12 done by the same CTA in 4 x 4 register tiles.
template <class T>
__global__ void __launch_bounds__(256) k_lu(int n, T* __restrict__ A, long long stride, int lda,
                                            int* __restrict__ piv_all, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);  // panel [n][PW+1]
  constexpr int pld = PW + 1;
  __shared__ int s_p;
  __shared__ int s_bad;
  const int e = blockIdx.x;
  T* Mx = A + (long long)e * stride;
  int* piv = piv_all + (long long)e * n;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += PW) {
    lu_panel<T>(n, k0, Mx, lda, piv, P, &s_p, &s_bad);
    const int bw = min(PW, n - k0), rest = n - k0 - bw;
    if (rest > 0) {
      // A22 -= L21 U12, 4x4 register tiles
      const int tr = (rest + 3) / 4, tcn = (rest + 3) / 4;
      for (int t = threadIdx.x; t < tr * tcn; t += blockDim.x) {
        const int bi = (t / tcn) * 4, bj = (t % tcn) * 4;
        T acc[4][4];
        for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        for (int c = 0; c < bw; ++c) {
          T l[4], u[4];
          for (int a = 0; a < 4; ++a) l[a] = (bi + a < rest) ? P[(bw + bi + a) * pld + c] : T(0);
          for (int b = 0; b < 4; ++b)
            u[b] = (bj + b < rest) ? Mx[(long long)(k0 + c) * lda + k0 + bw + bj + b] : T(0);
          for (int a = 0; a < 4; ++a) for (int b = 0; b < 4; ++b) acc[a][b] = fma(l[a], u[b], acc[a][b]);
        }
        for (int a = 0; a < 4; ++a) {
          if (bi + a >= rest) continue;
          for (int b = 0; b < 4; ++b) {
            if (bj + b >= rest) continue;
            Mx[(long long)(k0 + bw + bi + a) * lda + k0 + bw + bj + b] -= acc[a][b];
          }
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_bad) atomicCAS(status, -1, e);
}

// One panel step for every element (the trailing update is a separate batched GEMM).
template <class T>
__global__ void __launch_bounds__(256) k_lu_panel(int n, int k0, T* __restrict__ A, long long stride, int lda,
                                                  int* __restrict__ piv_all, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_p;
  __shared__ int s_bad;
  const int e = blockIdx.x;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  lu_panel<T>(n, k0, A + (long long)e * stride, lda, piv_all + (long long)e * n, P, &s_p, &s_bad);
  if (threadIdx.x == 0 && s_bad) atomicCAS(status, -1, e);
}

// The same panel step of an FP32 block with n - k0 <= NW R rows, held in registers: lane l
// is panel column l, warp w of NW holds panel rows w + NW r (r < R).  Pivoting is implicit (the
// pivot rows p_c are marked, nothing moves during the 32 eliminations); the pivot order is
// then turned into the interchange sequence that row-by-row partial pivoting records
// (piv[k0 + c] = k0 + position swapped with c), the panel is written in its final row
// order, and one thread per column outside the panel applies the interchanges to its
// column in registers and, right of the panel, forms U12 = L11^-1 A12 there.
// Two shapes: 8 warps x 62 rows (496, n_b up to N = 4) and 16 warps x 69 rows (1104, N = 5, 6).
constexpr int LPR_R = 62, LPR_ROWS = 8 * LPR_R;
constexpr int LPR2_W = 16, LPR2_R = 69, LPR2_ROWS = LPR2_W * LPR2_R;

template <int NW, int R>
__device__ void lu_panel_reg_body(int n, int k0, float* __restrict__ Mx, int lda, int* __restrict__ piv,
                                  int* __restrict__ status, int e) {
  constexpr int ROWS = NW * R, NT = (ROWS + 31) / 32, ND = (R + 63) / 64;
  static_assert(NT <= 64, "pivot-search mask");
  __shared__ float colk[2][ROWS];  // column c of the current panel
  __shared__ float rowk[PW];           // pivot row
  __shared__ float L11[PW][PW + 1];    // unit lower triangle of the factored panel, final order
  __shared__ int pk[PW], ipv[PW], xl[PW];
  __shared__ int at[ROWS], where_[ROWS];  // position -> physical row, inverse
  __shared__ int s_nx;
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int bw = min(PW, n - k0), rows = n - k0;
  float M[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = w + NW * r;
    M[r] = (i < rows && l < bw) ? Mx[(long long)(k0 + i) * lda + k0 + l] : 0.f;
  }
  if (l == 0) {
#pragma unroll
    for (int r = 0; r < R; ++r) colk[0][w + NW * r] = M[r];
  }
  for (int i = threadIdx.x; i < ROWS; i += blockDim.x) { at[i] = i; where_[i] = i; }
  if (threadIdx.x == 0) s_nx = 0;
  unsigned long long sel = 0;  // bit t: search row l + 32 t is a pivot row already, or past the panel
#pragma unroll
  for (int t = 0; t < NT; ++t)
    if (l + 32 * t >= rows) sel |= 1ull << t;
  unsigned long long done[ND];  // bit r: row w + NW r is a pivot row already, or past the panel
#pragma unroll
  for (int q = 0; q < ND; ++q) done[q] = 0ull;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (w + NW * r >= rows) done[r >> 6] |= 1ull << (r & 63);
  bool bad = false;
  __syncthreads();
  for (int c = 0; c < bw; ++c) {
    const float* ck = colk[c & 1];
    // pivot search, repeated by every warp: key = (|v| bits + 1, -row), NaN above numbers,
    // ties to the smallest row
    unsigned long long key = 0ull;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = l + 32 * t;
      if (!((sel >> t) & 1ull)) {
        const unsigned long long kv = ((unsigned long long)(__float_as_uint(fabsf(ck[i])) + 1u) << 32) |
                                      (unsigned)(0x7fffffff - i);
        key = kv > key ? kv : key;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, off);
      key = o > key ? o : key;
    }
    const int p = 0x7fffffff - (int)(unsigned)(key & 0xffffffffull);
    const float d = ck[p];
    bad |= !(fabsf(d) > 0.f);
    const float dinv = (d == 0.f) ? 0.f : 1.f / d;
    if (l == (p & 31)) sel |= 1ull << (p >> 5);
    if (w == p % NW) {
      const int pr = p / NW;
#pragma unroll
      for (int q = 0; q < ND; ++q)
        if ((pr >> 6) == q) done[q] |= 1ull << (pr & 63);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r == pr) rowk[l] = M[r];
    }
    if (threadIdx.x == 0) pk[c] = p;
    __syncthreads();
    const float rk = rowk[l];
    const int c1 = c + 1;
    float* cn = colk[c1 & 1];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = w + NW * r;
      if (!((done[r >> 6] >> (r & 63)) & 1ull)) {
        const float m = ck[i] * dinv;
        const float v = M[r];
        M[r] = (l == c) ? m : ((l > c) ? fmaf(-m, rk, v) : v);
      }
      if (l == c1) cn[i] = M[r];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int c = 0; c < bw; ++c) {
      const int p = pk[c], q = where_[p], rc = at[c];
      ipv[c] = q;
      at[c] = p; at[q] = rc;
      where_[p] = c; where_[rc] = q;
    }
  }
  __syncthreads();
  // positions below the panel's first bw that received another row (at most bw of them)
  for (int q = bw + threadIdx.x; q < rows; q += blockDim.x)
    if (at[q] != q) xl[atomicAdd(&s_nx, 1)] = q;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = w + NW * r;
    if (i < rows && l < bw) {
      const int pos = where_[i];
      Mx[(long long)(k0 + pos) * lda + k0 + l] = M[r];
      if (pos < bw) L11[pos][l] = M[r];
    }
  }
  if (threadIdx.x < bw) piv[k0 + threadIdx.x] = k0 + ipv[threadIdx.x];
  __syncthreads();
  const int nx = s_nx;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    if (j >= k0 && j < k0 + bw) continue;
    float v1[PW], v2[PW];
#pragma unroll
    for (int c = 0; c < PW; ++c) v1[c] = c < bw ? Mx[(long long)(k0 + at[c]) * lda + j] : 0.f;
#pragma unroll
    for (int q = 0; q < PW; ++q) v2[q] = q < nx ? Mx[(long long)(k0 + at[xl[q]]) * lda + j] : 0.f;
    // every load of the column precedes its stores (the two row sets overlap)
#pragma unroll
    for (int q = 0; q < PW; ++q)
      if (q < nx) Mx[(long long)(k0 + xl[q]) * lda + j] = v2[q];
    if (j >= k0 + bw) {
#pragma unroll
      for (int c = 0; c < PW; ++c)
#pragma unroll
        for (int i = c + 1; i < PW; ++i) v1[i] = fmaf(-L11[i][c], v1[c], v1[i]);
    }
#pragma unroll
    for (int c = 0; c < PW; ++c)
      if (c < bw) Mx[(long long)(k0 + c) * lda + j] = v1[c];
  }
  if (threadIdx.x == 0 && bad) atomicCAS(status, -1, e);
}

__global__ void __launch_bounds__(256, 2) k_lu_panel_reg(int n, int k0, float* __restrict__ A, long long stride,
                                                         int lda, int* __restrict__ piv_all,
                                                         int* __restrict__ status) {
  const int e = blockIdx.x;
  lu_panel_reg_body<8, LPR_R>(n, k0, A + (long long)e * stride, lda, piv_all + (long long)e * n, status, e);
}

__global__ void __launch_bounds__(32 * LPR2_W, 1) k_lu_panel_reg2(int n, int k0, float* __restrict__ A,
                                                                  long long stride, int lda,
                                                                  int* __restrict__ piv_all, int* __restrict__ status) {
  const int e = blockIdx.x;
  lu_panel_reg_body<LPR2_W, LPR2_R>(n, k0, A + (long long)e * stride, lda, piv_all + (long long)e * n, status, e);
}

__global__ void __launch_bounds__(256, 2) k_lu_panel_reg_grouped(const CondItem* __restrict__ items, int k0) {
  const CondItem it = items[blockIdx.x];
  if (it.nb <= k0) return;
  lu_panel_reg_body<8, LPR_R>(it.nb, k0, it.See, it.lds, it.piv, it.status, it.e);
}

__global__ void __launch_bounds__(32 * LPR2_W, 1) k_lu_panel_reg2_grouped(const CondItem* __restrict__ items, int k0) {
  const CondItem it = items[blockIdx.x];
  if (it.nb <= k0) return;
  lu_panel_reg_body<LPR2_W, LPR2_R>(it.nb, k0, it.See, it.lds, it.piv, it.status, it.e);
}

// ---- blocked Gauss-Jordan inverse (blocks too large for one CTA's registers) ----------
// A is inverted in place, 32 pivot columns K = k0 .. k0+31 at a time:
//   k_gjb_panel   Gauss-Jordan on the n x 32 panel (pivots among rows >= k0, implicit
//                 during the eliminations, then applied as row interchanges to every
//                 column): the pivot rows P = k0 .. k0+31 of the panel hold G^-1
//                 (G = A[P, K]), the other rows -A[R, K] G^-1;
//   k_gjb_update  A[P, J] <- G^-1 A[P, J] and A[R, J] <- A[R, J] - A[R, K] G^-1 A[P, J] for
//                 the columns J outside the panel, both as A[., J] (+)= panel x A_old[P, J];
//   k_gjb_unpermute  the row interchanges undone as column interchanges, last first.
// The panel kernel holds rows w + 16 r (r < 40) of lane l's column: n <= 640.
constexpr int GJB_R = 40, GJB_ROWS = 16 * GJB_R, GJB_CH = 64;

// Warp argmax of |v| over (value, row) with NaN above every number and ties to the
// smallest row; every lane ends with the same pair.
template <class T>
__device__ __forceinline__ bool gjb_better(T a, int ia, T b, int ib) {
  const bool na = a != a, nb_ = b != b;
  if (na || nb_) return na && (!nb_ || ia < ib);
  return a > b || (a == b && ia < ib);
}

template <class T>
__device__ void gjb_panel_body(int n, int k0, T* __restrict__ Mx, int lda, int* __restrict__ piv,
                               int* __restrict__ status, int e) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stage = reinterpret_cast<T*>(smem_raw);  // [2 PW][GJB_CH + 1]: moved rows of one column chunk
  __shared__ T colk[2][GJB_ROWS];
  __shared__ T rowk[PW];
  __shared__ int pk[PW], ipv[PW], xl[PW];
  __shared__ int at[GJB_ROWS], where_[GJB_ROWS];  // positions k0 + q (q relative) <-> rows
  __shared__ int s_nx;
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int bw = min(PW, n - k0), rows = n - k0;
  T M[GJB_R];
#pragma unroll
  for (int r = 0; r < GJB_R; ++r) {
    const int i = w + 16 * r;
    M[r] = (i < n && l < bw) ? Mx[(long long)i * lda + k0 + l] : T(0);
  }
  if (l == 0) {
#pragma unroll
    for (int r = 0; r < GJB_R; ++r) colk[0][w + 16 * r] = M[r];
  }
  for (int i = threadIdx.x; i < GJB_ROWS; i += blockDim.x) { at[i] = i; where_[i] = i; }
  if (threadIdx.x == 0) s_nx = 0;
  unsigned sel = 0;  // bit t: row l + 32 t is not a pivot candidate (above k0, chosen, or past n)
#pragma unroll
  for (int t = 0; t < GJB_ROWS / 32; ++t) {
    const int i = l + 32 * t;
    if (i < k0 || i >= n) sel |= 1u << t;
  }
  bool bad = false;
  __syncthreads();
  for (int c = 0; c < bw; ++c) {
    const T* ck = colk[c & 1];
    T best = T(-1);
    int bi = 0x7fffffff;
#pragma unroll
    for (int t = 0; t < GJB_ROWS / 32; ++t) {
      const int i = l + 32 * t;
      if (!((sel >> t) & 1u)) {
        const T a = tabs(ck[i]);
        if (gjb_better(a, i, best, bi)) { best = a; bi = i; }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (gjb_better(ob, oi, best, bi)) { best = ob; bi = oi; }
    }
    const int p = bi;
    const T d = ck[p];
    const bool ok = tabs(d) > T(0);
    bad |= !ok;
    const T pinv = ok ? T(1) / d : T(0);
    if (l == (p & 31)) sel |= 1u << (p >> 5);
    if (w == (p & 15)) {
      const int pr = p >> 4;
#pragma unroll
      for (int r = 0; r < GJB_R; ++r)
        if (r == pr) rowk[l] = M[r];
    }
    if (threadIdx.x == 0) pk[c] = p;
    __syncthreads();
    const T rk = rowk[l];
    const int c1 = c + 1;
    T* cn = colk[c1 & 1];
#pragma unroll
    for (int r = 0; r < GJB_R; ++r) {
      const int i = w + 16 * r;
      const T f = ck[i] * pinv;
      const T v = M[r];
      M[r] = (i == p) ? ((l == c) ? pinv : v * pinv) : ((l == c) ? -f : fma(-f, rk, v));
      if (l == c1) cn[i] = M[r];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int c = 0; c < bw; ++c) {
      const int p = pk[c] - k0, q = where_[p], rc = at[c];
      ipv[c] = q;
      at[c] = p; at[q] = rc;
      where_[p] = c; where_[rc] = q;
    }
  }
  __syncthreads();
  for (int q = bw + threadIdx.x; q < rows; q += blockDim.x)
    if (at[q] != q) xl[atomicAdd(&s_nx, 1)] = q;
#pragma unroll
  for (int r = 0; r < GJB_R; ++r) {
    const int i = w + 16 * r;
    if (i < n && l < bw) {
      const int pos = i < k0 ? i : k0 + where_[i - k0];
      Mx[(long long)pos * lda + k0 + l] = M[r];
    }
  }
  if (threadIdx.x < bw) piv[k0 + threadIdx.x] = k0 + ipv[threadIdx.x];
  __syncthreads();
  // the interchanges on the columns outside the panel, one chunk of columns at a time
  const int nm = bw + s_nx;  // moved positions: 0 .. bw-1, then xl[]
  for (int j0 = 0; j0 < n; j0 += GJB_CH) {
    for (int t = threadIdx.x; t < nm * GJB_CH; t += blockDim.x) {
      const int m = t / GJB_CH, j = j0 + t % GJB_CH;
      if (j < n && (j < k0 || j >= k0 + bw)) {
        const int src = k0 + (m < bw ? at[m] : at[xl[m - bw]]);
        stage[m * (GJB_CH + 1) + t % GJB_CH] = Mx[(long long)src * lda + j];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nm * GJB_CH; t += blockDim.x) {
      const int m = t / GJB_CH, j = j0 + t % GJB_CH;
      if (j < n && (j < k0 || j >= k0 + bw)) {
        const int dst = k0 + (m < bw ? m : xl[m - bw]);
        Mx[(long long)dst * lda + j] = stage[m * (GJB_CH + 1) + t % GJB_CH];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicCAS(status, -1, e);
}

template <class T>
__device__ void gjb_update_body(int n, int k0, T* __restrict__ Mx, int lda, int j0) {
  __shared__ T Ts[PW][GJB_CH];      // A_old[P, J] of this column block
  __shared__ T As[GJB_CH][PW + 1];  // panel columns of a 64-row tile
  const int bw = min(PW, n - k0);
  for (int t = threadIdx.x; t < PW * GJB_CH; t += blockDim.x) {
    const int k = t / GJB_CH, jj = t % GJB_CH, j = j0 + jj;
    Ts[k][jj] = (k < bw && j < n && (j < k0 || j >= k0 + bw)) ? Mx[(long long)(k0 + k) * lda + j] : T(0);
  }
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;  // rows 4 tr + a, columns tc + 16 b
  for (int i0 = 0; i0 < n; i0 += GJB_CH) {
    __syncthreads();
    for (int t = threadIdx.x; t < GJB_CH * PW; t += blockDim.x) {
      const int ii = t / PW, k = t % PW;
      As[ii][k] = (i0 + ii < n && k < bw) ? Mx[(long long)(i0 + ii) * lda + k0 + k] : T(0);
    }
    __syncthreads();
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
#pragma unroll 8
    for (int k = 0; k < PW; ++k) {
      T x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = As[4 * tr + a][k];
#pragma unroll
      for (int b = 0; b < 4; ++b) y[b] = Ts[k][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + 4 * tr + a;
      if (i >= n) continue;
      const bool pivot_row = i >= k0 && i < k0 + bw;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = j0 + tc + 16 * b;
        if (j >= n || (j >= k0 && j < k0 + bw)) continue;
        T* dst = Mx + (long long)i * lda + j;
        *dst = pivot_row ? acc[a][b] : *dst + acc[a][b];
      }
    }
  }
}

// Row equilibration before the blocked Gauss-Jordan: a row <- d_i row, d_i = 1 / max |a_i.|,
// one warp per row; the unpermute pass multiplies column j of the inverse by d_j.
template <class T>
__device__ void row_equilibrate_body(int n, T* __restrict__ Mx, int lda, T* __restrict__ dsc) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), l = threadIdx.x & 31;
  if (i >= n) return;
  T* row = Mx + (long long)i * lda;
  T mx = T(0);
  for (int j = l; j < n; j += 32) mx = fmax(mx, tabs(row[j]));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const T d = mx > T(0) ? T(1) / mx : T(1);
  for (int j = l; j < n; j += 32) row[j] *= d;
  if (l == 0) dsc[i] = d;
}

template <class T>
__device__ void gjb_unpermute_body(int n, T* __restrict__ Mx, int lda, const int* __restrict__ piv,
                                   const T* __restrict__ dsc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rowbuf = reinterpret_cast<T*>(smem_raw);  // [16 warps][GJB_ROWS]
  __shared__ int perm[GJB_ROWS];
  for (int j = threadIdx.x; j < n; j += blockDim.x) perm[j] = j;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = n - 1; k >= 0; --k) {
      const int p = piv[k];
      if (p != k) { const int t = perm[k]; perm[k] = perm[p]; perm[p] = t; }
    }
  __syncthreads();
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* rb = rowbuf + (size_t)w * GJB_ROWS;
  for (int i = w; i < n; i += 16) {
    for (int j = l; j < n; j += 32) rb[j] = Mx[(long long)i * lda + j];
    __syncwarp();
    for (int j = l; j < n; j += 32) Mx[(long long)i * lda + j] = rb[perm[j]] * dsc[j];
    __syncwarp();
  }
}

template <class T>
__global__ void __launch_bounds__(512, 1) k_gjb_panel(int n, int k0, T* __restrict__ A, long long stride, int lda,
                                                      int* __restrict__ piv_all, int* __restrict__ status) {
  const int e = blockIdx.x;
  gjb_panel_body<T>(n, k0, A + (long long)e * stride, lda, piv_all + (long long)e * n, status, e);
}

template <class T>
__global__ void __launch_bounds__(256) k_gjb_update(int n, int k0, T* __restrict__ A, long long stride, int lda) {
  gjb_update_body<T>(n, k0, A + (long long)blockIdx.y * stride, lda, blockIdx.x * GJB_CH);
}

template <class T>
__global__ void k_row_equilibrate(int n, T* __restrict__ A, long long stride, int lda, T* __restrict__ dsc) {
  row_equilibrate_body<T>(n, A + (long long)blockIdx.y * stride, lda, dsc + (long long)blockIdx.y * n);
}

template <class T>
__global__ void __launch_bounds__(512) k_gjb_unpermute(int n, T* __restrict__ A, long long stride, int lda,
                                                       const int* __restrict__ piv_all, const T* __restrict__ dsc) {
  const int e = blockIdx.x;
  gjb_unpermute_body<T>(n, A + (long long)e * stride, lda, piv_all + (long long)e * n, dsc + (long long)e * n);
}

// The same four steps for batched items (one item per CTA, blockIdx.y for the 2-D grids);
// items whose A_ii is done or narrower than the block return at once.
__global__ void k_copy_aii_grouped(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.y];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < it.ni * it.ni; t += gridDim.x * blockDim.x) {
    const int i = t / it.ni, j = t % it.ni;
    it.Ainv[(long long)i * it.ldi + j] = it.Aown[(long long)i * it.lda + j];
  }
}

__global__ void k_row_equilibrate_grouped(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.y];
  row_equilibrate_body<float>(it.ni, it.Ainv, it.ldi, it.dsc);
}

__global__ void __launch_bounds__(512, 1) k_gjb_panel_grouped(const CondItem* __restrict__ items, int k0) {
  const CondItem it = items[blockIdx.x];
  if (it.ni <= k0) return;
  gjb_panel_body<float>(it.ni, k0, it.Ainv, it.ldi, it.piv, it.status, it.e);
}

__global__ void __launch_bounds__(256) k_gjb_update_grouped(const CondItem* __restrict__ items, int k0) {
  const CondItem it = items[blockIdx.y];
  if (it.ni <= k0 || (int)blockIdx.x * GJB_CH >= it.ni) return;
  gjb_update_body<float>(it.ni, k0, it.Ainv, it.ldi, blockIdx.x * GJB_CH);
}

__global__ void __launch_bounds__(512) k_gjb_unpermute_grouped(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.x];
  gjb_unpermute_body<float>(it.ni, it.Ainv, it.ldi, it.piv, it.dsc);
}

// One panel step of every batched item whose S_ee extends beyond column k0.
__global__ void __launch_bounds__(256) k_lu_panel_grouped(const CondItem* __restrict__ items, int k0) {
  extern __shared__ unsigned char smem_raw[];
  float* P = reinterpret_cast<float*>(smem_raw);
  __shared__ int s_p;
  __shared__ int s_bad;
  const CondItem it = items[blockIdx.x];
  if (it.nb <= k0) return;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  lu_panel<float>(it.nb, k0, it.See, it.lds, it.piv, P, &s_p, &s_bad);
  if (threadIdx.x == 0 && s_bad) atomicCAS(it.status, -1, it.e);
}

// Replace every 32 x 32 diagonal block of the LU factors by the inverses of its
// triangles: strictly lower part <- (unit lower L_bb)^-1, upper part <- (U_bb)^-1.  The
// off-diagonal blocks (all the substitutions read besides these) are untouched.  One CTA
// per element, one warp per block, one lane per column.
template <class T>
__device__ void diag_inv_body(int n, T* __restrict__ M, int lda) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  T* Ds = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 2 * 32 * 33;  // block, then its inverse
  T* Is = Ds + 32 * 33;
  const int nblk = (n + 31) / 32;
  for (int b = warp; b < nblk; b += nw) {
    const int i0 = b * 32, bs = min(32, n - i0);
    for (int r = 0; r < bs; ++r) Ds[r * 33 + lane] = lane < bs ? M[(long long)(i0 + r) * lda + i0 + lane] : T(0);
    __syncwarp();
    if (lane < bs) {
      const int c = lane;
      // column c of L^-1 (unit lower)
      for (int i = 0; i < bs; ++i) {
        T x = T(0);
        if (i == c) x = T(1);
        else if (i > c) {
          for (int k = c; k < i; ++k) x = fma(-Ds[i * 33 + k], Is[k * 33 + c], x);
        }
        Is[i * 33 + c] = x;
      }
      // column c of U^-1 (upper), rows c down to 0, stored in the upper part
      T xc = T(1) / Ds[c * 33 + c];
      T col[32];
      col[c] = xc;
      for (int i = c - 1; i >= 0; --i) {
        T acc = T(0);
        for (int k = i + 1; k <= c; ++k) acc = fma(Ds[i * 33 + k], col[k], acc);
        col[i] = -acc / Ds[i * 33 + i];
      }
      for (int i = 0; i <= c; ++i) Is[i * 33 + c] = col[i];
    }
    __syncwarp();
    for (int r = 0; r < bs; ++r)
      if (lane < bs) M[(long long)(i0 + r) * lda + i0 + lane] = Is[r * 33 + lane];
    __syncwarp();
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_diag_inv(int n, T* __restrict__ LU, long long stride, int lda) {
  diag_inv_body<T>(n, LU + (long long)blockIdx.x * stride, lda);
}

__global__ void __launch_bounds__(256) k_diag_inv_grouped(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.x];
  diag_inv_body<float>(it.nb, it.See, it.lds);
}

// Sequential LAPACK-style row interchanges -> one gather permutation per element:
// row i of P A is row rowperm[i] of A.
__device__ void piv_to_perm_body(int n, const int* __restrict__ piv, int* __restrict__ rp) {
  for (int i = 0; i < n; ++i) rp[i] = i;
  for (int k = 0; k < n; ++k) {
    const int p = piv[k];
    if (p != k) { const int t = rp[k]; rp[k] = rp[p]; rp[p] = t; }
  }
}

__global__ void k_piv_to_perm(int n, const int* __restrict__ piv_all, int* __restrict__ rowperm, int nelem) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nelem) return;
  piv_to_perm_body(n, piv_all + (long long)e * n, rowperm + (long long)e * n);
}

__global__ void k_piv_to_perm_grouped(const CondItem* __restrict__ items, int nitems) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nitems) return;
  const CondItem it = items[t];
  piv_to_perm_body(it.nb, it.piv, it.rowperm);
}


// ---- block-Jacobi solve with partitioned inverses -----------------------------------
// With D_b the 32 x 32 diagonal blocks of the factors (their triangles replaced by the
// triangles' inverses, k_diag_inv), forward and backward substitution read
//   x_b = L_bb^-1 v_b - M_b x_{<b},   M_b = L_bb^-1 L_{b,<b}
//   z_b = U_bb^-1 x_b - N_b z_{>b},   N_b = U_bb^-1 U_{b,>b}
// so every step is one dot product per row and needs no triangular solve.  The solve
// layout stores, per element and 32-row block row b, columns in groups of four:
// element (row 32 b + r, column c) at [b][c / 4][r][c % 4] (npad = n rounded up to 4
// columns, rows beyond n zero).  A warp then reads one 4-column group of all 32 rows as
// 32 consecutive 16- (FP32) or 32-byte (FP64) pieces.

// Four consecutive stored factor entries (type TS) widened to the arithmetic type T.
template <class T, class TS> struct Quad;
template <> struct Quad<float, float> {
  float v[4];
  __device__ __forceinline__ void load(const float* p) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <> struct Quad<double, double> {
  double v[4];
  __device__ __forceinline__ void load(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
template <> struct Quad<float, __half> {
  float v[4];
  __device__ __forceinline__ void load(const __half* p) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

// One CTA per (block row b, element): D_b from the factors, then every column c of the
// block row: c < i0 -> M_b, diagonal block -> D_b, c >= i0 + 32 -> N_b.
// With LS16 non-null (FP32 factors only) the layout is also written in FP16; an entry
// beyond the FP16 range sets *ovf.
template <class T>
__device__ void solve_prep_body(int n, int b, const T* __restrict__ M, int lda, T* __restrict__ out, int npad,
                                __half* __restrict__ out16, int* __restrict__ ovf) {
  __shared__ T TL[32][33];  // L_bb^-1: unit diagonal, stored inverse below it
  __shared__ T TU[32][33];  // U_bb^-1: stored inverse on and above the diagonal
  __shared__ T D[32][33];   // diagonal block as stored (both inverse triangles)
  const int i0 = 32 * b, bs = min(32, n - i0);
  bool big = false;
  for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
    const int r = t / 32, k = t % 32;
    const T dv = (r < bs && k < bs) ? M[(long long)(i0 + r) * lda + i0 + k] : T(0);
    D[r][k] = dv;
    TL[r][k] = (r < bs && k < bs) ? (k < r ? dv : (k == r ? T(1) : T(0))) : T(0);
    TU[r][k] = (k >= r) ? dv : T(0);
  }
  __syncthreads();
  for (int cidx = threadIdx.x; cidx < npad; cidx += blockDim.x) {
    T col[32];
    const bool left = cidx < i0, right = cidx >= i0 + 32;
#pragma unroll
    for (int k = 0; k < 32; ++k)
      col[k] = (k < bs && cidx < n && (left || right)) ? M[(long long)(i0 + k) * lda + cidx] : T(0);
    const long long oo = (long long)(cidx / 4) * 128 + (cidx % 4);
    T* o = out + oo;
    for (int r = 0; r < 32; ++r) {
      T acc = T(0);
      if (left || right) {
        T(*Tm)[33] = left ? TL : TU;
#pragma unroll
        for (int k = 0; k < 32; ++k) acc = fma(Tm[r][k], col[k], acc);
      } else {
        acc = cidx < n ? D[r][cidx - i0] : T(0);
      }
      o[4 * r] = acc;
      if (out16) {
        out16[oo + 4 * r] = __float2half_rn((float)acc);
        big = big || !(fabs((double)acc) <= 65000.0);
      }
    }
  }
  if (out16 && big) atomicExch(ovf, 1);
}

template <class T>
__global__ void __launch_bounds__(256) k_solve_prep(int n, const T* __restrict__ LU, long long stride, int lda,
                                                    T* __restrict__ LS, long long lsstride, int npad,
                                                    __half* __restrict__ LS16, int* __restrict__ ovf) {
  const int b = blockIdx.x, e = blockIdx.y;
  const long long off = (long long)e * lsstride + (long long)b * 32 * npad;
  solve_prep_body<T>(n, b, LU + (long long)e * stride, lda, LS + off, npad, LS16 ? LS16 + off : nullptr, ovf);
}

__global__ void __launch_bounds__(256) k_solve_prep_grouped(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.y];
  const int b = blockIdx.x, nblk = (it.nb + 31) / 32, npad = (it.nb + 3) & ~3;
  if (b >= nblk) return;
  solve_prep_body<float>(it.nb, b, it.See, it.lds, it.Sls + (long long)b * 32 * npad, npad, nullptr, nullptr);
}

// In-place (L U)^-1 s of one element's factors Le in the solve layout, by one warp: lane r
// owns row 32 b + r of every block; s (shared memory, nblk * 32 entries, zero beyond n)
// holds the permuted right-hand side on entry and the solution on exit.
template <class T, class TS>
__device__ __forceinline__ void ls_solve_warp(int n, int nblk, const TS* __restrict__ Le, int npad, T* s, int lane) {
  // Lanes of padding rows (R >= n) load nothing, and in the diagonal block each lane
  // loads only the 4-column groups that hold entries of its own triangle: those sectors
  // are never fetched.
  const int nq = npad / 4;
  for (int b = 0; b < nblk; ++b) {  // forward: x_b = L_bb^-1 v_b - M_b x_{<b}
    const int i0 = 32 * b, R = i0 + lane;
    const bool live = R < n;
    const TS* row = Le + (long long)b * 32 * npad + 4 * lane;
    T a0 = T(0), a1 = T(0);
    if (live) {
#pragma unroll 8
      for (int q = 0; q < i0 / 4; ++q) {
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
        a0 = fma(m.v[0], s[4 * q], a0);
        a1 = fma(m.v[1], s[4 * q + 1], a1);
        a0 = fma(m.v[2], s[4 * q + 2], a0);
        a1 = fma(m.v[3], s[4 * q + 3], a1);
      }
    }
    T d = s[R];
    const int qd = min(i0 / 4 + 8, nq);  // the last block row may end before 32 columns
#pragma unroll
    for (int q = i0 / 4; q < qd; ++q) {
      if (live && 4 * q < R) {  // strictly lower part: columns < R
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j < R) d = fma(m.v[j], s[4 * q + j], d);
      }
    }
    __syncwarp();
    if (live) s[R] = d - (a0 + a1);
    __syncwarp();
  }
  for (int b = nblk - 1; b >= 0; --b) {  // backward: z_b = U_bb^-1 x_b - N_b z_{>b}
    const int i0 = 32 * b, R = i0 + lane;
    const bool live = R < n;
    const TS* row = Le + (long long)b * 32 * npad + 4 * lane;
    T d = T(0);
    const int qd = min(i0 / 4 + 8, nq);
#pragma unroll
    for (int q = i0 / 4; q < qd; ++q) {
      if (live && 4 * q + 3 >= R) {  // upper part: columns >= R
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j >= R) d = fma(m.v[j], s[4 * q + j], d);
      }
    }
    T a0 = T(0), a1 = T(0);
    if (live) {
#pragma unroll 8
      for (int q = i0 / 4 + 8; q < nq; ++q) {
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
        a0 = fma(m.v[0], s[4 * q], a0);
        a1 = fma(m.v[1], s[4 * q + 1], a1);
        a0 = fma(m.v[2], s[4 * q + 2], a0);
        a1 = fma(m.v[3], s[4 * q + 3], a1);
      }
    }
    __syncwarp();
    if (live) s[R] = d - (a0 + a1);
    __syncwarp();
  }
}

// The same substitutions by a CTA of W warps per element, for meshes with too few elements
// to fill the GPU one warp each: in every block row the W warps share the off-diagonal
// 4-column groups (strided), their partial dot products meet in shared memory, and warp
// 0 adds the diagonal block's part and writes the row.  Two CTA barriers per block row.
// ls_solve_warp with loads issued ahead of the dependence on s: each block row's diagonal
// block quads are loaded before its long dot product, and the first 8 quads of the next
// row's long part before the row's result is written.  The factor entries do not depend on
// the solution, so a warp keeps more loads in flight across the short, serial stretch at
// each block row; for launches with few warps per SM (one colour of the red-black sweep).
template <class T, class TS>
__device__ __forceinline__ void ls_solve_warp_pf(int n, int nblk, const TS* __restrict__ Le, int npad, T* s, int lane) {
  const int nq = npad / 4;
  Quad<T, TS> pre[8];
  bool have_pre = false;
  for (int b = 0; b < nblk; ++b) {  // forward: x_b = L_bb^-1 v_b - M_b x_{<b}
    const int i0 = 32 * b, R = i0 + lane;
    const bool live = R < n;
    const TS* row = Le + (long long)b * 32 * npad + 4 * lane;
    const int q0 = i0 / 4, qd = min(q0 + 8, nq);
    Quad<T, TS> dg[8];
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (live && q0 + t < qd && 4 * (q0 + t) < R) dg[t].load(row + (long long)(q0 + t) * 128);
    T a0 = T(0), a1 = T(0);
    if (live) {
      int q = 0;
      if (have_pre) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          a0 = fma(pre[t].v[0], s[4 * t], a0);
          a1 = fma(pre[t].v[1], s[4 * t + 1], a1);
          a0 = fma(pre[t].v[2], s[4 * t + 2], a0);
          a1 = fma(pre[t].v[3], s[4 * t + 3], a1);
        }
        q = 8;
      }
#pragma unroll 8
      for (; q < q0; ++q) {
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
        a0 = fma(m.v[0], s[4 * q], a0);
        a1 = fma(m.v[1], s[4 * q + 1], a1);
        a0 = fma(m.v[2], s[4 * q + 2], a0);
        a1 = fma(m.v[3], s[4 * q + 3], a1);
      }
    }
    T d = s[R];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int q = q0 + t;
      if (live && q < qd && 4 * q < R) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j < R) d = fma(dg[t].v[j], s[4 * q + j], d);
      }
    }
    // the next row's first 8 quads (columns 0..31: its long part starts there)
    have_pre = b + 1 < nblk && 32 * (b + 1) + lane < n;
    if (have_pre) {
      const TS* nrow = row + (long long)32 * npad;
#pragma unroll
      for (int t = 0; t < 8; ++t) pre[t].load(nrow + (long long)t * 128);
    }
    __syncwarp();
    if (live) s[R] = d - (a0 + a1);
    __syncwarp();
  }
  have_pre = false;
  for (int b = nblk - 1; b >= 0; --b) {  // backward: z_b = U_bb^-1 x_b - N_b z_{>b}
    const int i0 = 32 * b, R = i0 + lane;
    const bool live = R < n;
    const TS* row = Le + (long long)b * 32 * npad + 4 * lane;
    const int q0 = i0 / 4, qd = min(q0 + 8, nq);
    Quad<T, TS> dg[8];
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (live && q0 + t < qd && 4 * (q0 + t) + 3 >= R) dg[t].load(row + (long long)(q0 + t) * 128);
    T a0 = T(0), a1 = T(0);
    if (live) {
      int q = q0 + 8;
      if (have_pre) {  // the row's last 8 quads, loaded during the previous block row
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int qq = nq - 8 + t;
          a0 = fma(pre[t].v[0], s[4 * qq], a0);
          a1 = fma(pre[t].v[1], s[4 * qq + 1], a1);
          a0 = fma(pre[t].v[2], s[4 * qq + 2], a0);
          a1 = fma(pre[t].v[3], s[4 * qq + 3], a1);
        }
      }
      const int qend = have_pre ? nq - 8 : nq;
#pragma unroll 8
      for (; q < qend; ++q) {
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
        a0 = fma(m.v[0], s[4 * q], a0);
        a1 = fma(m.v[1], s[4 * q + 1], a1);
        a0 = fma(m.v[2], s[4 * q + 2], a0);
        a1 = fma(m.v[3], s[4 * q + 3], a1);
      }
    }
    T d = T(0);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int q = q0 + t;
      if (live && q < qd && 4 * q + 3 >= R) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j >= R) d = fma(dg[t].v[j], s[4 * q + j], d);
      }
    }
    // the previous row's last 8 quads (its long part, [q0 of this row, nq), holds at least 8)
    have_pre = b >= 1 && 32 * (b - 1) + lane < n && nq - 8 >= (32 * (b - 1)) / 4 + 8;
    if (have_pre) {
      const TS* prow = row - (long long)32 * npad;
#pragma unroll
      for (int t = 0; t < 8; ++t) pre[t].load(prow + (long long)(nq - 8 + t) * 128);
    }
    __syncwarp();
    if (live) s[R] = d - (a0 + a1);
    __syncwarp();
  }
}

template <class T, class TS, int W>
__device__ __forceinline__ void ls_solve_cta(int n, int nblk, const TS* __restrict__ Le, int npad, T* s, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nq = npad / 4;
  for (int b = 0; b < nblk; ++b) {  // forward
    const int i0 = 32 * b, R = i0 + lane;
    const bool live = R < n;
    const TS* row = Le + (long long)b * 32 * npad + 4 * lane;
    T a0 = T(0), a1 = T(0);
    if (live) {
#pragma unroll 4
      for (int q = w; q < i0 / 4; q += W) {
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
        a0 = fma(m.v[0], s[4 * q], a0);
        a1 = fma(m.v[1], s[4 * q + 1], a1);
        a0 = fma(m.v[2], s[4 * q + 2], a0);
        a1 = fma(m.v[3], s[4 * q + 3], a1);
      }
    }
    red[w * 32 + lane] = a0 + a1;
    __syncthreads();
    if (w == 0) {
      T d = s[R];
      const int qd = min(i0 / 4 + 8, nq);
#pragma unroll
      for (int q = i0 / 4; q < qd; ++q) {
        if (live && 4 * q < R) {
          Quad<T, TS> m;
          m.load(row + (long long)q * 128);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (4 * q + j < R) d = fma(m.v[j], s[4 * q + j], d);
        }
      }
      T sum = T(0);
#pragma unroll
      for (int k = 0; k < W; ++k) sum += red[k * 32 + lane];
      __syncwarp();
      if (live) s[R] = d - sum;
    }
    __syncthreads();
  }
  for (int b = nblk - 1; b >= 0; --b) {  // backward
    const int i0 = 32 * b, R = i0 + lane;
    const bool live = R < n;
    const TS* row = Le + (long long)b * 32 * npad + 4 * lane;
    T a0 = T(0), a1 = T(0);
    if (live) {
#pragma unroll 4
      for (int q = i0 / 4 + 8 + w; q < nq; q += W) {
        Quad<T, TS> m;
        m.load(row + (long long)q * 128);
        a0 = fma(m.v[0], s[4 * q], a0);
        a1 = fma(m.v[1], s[4 * q + 1], a1);
        a0 = fma(m.v[2], s[4 * q + 2], a0);
        a1 = fma(m.v[3], s[4 * q + 3], a1);
      }
    }
    red[w * 32 + lane] = a0 + a1;
    __syncthreads();
    if (w == 0) {
      T d = T(0);
      const int qd = min(i0 / 4 + 8, nq);
#pragma unroll
      for (int q = i0 / 4; q < qd; ++q) {
        if (live && 4 * q + 3 >= R) {
          Quad<T, TS> m;
          m.load(row + (long long)q * 128);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (4 * q + j >= R) d = fma(m.v[j], s[4 * q + j], d);
        }
      }
      T sum = T(0);
#pragma unroll
      for (int k = 0; k < W; ++k) sum += red[k * 32 + lane];
      __syncwarp();
      if (live) s[R] = d - sum;
    }
    __syncthreads();
  }
}

constexpr int kSolveCtaWarps = 8;

// Element lists (red-black sweep): CTA / warp i serves element elist[i] (all elements when
// elist is null); its factors are number i of LS / rowperm when compact, else number e;
// vsub (optional) is subtracted from v on input.
template <class T, class TS, int W = kSolveCtaWarps>
__global__ void __launch_bounds__(32 * W) k_lu_solve_cta(int n, int nblk, const TS* __restrict__ LS,
                                                                      long long lsstride, int npad,
                                                                      const int* __restrict__ rowperm,
                                                                      const double* __restrict__ v,
                                                                      double* __restrict__ z, T* __restrict__ zt,
                                                                      const int* __restrict__ elist, int compact,
                                                                      const double* __restrict__ vsub) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int e = elist ? __ldg(elist + blockIdx.x) : blockIdx.x, ls = nblk * 32;
  const int f = compact ? blockIdx.x : e;
  T* s = reinterpret_cast<T*>(smem_raw);
  T* red = s + ls;
  const int* rp = rowperm + (long long)f * n;
  const double* ve = v + (long long)e * n;
  const double* we = vsub ? vsub + (long long)e * n : nullptr;
  for (int i = threadIdx.x; i < ls; i += blockDim.x) {
    T val = T(0);
    if (i < n) {
      const int r = __ldg(rp + i);
      val = we ? (T)(ve[r] - we[r]) : (T)ve[r];
    }
    s[i] = val;
  }
  __syncthreads();
  ls_solve_cta<T, TS, W>(n, nblk, LS + (long long)f * lsstride, npad, s, red);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (z) z[(long long)e * n + i] = (double)s[i];
    if (zt) zt[(long long)e * n + i] = s[i];
  }
}

// z = (P^T L U)^-1 v, one warp per element (4 per CTA); the running vector (v, then x,
// then z) sits in shared memory.  Arithmetic in the factor precision T; v in double,
// outputs z (double) and / or zt (T).
template <class T, class TS, bool PF = false>
__global__ void __launch_bounds__(128) k_lu_solve(int n, int nblk, const TS* __restrict__ LS, long long lsstride,
                                                  int npad, const int* __restrict__ rowperm,
                                                  const double* __restrict__ v, double* __restrict__ z,
                                                  T* __restrict__ zt, int nelem, const int* __restrict__ elist,
                                                  int compact,
                                                  const double* __restrict__ vsub) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int idx = blockIdx.x * 4 + warp;
  if (idx >= nelem) return;  // whole warps leave; no block-level barrier follows
  const int e = elist ? __ldg(elist + idx) : idx, f = compact ? idx : e;
  const int ls = nblk * 32;
  T* s = reinterpret_cast<T*>(smem_raw) + (size_t)warp * ls;
  const int* rp = rowperm + (long long)f * n;
  const double* ve = v + (long long)e * n;
  const double* we = vsub ? vsub + (long long)e * n : nullptr;
  for (int i = lane; i < ls; i += 32) {
    T val = T(0);
    if (i < n) {
      const int r = __ldg(rp + i);
      val = we ? (T)(ve[r] - we[r]) : (T)ve[r];
    }
    s[i] = val;
  }
  __syncwarp();
  if constexpr (PF)
    ls_solve_warp_pf<T, TS>(n, nblk, LS + (long long)f * lsstride, npad, s, lane);
  else
    ls_solve_warp<T, TS>(n, nblk, LS + (long long)f * lsstride, npad, s, lane);
  for (int i = lane; i < n; i += 32) {
    const T val = s[i];
    if (z) z[(long long)e * n + i] = (double)val;
    if (zt) zt[(long long)e * n + i] = val;
  }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

namespace sc {

// Blocked LU of the S_ee blocks with the trailing updates A22 -= L21 U12 as batched TF32
// tensor-core GEMMs (mixed arm): per panel one k_lu_panel launch and one GEMM.
// Blocked LU with partial pivoting of `batch` n_b x n_b blocks (row stride lds, block stride
// n_b lds): panels of PW columns, TF32 tensor-core trailing updates; pivots in piv, the first
// singular block's index in *status.
static cudaError_t lu_blocked_tf32_batch(sc_ctx* c, float* See, int K, int* piv, int* status) {
  const Geo& G = c->G;
  const int nb = G.nb, lds = G.lds;
  const long long sS = (long long)nb * lds;
  const size_t smem = (size_t)nb * (PW + 1) * sizeof(float);
  const bool reg = nb <= LPR_ROWS, reg2 = !reg && nb <= LPR2_ROWS;
  cudaError_t err = cudaFuncSetAttribute(k_lu_panel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  for (int k0 = 0; k0 < nb; k0 += PW) {
    const int bw = min(PW, nb - k0), rest = nb - k0 - bw;
    if (k0 > 0) count_launch(c);
    if (reg)
      k_lu_panel_reg<<<K, 256, 0, c->stream>>>(nb, k0, See, sS, lds, piv, status);
    else if (reg2)
      k_lu_panel_reg2<<<K, 32 * LPR2_W, 0, c->stream>>>(nb, k0, See, sS, lds, piv, status);
    else
      k_lu_panel<float><<<K, 256, smem, c->stream>>>(nb, k0, See, sS, lds, piv, status);
    if (rest > 0) {
      count_launch(c);
      err = gemm_tf32(c->stream, rest, rest, bw, -1.0f, See + (size_t)(k0 + bw) * lds + k0, sS, lds, false,
                      See + (size_t)k0 * lds + k0 + bw, sS, lds, false, 1.0f, See + (size_t)(k0 + bw) * lds + k0 + bw,
                      sS, lds, K, c->d_status);
      if (err != cudaSuccess) return err;
    }
  }
  return cudaGetLastError();
}

cudaError_t lu_blocked_tf32(sc_ctx* c, float* See) {
  ProfScope ps(c, SCK_LU);  // one measured span over all panels
  return lu_blocked_tf32_batch(c, See, c->G.K, c->piv, c->d_status);
}

// A_ii^-1 of blocks with n_i > 136 (FP32) or too large for a shared-memory copy (FP64):
// copy A_ii into Ainv, equilibrate its rows, blocked Gauss-Jordan there, undo the
// interchanges and the row scaling.  The pivot
// indices use the S_ee pivot array as scratch (n_i <= n_b), which the LU overwrites later.
template <class T>
cudaError_t gj_blocked(sc_ctx* c, const T* Aown, long long sA, int lda, T* Ainv, int ldi) {
  const Geo& G = c->G;
  const int ni = G.ni, K = G.K;
  const long long sI = (long long)ni * ldi;
  if (ni > GJB_ROWS) return cudaErrorInvalidValue;
  const size_t psm = (size_t)2 * PW * (GJB_CH + 1) * sizeof(T);
  const size_t usm = (size_t)16 * GJB_ROWS * sizeof(T);
  cudaError_t err = cudaFuncSetAttribute(k_gjb_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_gjb_unpermute<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usm);
  if (err != cudaSuccess) return err;
  ProfScope ps(c, SCK_GJ_INV);
  count_launch(c, 2 + 2 * ((ni + PW - 1) / PW));
  T* dsc = reinterpret_cast<T*>(c->gj_scale);
  k_copy_block<T><<<dim3(cdiv((long long)ni * ni, 256 * 8), K), 256, 0, c->stream>>>(ni, ni, Aown, sA, lda, Ainv, sI, ldi);
  k_row_equilibrate<T><<<dim3(cdiv(ni, 8), K), 256, 0, c->stream>>>(ni, Ainv, sI, ldi, dsc);
  for (int k0 = 0; k0 < ni; k0 += PW) {
    k_gjb_panel<T><<<K, 512, psm, c->stream>>>(ni, k0, Ainv, sI, ldi, c->piv, c->d_status);
    k_gjb_update<T><<<dim3(cdiv(ni, GJB_CH), K), 256, 0, c->stream>>>(ni, k0, Ainv, sI, ldi);
  }
  k_gjb_unpermute<T><<<K, 512, usm, c->stream>>>(ni, Ainv, sI, ldi, c->piv, dsc);
  return cudaGetLastError();
}

// Condensation set-up: A_ii^-1 (Gauss-Jordan), Y = A_ii^-1 A_ib,ee, S_ee = A_bb,ee -
// A_bi,ee Y and the LU of S_ee.  With `tc` (FP32 only) the two products and the LU's
// trailing updates run on the TF32 tensor cores and Y is kept transposed (nb x ldi), the
// K-major operand layout of the second product.
template <class T>
cudaError_t condense_t(sc_ctx* c, T* Aown, T* Ainv, T* Y, T* See, bool tc, bool have_inv = false) {
  const Geo& G = c->G;
  const int ni = G.ni, nb = G.nb, K = G.K, lda = G.lda, cb0 = G.cb0, ldi = G.ldi, lds = G.lds;
  const long long sA = (long long)own_stride(G);
  cudaError_t err;
  if (ni > 0) {
    bool done = have_inv;  // A_ii^-1 already in Ainv
    if constexpr (std::is_same<T, float>::value) {
      if (ni <= GJR_N) {
        const size_t smem = (size_t)GJR_N * GJR_LDS * sizeof(float);
        err = cudaFuncSetAttribute(k_gj_inv_reg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        ProfScope ps(c, SCK_GJ_INV);
        k_gj_inv_reg<<<K, 256, smem, c->stream>>>(ni, Aown, sA, lda, Ainv, (long long)ni * ldi, ldi, c->d_status);
        done = true;
      }
    }
    const size_t smem = (size_t)ni * (ni + 1) * sizeof(T) + ni * sizeof(T) + ni * sizeof(int);
    if (!done && (ni > GJR_N || std::is_same<T, double>::value) && smem > kGjSmemMax) {
      err = gj_blocked<T>(c, Aown, sA, lda, Ainv, ldi);
      if (err != cudaSuccess) return err;
      done = true;
    }
    if (!done) {
      err = cudaFuncSetAttribute(k_gj_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      ProfScope ps(c, SCK_GJ_INV);
      k_gj_inv<T><<<K, 256, smem, c->stream>>>(ni, Aown, sA, lda, Ainv, (long long)ni * ldi, ldi, c->d_status);
    }
  }
  if (ni > 0) {
    count_launch(c);
    if constexpr (std::is_same<T, float>::value) {
      if (tc) {
        // Y^T = A_ib,ee^T A_ii^-T  (nb x ni)
        err = gemm_tf32(c->stream, nb, ni, ni, 1.0f, Aown + cb0, sA, lda, true, Ainv, (long long)ni * ldi, ldi, true,
                        0.0f, Y, (long long)nb * ldi, ldi, K, c->d_status);
        if (err != cudaSuccess) return err;
      }
    }
    if (!tc) {
      // Y = A_ii^-1 * A_ib,ee  (ni x nb)
      dim3 g1(cdiv(nb, 64), cdiv(ni, 64), K);
      k_gemm<T><<<g1, 256, 0, c->stream>>>(ni, nb, ni, T(1), Ainv, (long long)ni * ldi, ldi, Aown + cb0, sA, lda,
                                           T(0), Y, (long long)ni * nb, nb);
    }
  }
  // S_ee = A_bb,ee - A_bi,ee * Y
  count_launch(c);
  dim3 gc(cdiv((long long)nb * nb, 256 * 8), K);
  k_copy_block<T><<<gc, 256, 0, c->stream>>>(nb, nb, Aown + (size_t)ni * lda + cb0, sA, lda, See, (long long)nb * lds,
                                             lds);
  if (ni > 0) {
    ProfScope ps(c, SCK_GEMM);
    if constexpr (std::is_same<T, float>::value) {
      if (tc) {
        err = gemm_tf32(c->stream, nb, nb, ni, -1.0f, Aown + (size_t)ni * lda, sA, lda, false, Y, (long long)nb * ldi,
                        ldi, true, 1.0f, See, (long long)nb * lds, lds, K, c->d_status);
        if (err != cudaSuccess) return err;
      }
    }
    if (!tc) {
      dim3 g2(cdiv(nb, 64), cdiv(nb, 64), K);
      k_gemm<T><<<g2, 256, 0, c->stream>>>(nb, nb, ni, T(-1), Aown + (size_t)ni * lda, sA, lda, Y,
                                           (long long)ni * nb, nb, T(1), See, (long long)nb * lds, lds);
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if (c->Sdiag) {  // diagonal node blocks of S_ee for the learned correction's features
      err = extract_sdiag(c, See);
      if (err != cudaSuccess) return err;
      c->Sdiag_valid = true;
    }
    err = gather_black_see(c, See);  // uncorrected black blocks for the learned correction
    if (err != cudaSuccess) return err;
  }
  c->red_compact = false;
  if (c->cfg.precond != SC_PC_NONE) {
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (tc && c->cfg.precond == SC_PC_RB_SCHUR && c->SeeL) {
        // the Schur-corrected sweep factorises only the red blocks here; the black ones are
        // factorised once, after their correction
        err = red_factor32(c, See);
        if (err != cudaSuccess) return err;
        c->red_compact = true;
        return cudaGetLastError();
      }
      if (tc) {
        err = lu_blocked_tf32(c, See);
        if (err != cudaSuccess) return err;
        done = true;
      }
    }
    if (!done) {
      const size_t smem = (size_t)nb * (PW + 1) * sizeof(T);
      err = cudaFuncSetAttribute(k_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
      ProfScope ps(c, SCK_LU);
      k_lu<T><<<K, 256, smem, c->stream>>>(nb, See, (long long)nb * lds, lds, c->piv, c->d_status);
    }
    count_launch(c, 2);
    k_piv_to_perm<<<cdiv(K, 128), 128, 0, c->stream>>>(nb, c->piv, c->rowperm, K);
    const size_t dsm = (size_t)8 * 2 * 32 * 33 * sizeof(T);
    err = cudaFuncSetAttribute(k_diag_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    if (err != cudaSuccess) return err;
    k_diag_inv<T><<<K, 256, dsm, c->stream>>>(nb, See, (long long)nb * lds, lds);
    count_launch(c);
    T* LS = nullptr;
    if constexpr (std::is_same<T, float>::value) LS = c->Sls32; else LS = c->Sls;
    const int nblk = (nb + 31) / 32, npad = (nb + 3) & ~3;
    __half* LS16 = nullptr;
    if constexpr (std::is_same<T, float>::value) LS16 = c->Sls16;
    k_solve_prep<T><<<dim3(nblk, K), 256, 0, c->stream>>>(nb, See, (long long)nb * lds, lds, LS,
                                                           (long long)nblk * 32 * npad, npad, LS16, c->d_status + 1);
  }
  return cudaGetLastError();
}

// Condensation set-up: A_ii^-1, Y = A_ii^-1 A_ib,ee, S_ee = A_bb,ee - A_bi,ee Y, LU(S_ee);
// FP64 arm in place on the FP64 blocks, mixed arm on FP32 copies.
cudaError_t launch_condense(sc_ctx* c) {
  const Geo& G = c->G;
  cudaError_t pe = pack_own(c);
  if (pe != cudaSuccess) return pe;
  c->packed = true;
  if (c->cfg.precision == SC_PREC_MIXED) {  // the packing pass wrote the FP32 own blocks
    count_launch(c);
    const size_t nx = (size_t)G.K * G.NP * 25;
    k_to_float<<<608, 256, 0, c->stream>>>(c->X, c->X32, nx);
    bool have_inv = false;
    if (c->cfg.interior_fp64 && c->Ainv && G.ni > GJR_N) {
      // A_ii^-1 in FP64 from the FP64 own blocks, rounded to FP32 for the operator
      cudaError_t e = gj_blocked<double>(c, c->Aown, (long long)own_stride(G), G.lda, c->Ainv, G.ldi);
      if (e != cudaSuccess) return e;
      count_launch(c);
      k_to_float<<<608, 256, 0, c->stream>>>(c->Ainv, c->Ainv32, (size_t)G.K * G.ni * G.ldi);
      have_inv = true;
    }
    return condense_t<float>(c, c->Aown32, c->Ainv32, c->Y32, c->See32, c->cfg.tensor_cores != 0, have_inv);
  }
  return condense_t<double>(c, c->Aown, c->Ainv, c->Ytmp, c->See, false);
}

// Solve-layout geometry of the S_ee factors.
inline int ls_nblk(const Geo& G) { return (G.nb + 31) / 32; }
inline int ls_npad(const Geo& G) { return (G.nb + 3) & ~3; }
inline long long ls_stride(const Geo& G) { return (long long)ls_nblk(G) * 32 * ls_npad(G); }

// Meshes with fewer elements than this solve the block-Jacobi system with a CTA per element;
// element lists (the red-black sweep's colours) below the second bound.
constexpr int kSolveCtaMaxElems = 2048;
constexpr int kSolveListCtaMaxElems = 1024;

template <class T, class TS>
cudaError_t lu_solve_t(sc_ctx* c, const TS* LS, const double* v, double* z, T* zt) {
  const Geo& G = c->G;
  ProfScope ps(c, SCK_LU_SOLVE);
  const size_t smem = (size_t)4 * ls_nblk(G) * 32 * sizeof(T);
  if (G.K < kSolveCtaMaxElems) {
    const size_t csm = (size_t)(ls_nblk(G) + kSolveCtaWarps) * 32 * sizeof(T);
    k_lu_solve_cta<T, TS><<<G.K, 32 * kSolveCtaWarps, csm, c->stream>>>(G.nb, ls_nblk(G), LS, ls_stride(G),
                                                                       ls_npad(G), c->rowperm, v, z, zt, nullptr, 0,
                                                                       nullptr);
    return cudaGetLastError();
  }
  k_lu_solve<T, TS><<<cdiv(G.K, 4), 128, smem, c->stream>>>(G.nb, ls_nblk(G), LS, ls_stride(G), ls_npad(G),
                                                            c->rowperm, v, z, zt, G.K, nullptr, 0, nullptr);
  return cudaGetLastError();
}

// Block solves of a list of elements (one colour of the red-black sweep): factors LS /
// rowperm by element, or compact (number i for list entry i); vsub subtracted from v.
template <class T, class TS>
cudaError_t lu_solve_list_t(sc_ctx* c, const TS* LS, const int* rowperm, int compact, const int* elist, int nlist,
                            const double* v, const double* vsub, double* z, T* zt) {
  const Geo& G = c->G;
  if (nlist <= 0) return cudaSuccess;
  ProfScope ps(c, SCK_LU_SOLVE, nlist);
  // lists of 1024 elements or more keep one warp per element: at 2048 elements (one colour of
  // 16^3) it takes 0.49 ms per launch against 0.57 ms with 4 and 0.64 ms with 8 warps per
  // element (CTA kernel)
  if (nlist < kSolveListCtaMaxElems) {
    const size_t csm = (size_t)(ls_nblk(G) + kSolveCtaWarps) * 32 * sizeof(T);
    k_lu_solve_cta<T, TS><<<nlist, 32 * kSolveCtaWarps, csm, c->stream>>>(G.nb, ls_nblk(G), LS, ls_stride(G),
                                                                         ls_npad(G), rowperm, v, z, zt, elist,
                                                                         compact, vsub);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)4 * ls_nblk(G) * 32 * sizeof(T);
  // FP32 factors: loads issued ahead (128 registers, 4 CTAs per SM hold one colour of 16^3)
  constexpr bool pf = std::is_same<T, float>::value && std::is_same<TS, float>::value;
  k_lu_solve<T, TS, pf><<<cdiv(nlist, 4), 128, smem, c->stream>>>(G.nb, ls_nblk(G), LS, ls_stride(G),
                                                                  ls_npad(G), rowperm, v, z, zt, nlist, elist,
                                                                  compact, vsub);
  return cudaGetLastError();
}

cudaError_t lu_solve_list(sc_ctx* c, const double* LS, const int* rowperm, int compact, const int* elist, int nlist,
                          const double* v, const double* vsub, double* z) {
  return lu_solve_list_t<double, double>(c, LS, rowperm, compact, elist, nlist, v, vsub, z, nullptr);
}

cudaError_t lu_solve_list32(sc_ctx* c, const float* LS, const int* rowperm, int compact, const int* elist, int nlist,
                            const double* v, const double* vsub, double* z, float* zt) {
  return lu_solve_list_t<float, float>(c, LS, rowperm, compact, elist, nlist, v, vsub, z, zt);
}

cudaError_t precond_apply(sc_ctx* c, const double* v, double* z) {
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb;
  if (c->cfg.precond == SC_PC_NONE) {
    return cudaMemcpyAsync(z, v, n1 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  }
  if (rb_active(c)) return precond_rb(c, v, z);
  return lu_solve_t<double, double>(c, c->Sls, v, z, nullptr);
}

// Block-Jacobi with the FP32 factors; writes z in double and / or zf in float.
cudaError_t precond_apply32(sc_ctx* c, const double* v, double* z, float* zf) {
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb;
  if (c->cfg.precond == SC_PC_NONE) {
    cudaError_t e = cudaSuccess;
    if (z) e = cudaMemcpyAsync(z, v, n1 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && zf) e = vec_to_float(c, zf, v, n1);
    return e;
  }
  if (rb_active(c)) return precond_rb32(c, v, z, zf);
  if (c->ls16_ok) return lu_solve_t<float, __half>(c, c->Sls16, v, z, zf);
  return lu_solve_t<float, float>(c, c->Sls32, v, z, zf);
}

size_t solve_layout_elems(const Geo& G) { return (size_t)G.K * ls_stride(G); }

// ---- grouped launches of the batched condensation (one CTA per CondItem) --------------
cudaError_t grouped_gj(cudaStream_t st, const CondItem* items, int n, int nbig, int max_ni) {
  // items [0, nbig): n_i > 136, blocked Gauss-Jordan; the rest in registers
  cudaError_t e = cudaSuccess;
  if (nbig > 0) {
    const size_t psm = (size_t)2 * PW * (GJB_CH + 1) * sizeof(float);
    const size_t usm = (size_t)16 * GJB_ROWS * sizeof(float);
    e = cudaFuncSetAttribute(k_gjb_panel_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_gjb_unpermute_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usm);
    if (e != cudaSuccess) return e;
    k_copy_aii_grouped<<<dim3(cdiv((long long)max_ni * max_ni, 256 * 8), nbig), 256, 0, st>>>(items);
    k_row_equilibrate_grouped<<<dim3(cdiv(max_ni, 8), nbig), 256, 0, st>>>(items);
    for (int k0 = 0; k0 < max_ni; k0 += PW) {
      k_gjb_panel_grouped<<<nbig, 512, psm, st>>>(items, k0);
      k_gjb_update_grouped<<<dim3(cdiv(max_ni, GJB_CH), nbig), 256, 0, st>>>(items, k0);
    }
    k_gjb_unpermute_grouped<<<nbig, 512, usm, st>>>(items);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (n > nbig) {
    const size_t smem = (size_t)GJR_N * GJR_LDS * sizeof(float);
    e = cudaFuncSetAttribute(k_gj_inv_reg_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gj_inv_reg_grouped<<<n - nbig, 256, smem, st>>>(items + nbig);
  }
  return cudaGetLastError();
}

int grouped_gj_launches(int nbig, int n, int max_ni) {
  return (nbig > 0 ? 3 + 2 * ((max_ni + PW - 1) / PW) : 0) + (n > nbig ? 1 : 0);
}

bool gj_blocked_item(int ni) { return ni > GJR_N; }
bool lu_panel_smem_item(int nb) { return nb > LPR_ROWS; }

cudaError_t grouped_copy_bb(cudaStream_t st, const CondItem* items, int n) {
  k_copy_bb_grouped<<<n, 256, 0, st>>>(items);
  return cudaGetLastError();
}

cudaError_t grouped_lu_panel(cudaStream_t st, const CondItem* items, int n, int nbig, int k0, int max_nb) {
  // items [0, nbig): n_b > 496, 16-warp register panel (shared memory beyond 1104 rows);
  // the rest in the 8-warp register panel
  if (nbig > 0 && max_nb <= LPR2_ROWS) {
    k_lu_panel_reg2_grouped<<<nbig, 32 * LPR2_W, 0, st>>>(items, k0);
  } else if (nbig > 0) {
    const size_t smem = (size_t)max_nb * (PW + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_lu_panel_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_lu_panel_grouped<<<nbig, 256, smem, st>>>(items, k0);
  }
  if (n > nbig) k_lu_panel_reg_grouped<<<n - nbig, 256, 0, st>>>(items + nbig, k0);
  return cudaGetLastError();
}

cudaError_t grouped_finish(cudaStream_t st, const CondItem* items, int n, int max_nb) {
  k_piv_to_perm_grouped<<<cdiv(n, 128), 128, 0, st>>>(items, n);
  const size_t dsm = (size_t)8 * 2 * 32 * 33 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_diag_inv_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
  if (e != cudaSuccess) return e;
  k_diag_inv_grouped<<<n, 256, dsm, st>>>(items);
  k_solve_prep_grouped<<<dim3((max_nb + 31) / 32, n), 256, 0, st>>>(items);
  return cudaGetLastError();
}

cudaError_t to_float(sc_ctx* c, const double* a, float* b, size_t n) {
  count_launch(c);
  k_to_float<<<608, 256, 0, c->stream>>>(a, b, n);
  return cudaGetLastError();
}

// C = A B for `batch` row-major FP32 blocks on the CUDA cores.
// C -= A B for one large row-major problem on the CUDA cores (64 x 64 tiles).
template <class T>
cudaError_t gemm_update(sc_ctx* c, int M, int N, int K, const T* A, int lda, const T* B, int ldb, T* C, int ldc) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  count_launch(c);
  dim3 g(cdiv(N, 64), cdiv(M, 64), 1);
  k_gemm<T><<<g, 256, 0, c->stream>>>(M, N, K, T(-1), A, 0, lda, B, 0, ldb, T(1), C, 0, ldc);
  return cudaGetLastError();
}
template cudaError_t gemm_update<float>(sc_ctx*, int, int, int, const float*, int, const float*, int, float*, int);
template cudaError_t gemm_update<double>(sc_ctx*, int, int, int, const double*, int, const double*, int, double*, int);

cudaError_t gemm_fp32(sc_ctx* c, int M, int N, int K, const float* A, long long sA, int lda, const float* B,
                      long long sB, int ldb, float* C, long long sC, int ldc, int batch) {
  dim3 g(cdiv(N, 64), cdiv(M, 64), batch);
  k_gemm<float><<<g, 256, 0, c->stream>>>(M, N, K, 1.0f, A, sA, lda, B, sB, ldb, 0.0f, C, sC, ldc);
  return cudaGetLastError();
}
long long solve_layout_stride(const Geo& G) { return ls_stride(G); }

// LU with partial pivoting of `batch` FP32 n x n blocks (row-major, lda, `stride` apart),
// then the gather permutation and the partitioned-inverse solve layout LS.
cudaError_t factor_batch32(sc_ctx* c, float* A, int n, int lda, long long stride, int batch, int* piv, int* rowperm,
                           float* LS, int* status) {
  cudaError_t err;
  if (c->cfg.tensor_cores && n == c->G.nb && lda == c->G.lds && stride == (long long)n * lda) {
    err = lu_blocked_tf32_batch(c, A, batch, piv, status);  // element-block sized: TF32 trailing updates
    if (err != cudaSuccess) return err;
    count_launch(c, 3);
  } else {
    const size_t smem = (size_t)n * (PW + 1) * sizeof(float);
    err = cudaFuncSetAttribute(k_lu<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    count_launch(c, 4);
    k_lu<float><<<batch, 256, smem, c->stream>>>(n, A, stride, lda, piv, status);
  }
  k_piv_to_perm<<<cdiv(batch, 128), 128, 0, c->stream>>>(n, piv, rowperm, batch);
  const size_t dsm = (size_t)8 * 2 * 32 * 33 * sizeof(float);
  err = cudaFuncSetAttribute(k_diag_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
  if (err != cudaSuccess) return err;
  k_diag_inv<float><<<batch, 256, dsm, c->stream>>>(n, A, stride, lda);
  const int nblk = (n + 31) / 32, npad = (n + 3) & ~3;
  k_solve_prep<float><<<dim3(nblk, batch), 256, 0, c->stream>>>(n, A, stride, lda, LS, (long long)nblk * 32 * npad,
                                                               npad, nullptr, nullptr);
  return cudaGetLastError();
}

// Diagonal node blocks of the inverses of the element blocks, [S_ee^-1]_kk for every
// (element, boundary node) sample: warp w solves S_ee x = e_c for column c = 5 a + var of
// sample w / 5 with the condensation's factors, and keeps rows 5 a .. 5 a + 4 as column var.
__global__ void __launch_bounds__(128) k_inv_node_blocks(int n, int nblk, const float* __restrict__ LS,
                                                         long long lsstride, int npad, const int* __restrict__ rowperm,
                                                         int nw_total, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int w = blockIdx.x * 4 + warp;
  if (w >= nw_total) return;
  const int smp = w / 5, var = w - 5 * smp, nbn = n / 5;
  const int e = smp / nbn, a = smp % nbn, col = 5 * a + var;
  const int ls = nblk * 32;
  float* s = reinterpret_cast<float*>(smem_raw) + (size_t)warp * ls;
  const int* rp = rowperm + (long long)e * n;
  for (int i = lane; i < ls; i += 32) s[i] = (i < n && __ldg(rp + i) == col) ? 1.f : 0.f;
  __syncwarp();
  ls_solve_warp<float, float>(n, nblk, LS + (long long)e * lsstride, npad, s, lane);
  if (lane < 5) out[(long long)smp * 25 + 5 * lane + var] = s[5 * a + lane];
}

cudaError_t inverse_node_blocks32(sc_ctx* c, float* out) {
  const Geo& G = c->G;
  const int nblk = ls_nblk(G);
  const size_t smem = (size_t)4 * nblk * 32 * sizeof(float);
  cudaError_t err = cudaFuncSetAttribute(k_inv_node_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  count_launch(c);
  const long long nw = (long long)G.K * G.nbn * 5;
  k_inv_node_blocks<<<cdiv(nw, 4), 128, smem, c->stream>>>(G.nb, nblk, c->Sls32, ls_stride(G), ls_npad(G), c->rowperm,
                                                           (int)nw, out);
  return cudaGetLastError();
}


// ls_solve_warp for R right-hand sides at once (s: R vectors of nblk * 32 entries, stride
// ls, zero beyond n): every factor entry the warp loads serves all R columns.
// The forward pass starts at block row b0: the right-hand sides are zero above row 32 b0.
template <int R>
__device__ __forceinline__ void ls_solve_warp_multi(int n, int nblk, const float* __restrict__ Le, int npad,
                                                    float* s, int ls, int lane, int b0) {
  const int nq = npad / 4;
  for (int b = b0; b < nblk; ++b) {  // forward: x_b = L_bb^-1 v_b - M_b x_{<b}
    const int i0 = 32 * b, Rw = i0 + lane;
    const bool live = Rw < n;
    const float* row = Le + (long long)b * 32 * npad + 4 * lane;
    float a[R], d[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = 0.f;
    if (live) {
#pragma unroll 2
      for (int q = 8 * b0; q < i0 / 4; ++q) {
        Quad<float, float> m;
        m.load(row + (long long)q * 128);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4 x = *reinterpret_cast<const float4*>(s + r * ls + 4 * q);
          a[r] = fmaf(m.v[0], x.x, a[r]);
          a[r] = fmaf(m.v[1], x.y, a[r]);
          a[r] = fmaf(m.v[2], x.z, a[r]);
          a[r] = fmaf(m.v[3], x.w, a[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) d[r] = s[r * ls + Rw];
    const int qd = min(i0 / 4 + 8, nq);
    for (int q = i0 / 4; q < qd; ++q) {
      if (live && 4 * q < Rw) {  // strictly lower part: columns < Rw
        Quad<float, float> m;
        m.load(row + (long long)q * 128);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j < Rw) {
#pragma unroll
            for (int r = 0; r < R; ++r) d[r] = fmaf(m.v[j], s[r * ls + 4 * q + j], d[r]);
          }
      }
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[r * ls + Rw] = d[r] - a[r];
    }
    __syncwarp();
  }
  for (int b = nblk - 1; b >= 0; --b) {  // backward: z_b = U_bb^-1 x_b - N_b z_{>b}
    const int i0 = 32 * b, Rw = i0 + lane;
    const bool live = Rw < n;
    const float* row = Le + (long long)b * 32 * npad + 4 * lane;
    float a[R], d[R];
#pragma unroll
    for (int r = 0; r < R; ++r) a[r] = d[r] = 0.f;
    const int qd = min(i0 / 4 + 8, nq);
    for (int q = i0 / 4; q < qd; ++q) {
      if (live && 4 * q + 3 >= Rw) {  // upper part: columns >= Rw
        Quad<float, float> m;
        m.load(row + (long long)q * 128);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * q + j >= Rw) {
#pragma unroll
            for (int r = 0; r < R; ++r) d[r] = fmaf(m.v[j], s[r * ls + 4 * q + j], d[r]);
          }
      }
    }
    if (live) {
#pragma unroll 2
      for (int q = i0 / 4 + 8; q < nq; ++q) {
        Quad<float, float> m;
        m.load(row + (long long)q * 128);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4 x = *reinterpret_cast<const float4*>(s + r * ls + 4 * q);
          a[r] = fmaf(m.v[0], x.x, a[r]);
          a[r] = fmaf(m.v[1], x.y, a[r]);
          a[r] = fmaf(m.v[2], x.z, a[r]);
          a[r] = fmaf(m.v[3], x.w, a[r]);
        }
      }
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[r * ls + Rw] = d[r] - a[r];
    }
    __syncwarp();
  }
}

namespace {

constexpr int kInvCols = 4;   // right-hand sides per warp in k_inv_columns
constexpr int kInvWarps = 4;  // warps per CTA

// Explicit inverses of the element blocks listed: warp w solves S_ee X = I[:, c0 .. c0 + R - 1]
// (R = kInvCols) for element list[w / ngrp], c0 = R (w % ngrp), with the condensation's factors, and writes
// the columns contiguously: out[(i n + c) n + r] = (S_ee^-1)[r][c], i the list index.
__global__ void __launch_bounds__(32 * kInvWarps) k_inv_columns(int n, int nblk, const float* __restrict__ LS,
                                                               long long lsstride, int npad,
                                                               const int* __restrict__ rowperm,
                                                               const int* __restrict__ list, int nlist,
                                                               float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int ngrp = (n + kInvCols - 1) / kInvCols;
  const long long w = (long long)blockIdx.x * kInvWarps + warp;
  if (w >= (long long)nlist * ngrp) return;
  const int li = (int)(w / ngrp), c0 = (int)(w % ngrp) * kInvCols;
  const int e = list ? __ldg(list + li) : li;  // no list: entries in list order (compact factors)
  const int ls = nblk * 32;
  float* s = reinterpret_cast<float*>(smem_raw) + (size_t)warp * kInvCols * ls;
  const int* rp = rowperm + (long long)e * n;
  int first = n;  // the lowest row holding a one: the forward pass starts at its block
  for (int i = lane; i < ls; i += 32) {
    const int pi = i < n ? __ldg(rp + i) : -1;
    if (pi >= c0 && pi < c0 + kInvCols) first = min(first, i);
#pragma unroll
    for (int r = 0; r < kInvCols; ++r) s[r * ls + i] = pi == c0 + r ? 1.f : 0.f;
  }
  first = __reduce_min_sync(0xffffffffu, first);
  __syncwarp();
  ls_solve_warp_multi<kInvCols>(n, nblk, LS + (long long)e * lsstride, npad, s, ls, lane, min(first, n - 1) / 32);
  for (int r = 0; r < kInvCols && c0 + r < n; ++r) {
    float* o = out + ((long long)li * n + c0 + r) * n;
    for (int i = lane; i < n; i += 32) o[i] = s[r * ls + i];
  }
}

}  // namespace

cudaError_t inverse_columns32(sc_ctx* c, const int* list, int nlist, float* out) {
  const Geo& G = c->G;
  if (nlist == 0) return cudaSuccess;
  const int nblk = ls_nblk(G);
  const size_t smem = (size_t)kInvWarps * kInvCols * nblk * 32 * sizeof(float);
  cudaError_t err = cudaFuncSetAttribute(k_inv_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  count_launch(c);
  const long long nw = (long long)nlist * cdiv(G.nb, kInvCols);
  k_inv_columns<<<(unsigned)cdiv(nw, kInvWarps), 32 * kInvWarps, smem, c->stream>>>(G.nb, nblk, c->Sls32, ls_stride(G), ls_npad(G),
                                                                 c->rowperm, list, nlist, out);
  return cudaGetLastError();
}

}  // namespace sc
