// The learned correction of the condensed-system preconditioner: a 128 -> 256 -> 256 -> 25
// network with ReLU hidden layers, BF16 weights and FP32 arithmetic (not in the paper; a
// learned part of the condensed-system preconditioner of Sec. 2.2/4), with its training loop
// (shuffled mini-batch Adam) and a file format for its parameters.
//
// All layers run through one SIMT tile kernel, C (+)= op(A) op(B), 64 x 64 tiles, 16-deep
// K chunks staged in shared memory (BF16 operands widened to FP32 on the way), 4 x 4
// outputs per thread, with the epilogue each use needs:
//   forward      Z = X W^T + b, H = relu(Z)          (A = X, B = W stored out x in)
//   backward dX  dZ_prev = (dZ W) * [Z_prev > 0]      (A = dZ, B = W)
//   backward dW  gW += dZ^T X, split over samples     (A = dZ stored n x out)
// plus the loss, bias-gradient and Adam kernels.  Tensor cores stay with the Schur
// products; the network is ~0.2 MFLOP per boundary node.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sc_internal.cuh"

namespace {

constexpr int NI = sc::kMlpInputs, NH = 256, NO = 25;
constexpr int OFF_W2 = NH * NI, OFF_W3 = OFF_W2 + NH * NH, N_W = OFF_W3 + NO * NH;  // 104,704
constexpr int OFF_B2 = NH, OFF_B3 = 2 * NH, N_B = 2 * NH + NO;                     // 537

template <class T> __device__ __forceinline__ float ldf(const T* p);
template <> __device__ __forceinline__ float ldf<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

enum Epi { EPI_BIAS = 0, EPI_BIAS_RELU = 1, EPI_MASK = 2, EPI_ATOMIC = 3 };

// C[M x N] from op(A)[M x K] op(B)[K x N]; A stored M x K (lda) or K x M when TA;
// B stored K x N (ldb) or N x K when TB.  gridDim.z splits K (EPI_ATOMIC only).
template <class TA_, class TB_, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_mlp_gemm(int M, int N, int K, const TA_* __restrict__ A, int lda,
                                                  const TB_* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                                  const float* __restrict__ bias, float* __restrict__ Zout,
                                                  const float* __restrict__ mask, int kchunk) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      const int kk = t / 64, mm = t % 64;
      const int gk = k0 + kk, gm = m0 + mm, gn = n0 + mm;
      float a = 0.f, b = 0.f;
      if (gk < ke && gm < M) a = TA ? ldf(A + (size_t)gk * lda + gm) : ldf(A + (size_t)gm * lda + gk);
      if (gk < ke && gn < N) b = TB ? ldf(B + (size_t)gn * ldb + gk) : ldf(B + (size_t)gk * ldb + gn);
      As[kk][mm] = a;
      Bs[kk][mm] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty + 16 * i]; b[i] = Bs[kk][tx + 16 * i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = n0 + tx + 16 * j;
      if (cc >= N) continue;
      float v = acc[i][j];
      if (EPI == EPI_ATOMIC) {
        atomicAdd(C + (size_t)r * ldc + cc, v);
      } else {
        if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) {
          v += bias[cc];
          if (Zout) Zout[(size_t)r * ldc + cc] = v;
          if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
        } else if (EPI == EPI_MASK) {
          if (!(mask[(size_t)r * ldc + cc] > 0.f)) v = 0.f;
        }
        C[(size_t)r * ldc + cc] = v;
      }
    }
  }
}

// gb[c] += sum_s dZ[s][c]
__global__ void k_mlp_colsum(int n, int m, const float* __restrict__ dZ, float* __restrict__ gb) {
  const int c = blockIdx.x;
  float s = 0.f;
  for (int r = threadIdx.x; r < n; r += blockDim.x) s += dZ[(size_t)r * m + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float part[32];
  if (threadIdx.x % 32 == 0) part[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < blockDim.x / 32 ? part[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) gb[c] += s;
  }
}

// Mean squared relative Frobenius error of the 25-entry outputs, and its gradient.
__global__ void k_mlp_loss(int n, const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                           float* __restrict__ loss_sum) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (s < n) {
    float num = 0.f, den = 1e-12f;
    for (int j = 0; j < NO; ++j) {
      const float d = Y[(size_t)s * NO + j] - T[(size_t)s * NO + j];
      const float t = T[(size_t)s * NO + j];
      num = fmaf(d, d, num);
      den = fmaf(t, t, den);
    }
    l = num / den / (float)n;
    if (dY)
      for (int j = 0; j < NO; ++j)
        dY[(size_t)s * NO + j] = 2.f * (Y[(size_t)s * NO + j] - T[(size_t)s * NO + j]) / den / (float)n;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (loss_sum && threadIdx.x % 32 == 0) atomicAdd(loss_sum, l);
}

// Adam (bias-corrected moments) over the FP32 master parameters; refreshes the BF16
// weight copy and clears the gradient it consumed.
__global__ void k_mlp_adam(int nw, int nbias, float* __restrict__ W, __nv_bfloat16* __restrict__ Wh,
                           float* __restrict__ bias, float* __restrict__ gW, float* __restrict__ gb,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nw + nbias) return;
  float* p = t < nw ? W + t : bias + (t - nw);
  float* g = t < nw ? gW + t : gb + (t - nw);
  const float gv = *g;
  const float mv = b1 * m[t] + (1.f - b1) * gv;
  const float vv = b2 * v[t] + (1.f - b2) * gv * gv;
  m[t] = mv;
  v[t] = vv;
  const float upd = lr * (mv / c1) / (sqrtf(vv / c2) + eps);
  const float np = *p - upd;
  *p = np;
  if (t < nw) Wh[t] = __float2bfloat16_rn(np);
  *g = 0.f;
}

template <class TA_, class TB_, bool TA, bool TB, int EPI>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, const TA_* A, int lda, const TB_* B, int ldb, float* C,
                 int ldc, const float* bias, float* Z, const float* mask, int splits = 1) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
  const int nz = (K + kchunk - 1) / kchunk;
  dim3 grid((N + 63) / 64, (M + 63) / 64, nz);
  k_mlp_gemm<TA_, TB_, TA, TB, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, mask, kchunk);
  return cudaGetLastError();
}

// Rows perm[i0 .. i0 + nb) of X (64 wide) and T (25 wide) into contiguous batch buffers.
__global__ void k_gather_batch(const int* __restrict__ perm, int i0, int nb, const float* __restrict__ X,
                               const float* __restrict__ T, float* __restrict__ Xb, float* __restrict__ Tb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * (NI + NO)) return;
  const int r = t / (NI + NO), c = t % (NI + NO);
  const long long src = __ldg(perm + i0 + r);
  if (c < NI) Xb[(long long)r * NI + c] = X[src * NI + c];
  else Tb[(long long)r * NO + c - NI] = T[src * NO + c - NI];
}

__global__ void k_to_bf16(const float* __restrict__ W, __nv_bfloat16* __restrict__ Wh, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) Wh[t] = __float2bfloat16_rn(W[t]);
}

// splitmix64 step (Steele, Lea and Flood 2014): the shuffles' random stream.
uint64_t splitmix64_next(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

constexpr char kMlpMagic[8] = {'S', 'C', 'M', 'L', 'P', '0', '0', '1'};

}  // namespace

namespace sc {

// Inference: Y = net(X) with the hidden activations in h1, h2 (n x 256 each).
cudaError_t mlp_forward(cudaStream_t st, const uint16_t* Wbf16, const float* bias, const float* X, int n, float* Y,
                        float* h1, float* h2) {
  const __nv_bfloat16* W = reinterpret_cast<const __nv_bfloat16*>(Wbf16);
  cudaError_t e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS_RELU>(st, n, NH, NI, X, NI, W, NI, h1, NH, bias,
                                                                         nullptr, nullptr);
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS_RELU>(st, n, NH, NH, h1, NH, W + OFF_W2, NH, h2, NH,
                                                               bias + OFF_B2, nullptr, nullptr);
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS>(st, n, NO, NH, h2, NH, W + OFF_W3, NH, Y, NO, bias + OFF_B3,
                                                          nullptr, nullptr);
  return e;
}

}  // namespace sc

extern "C" {

sc_status sc_mlp_forward(const uint16_t* Wbf16, const float* bias, const float* X, int n, float* Y, float* cache,
                         void* cuda_stream) {
  if (!Wbf16 || !bias || !X || !Y || n < 0) return SC_ERR_ARG;
  if (n == 0) return SC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const __nv_bfloat16* W = reinterpret_cast<const __nv_bfloat16*>(Wbf16);
  // cache: [z1 | h1 | z2 | h2], each n x 256 (pre- and post-activations)
  float* z1 = cache;
  float* h1 = cache ? cache + (size_t)n * NH : nullptr;
  float* z2 = cache ? cache + 2 * (size_t)n * NH : nullptr;
  float* h2 = cache ? cache + 3 * (size_t)n * NH : nullptr;
  float* tmp1 = nullptr;
  float* tmp2 = nullptr;
  cudaError_t e = cudaSuccess;
  if (!cache) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&tmp1), (size_t)n * NH * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&tmp2), (size_t)n * NH * sizeof(float), st);
    if (e != cudaSuccess) return SC_ERR_OOM;
    h1 = tmp1;
    h2 = tmp2;
  }
  e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS_RELU>(st, n, NH, NI, X, NI, W, NI, h1, NH, bias, z1, nullptr);
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS_RELU>(st, n, NH, NH, h1, NH, W + OFF_W2, NH, h2, NH,
                                                               bias + OFF_B2, z2, nullptr);
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS>(st, n, NO, NH, h2, NH, W + OFF_W3, NH, Y, NO, bias + OFF_B3,
                                                          nullptr, nullptr);
  if (tmp1) cudaFreeAsync(tmp1, st);
  if (tmp2) cudaFreeAsync(tmp2, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

sc_status sc_mlp_backward(const uint16_t* Wbf16, const float* X, const float* cache, const float* dY, int n,
                          float* gW, float* gb, float* work, void* cuda_stream) {
  if (!Wbf16 || !X || !cache || !dY || !gW || !gb || !work || n <= 0) return SC_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const __nv_bfloat16* W = reinterpret_cast<const __nv_bfloat16*>(Wbf16);
  const float* z1 = cache;
  const float* h1 = cache + (size_t)n * NH;
  const float* z2 = cache + 2 * (size_t)n * NH;
  const float* h2 = cache + 3 * (size_t)n * NH;
  float* dz2 = work;                      // n x 256
  float* dz1 = work + (size_t)n * NH;     // n x 256
  const int splits = (n + 2047) / 2048;   // sample chunks of the weight gradients
  cudaError_t e;
  // layer 3: gW3 += dY^T h2, gb3 += colsum dY, dz2 = (dY W3) * [z2 > 0]
  e = gemm<float, float, true, false, EPI_ATOMIC>(st, NO, NH, n, dY, NO, h2, NH, gW + OFF_W3, NH, nullptr, nullptr,
                                                  nullptr, splits);
  if (e == cudaSuccess) { k_mlp_colsum<<<NO, 256, 0, st>>>(n, NO, dY, gb + OFF_B3); e = cudaGetLastError(); }
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16, false, false, EPI_MASK>(st, n, NH, NO, dY, NO, W + OFF_W3, NH, dz2, NH, nullptr,
                                                           nullptr, z2);
  // layer 2
  if (e == cudaSuccess)
    e = gemm<float, float, true, false, EPI_ATOMIC>(st, NH, NH, n, dz2, NH, h1, NH, gW + OFF_W2, NH, nullptr, nullptr,
                                                    nullptr, splits);
  if (e == cudaSuccess) { k_mlp_colsum<<<NH, 256, 0, st>>>(n, NH, dz2, gb + OFF_B2); e = cudaGetLastError(); }
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16, false, false, EPI_MASK>(st, n, NH, NH, dz2, NH, W + OFF_W2, NH, dz1, NH, nullptr,
                                                           nullptr, z1);
  // layer 1
  if (e == cudaSuccess)
    e = gemm<float, float, true, false, EPI_ATOMIC>(st, NH, NI, n, dz1, NH, X, NI, gW, NI, nullptr, nullptr, nullptr,
                                                    splits);
  if (e == cudaSuccess) { k_mlp_colsum<<<NH, 256, 0, st>>>(n, NH, dz1, gb); e = cudaGetLastError(); }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

sc_status sc_mlp_loss(const float* Y, const float* T, int n, float* dY, float* loss_sum, void* cuda_stream) {
  if (!Y || !T || n <= 0) return SC_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_mlp_loss<<<(n + 255) / 256, 256, 0, st>>>(n, Y, T, dY, loss_sum);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

sc_status sc_mlp_adam(float* W, uint16_t* Wbf16, float* bias, float* gW, float* gb, float* m, float* v, int step,
                      float lr, void* cuda_stream) {
  if (!W || !Wbf16 || !bias || !gW || !gb || !m || !v || step < 1) return SC_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  const int tot = N_W + N_B;
  k_mlp_adam<<<(tot + 255) / 256, 256, 0, st>>>(N_W, N_B, W, reinterpret_cast<__nv_bfloat16*>(Wbf16), bias, gW, gb,
                                                 m, v, lr, b1, b2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

sc_status sc_mlp_bf16(const float* W, uint16_t* Wbf16, int n, void* cuda_stream) {
  if (!W || !Wbf16 || n < 0) return SC_ERR_ARG;
  if (n == 0) return SC_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(W, reinterpret_cast<__nv_bfloat16*>(Wbf16), n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

sc_status sc_mlp_train(float* W, uint16_t* Wbf16, float* bias, float* m, float* v, int* step, const float* X,
                       const float* T, int n, int epochs, int batch, float lr, uint64_t seed, float* loss_hist,
                       void* cuda_stream) {
  if (!W || !Wbf16 || !bias || !m || !v || !step || !X || !T || n < 1 || epochs < 0 || batch < 1 || *step < 0)
    return SC_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int bmax = batch < n ? batch : n;
  float *gW = nullptr, *gb = nullptr, *cache = nullptr, *work = nullptr, *Y = nullptr, *dY = nullptr;
  float *Xb = nullptr, *Tb = nullptr, *acc = nullptr;
  int* perm = nullptr;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(cudaMalloc(&gW, (size_t)N_W * sizeof(float))); A(cudaMalloc(&gb, (size_t)N_B * sizeof(float)));
  A(cudaMalloc(&cache, (size_t)4 * bmax * NH * sizeof(float))); A(cudaMalloc(&work, (size_t)2 * bmax * NH * sizeof(float)));
  A(cudaMalloc(&Y, (size_t)bmax * NO * sizeof(float))); A(cudaMalloc(&dY, (size_t)bmax * NO * sizeof(float)));
  A(cudaMalloc(&Xb, (size_t)bmax * NI * sizeof(float))); A(cudaMalloc(&Tb, (size_t)bmax * NO * sizeof(float)));
  A(cudaMalloc(&acc, sizeof(float))); A(cudaMalloc(&perm, (size_t)n * sizeof(int)));
  sc_status s = e == cudaSuccess ? SC_OK : SC_ERR_OOM;
  if (s == SC_OK) {
    A(cudaMemsetAsync(gW, 0, (size_t)N_W * sizeof(float), st));
    A(cudaMemsetAsync(gb, 0, (size_t)N_B * sizeof(float), st));
    if (e != cudaSuccess) s = SC_ERR_CUDA;
  }
  std::vector<int> hp(n);
  uint64_t rs = seed;
  const int nbatch = (n + bmax - 1) / bmax;
  for (int ep = 0; ep < epochs && s == SC_OK; ++ep) {
    // Fisher-Yates shuffle of all samples: batches mix systems, elements and nodes
    for (int i = 0; i < n; ++i) hp[i] = i;
    for (int i = n - 1; i > 0; --i) {
      const int j = (int)(splitmix64_next(rs) % (uint64_t)(i + 1));
      std::swap(hp[i], hp[j]);
    }
    A(cudaMemcpyAsync(perm, hp.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st));
    A(cudaMemsetAsync(acc, 0, sizeof(float), st));
    if (e != cudaSuccess) { s = SC_ERR_CUDA; break; }
    for (int b = 0; b < nbatch && s == SC_OK; ++b) {
      const int i0 = b * bmax, nb = (n - i0) < bmax ? (n - i0) : bmax;
      k_gather_batch<<<(nb * (NI + NO) + 255) / 256, 256, 0, st>>>(perm, i0, nb, X, T, Xb, Tb);
      if (cudaGetLastError() != cudaSuccess) { s = SC_ERR_CUDA; break; }
      s = sc_mlp_forward(Wbf16, bias, Xb, nb, Y, cache, st);
      if (s == SC_OK) s = sc_mlp_loss(Y, Tb, nb, dY, acc, st);
      if (s == SC_OK) s = sc_mlp_backward(Wbf16, Xb, cache, dY, nb, gW, gb, work, st);
      if (s == SC_OK) s = sc_mlp_adam(W, Wbf16, bias, gW, gb, m, v, ++*step, lr, st);
    }
    if (s == SC_OK && loss_hist) {
      float a = 0.f;
      if (cudaMemcpyAsync(&a, acc, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) s = SC_ERR_CUDA;
      loss_hist[ep] = a / (float)nbatch;
    }
  }
  cudaFree(gW); cudaFree(gb); cudaFree(cache); cudaFree(work); cudaFree(Y); cudaFree(dY); cudaFree(Xb); cudaFree(Tb);
  cudaFree(acc); cudaFree(perm);
  return s;
}

sc_status sc_mlp_save(const char* path, const float* W, const float* bias) {
  if (!path || !W || !bias) return SC_ERR_ARG;
  std::vector<float> hw(N_W), hb(N_B);
  if (cudaMemcpy(hw.data(), W, (size_t)N_W * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hb.data(), bias, (size_t)N_B * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SC_ERR_CUDA;
  FILE* f = std::fopen(path, "wb");
  if (!f) return SC_ERR_ARG;
  const int32_t counts[2] = {N_W, N_B};
  bool ok = std::fwrite(kMlpMagic, 1, 8, f) == 8 && std::fwrite(counts, sizeof(int32_t), 2, f) == 2 &&
            std::fwrite(hw.data(), sizeof(float), N_W, f) == (size_t)N_W &&
            std::fwrite(hb.data(), sizeof(float), N_B, f) == (size_t)N_B;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SC_OK : SC_ERR_ARG;
}

sc_status sc_mlp_load(const char* path, float* W, uint16_t* Wbf16, float* bias) {
  if (!path || !W || !Wbf16 || !bias) return SC_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return SC_ERR_ARG;
  char magic[8];
  int32_t counts[2] = {0, 0};
  std::vector<float> hw(N_W), hb(N_B);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMlpMagic, 8) == 0 &&
            std::fread(counts, sizeof(int32_t), 2, f) == 2 && counts[0] == N_W && counts[1] == N_B &&
            std::fread(hw.data(), sizeof(float), N_W, f) == (size_t)N_W &&
            std::fread(hb.data(), sizeof(float), N_B, f) == (size_t)N_B;
  std::fclose(f);
  if (!ok) return SC_ERR_ARG;
  if (cudaMemcpy(W, hw.data(), (size_t)N_W * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(bias, hb.data(), (size_t)N_B * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return SC_ERR_CUDA;
  return sc_mlp_bf16(W, Wbf16, N_W, nullptr);
}

}  // extern "C"
