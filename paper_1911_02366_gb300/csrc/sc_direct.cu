// Direct solves of the Newton system by dense LU on the GPU (Sec. 4): the global Jacobian
// A, or the condensed matrix S of Sec. 2.2 (eq. SC_step1) followed by the back-substitution
// of eq. SC_step2 -- the two paths whose factorisation and per-solve costs the paper compares
// (Tables tab:Advantages and tab:Advantages2; it uses a sparse direct solver on the CPU).
//
// Forming the dense matrices: A from the own element blocks and the neighbour couplings
// (scatter); S column by column through the condensed operator (S e_j), the system the
// condensation forms.  LU with partial pivoting (the first row of largest |a| wins), right
// looking in panels of 64 columns:
//   per column j of a panel: pivot search (block partial maxima, then one block), the row
//   interchange over the whole row, scaling of column j and the rank-1 update of the rest of
//   the panel;
//   per panel: U12 = L11^-1 A12 (unit lower triangle in shared memory, 32-column tiles), then
//   the trailing update A22 -= L21 U12 on the TF32 tensor cores (mixed arm, tensor_cores) or
//   the CUDA cores (64 x 64 tiles; FP64 on the FP64 arm).
// Solves: the row interchanges as one gather, then blocked forward and backward
// substitution (64-row blocks: off-diagonal dot products by 32 warps, the 64 x 64 triangle
// by one warp).  The mixed arm stores the factors in FP32 and refines in FP64 on the global
// residual B - A dQ until rel_tol.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sc_internal.cuh"

namespace {

#define DC_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess) { c->err = std::string(#call) + ": " + cudaGetErrorString(_e); return SC_ERR_CUDA; } \
  } while (0)

constexpr int kPanel = 64;
constexpr int kPivBlocks = 152;

inline unsigned cdivu(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ---- dense global matrix ------------------------------------------------------------
template <class T>
__global__ void k_dense_own(Geo G, const double* __restrict__ Aown, const int* __restrict__ perm, T* __restrict__ D,
                            long long ldd) {
  const long long ne = G.ne;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)G.K * ne * ne) return;
  const int e = (int)(t / (ne * ne));
  const int r = (int)((t / ne) % ne), cc = (int)(t % ne);
  const int j = r / 5, k = r % 5, m = cc / 5, l = cc % 5;
  const double v = Aown[(size_t)e * own_stride(G) + (size_t)(5 * __ldg(perm + j) + k) * G.lda +
                        own_col(G, __ldg(perm + m), l)];
  D[((long long)e * ne + r) * ldd + (long long)e * ne + cc] = (T)v;
}

// Neighbour couplings X[e][k][pair][l] added at (row node of the pair, its neighbour's column
// node); atomics, because on small periodic meshes several slots name the same element.
template <class T>
__global__ void k_dense_cross(Geo G, const double* __restrict__ X, const int* __restrict__ nbr,
                              const int* __restrict__ prow, const int* __restrict__ pslot,
                              const int* __restrict__ pcol, T* __restrict__ D, long long ldd) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long per = (long long)G.NP * 25;
  if (t >= (long long)G.K * per) return;
  const int e = (int)(t / per);
  const int rem = (int)(t % per);
  const int k = rem / (G.NP * 5), p = (rem / 5) % G.NP, l = rem % 5;
  const long long row = (long long)e * G.ne + 5 * __ldg(prow + p) + k;
  const long long col = (long long)__ldg(nbr + e * 18 + __ldg(pslot + p)) * G.ne + 5 * __ldg(pcol + p) + l;
  atomicAdd(&D[row * ldd + col], (T)X[(size_t)e * per + ((size_t)k * G.NP + p) * 5 + l]);
}

__global__ void k_unit_vec(double* x, long long on, long long off) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (off >= 0) x[off] = 0.0;
    x[on] = 1.0;
  }
}

// D[:, j] = col (n entries).
template <class T>
__global__ void k_put_column(const double* __restrict__ col, int n, int j, T* __restrict__ D, long long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) D[(long long)i * ldd + j] = (T)col[i];
}

// ---- LU with partial pivoting -------------------------------------------------------
// Pivot search in column j, rows j..n-1: every block leaves its largest |a| and the first row
// holding it; the final block reduces the partials (ties: the smaller row).
template <class T>
__global__ void k_piv_partial(const T* __restrict__ D, long long ldd, int n, int j, double* __restrict__ pval,
                              int* __restrict__ prow) {
  __shared__ double sv[256];
  __shared__ int sr[256];
  double best = -1.0;
  int brow = n;
  for (int r = j + blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const double a = fabs((double)D[(long long)r * ldd + j]);
    if (a > best) { best = a; brow = r; }
  }
  sv[threadIdx.x] = best;
  sr[threadIdx.x] = brow;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double ov = sv[threadIdx.x + s];
      const int orow = sr[threadIdx.x + s];
      if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && orow < sr[threadIdx.x])) {
        sv[threadIdx.x] = ov;
        sr[threadIdx.x] = orow;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { pval[blockIdx.x] = sv[0]; prow[blockIdx.x] = sr[0]; }
}

__global__ void k_piv_final(int nparts, const double* __restrict__ pval, const int* __restrict__ prow, int j,
                            int* __restrict__ piv, int* __restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double best = -1.0;
  int brow = -1;
  for (int b = 0; b < nparts; ++b)
    if (pval[b] > best || (pval[b] == best && prow[b] < brow)) { best = pval[b]; brow = prow[b]; }
  if (!(best > 0.0)) {  // zero (or NaN) column: record the first such column, keep the row
    if (status[0] < 0) status[0] = j;
    brow = j;
  }
  piv[j] = brow;
}

// Interchange rows j and piv[j] over all n columns.
template <class T>
__global__ void k_swap_rows(T* __restrict__ D, long long ldd, int n, int j, const int* __restrict__ piv) {
  const int p = piv[j];
  if (p == j) return;
  for (int cc = blockIdx.x * blockDim.x + threadIdx.x; cc < n; cc += gridDim.x * blockDim.x) {
    const T a = D[(long long)j * ldd + cc];
    D[(long long)j * ldd + cc] = D[(long long)p * ldd + cc];
    D[(long long)p * ldd + cc] = a;
  }
}

// Column j below the diagonal divided by the pivot, then the rank-1 update of the panel
// columns j+1 .. jend-1; one thread per row (the pivot row is only read).
template <class T>
__global__ void k_panel_col(T* __restrict__ D, long long ldd, int n, int j, int jend) {
  const T pivot = D[(long long)j * ldd + j];
  if (pivot == T(0)) return;
  const T inv = T(1) / pivot;
  for (int r = j + 1 + blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    T* row = D + (long long)r * ldd;
    const T l = row[j] * inv;
    row[j] = l;
    for (int cc = j + 1; cc < jend; ++cc) row[cc] -= l * D[(long long)j * ldd + cc];
  }
}

// U12 = L11^-1 A12 for columns >= k0 + kb: one CTA per 32-column tile, L11 (unit lower,
// kb <= 64) and the tile in shared memory, one barrier per eliminated row.
constexpr int kLdL = kPanel + 1, kLdT = 33;
template <class T>
constexpr size_t trsm_smem() { return (size_t)(kPanel * kLdL + kPanel * kLdT) * sizeof(T); }

template <class T>
__global__ void __launch_bounds__(256) k_trsm_panel(T* __restrict__ D, long long ldd, int n, int k0, int kb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* L = reinterpret_cast<T*>(smem_raw);  // kPanel x kLdL
  T* tile = L + kPanel * kLdL;            // kPanel x kLdT
  const int c0 = k0 + kb + blockIdx.x * 32;
  for (int i = threadIdx.x; i < kb * kb; i += blockDim.x) {
    const int r = i / kb, cc = i % kb;
    L[r * kLdL + cc] = D[(long long)(k0 + r) * ldd + k0 + cc];
  }
  for (int i = threadIdx.x; i < kb * 32; i += blockDim.x) {
    const int r = i / 32, cc = i % 32;
    tile[r * kLdT + cc] = c0 + cc < n ? D[(long long)(k0 + r) * ldd + c0 + cc] : T(0);
  }
  __syncthreads();
  for (int i = 0; i < kb - 1; ++i) {
    for (int q = threadIdx.x; q < (kb - 1 - i) * 32; q += blockDim.x) {
      const int r = i + 1 + q / 32, cc = q % 32;
      tile[r * kLdT + cc] -= L[r * kLdL + i] * tile[i * kLdT + cc];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kb * 32; i += blockDim.x) {
    const int r = i / 32, cc = i % 32;
    if (c0 + cc < n) D[(long long)(k0 + r) * ldd + c0 + cc] = tile[r * kLdT + cc];
  }
}

// ---- triangular solves --------------------------------------------------------------
// y[i] = b[perm[i]] in the factor precision.
template <class T>
__global__ void k_permute_in(int n, const int* __restrict__ perm, const double* __restrict__ b, T* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (T)b[perm[i]];
}

template <class T>
__global__ void k_to_double(int n, const T* __restrict__ y, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (double)y[i];
}

// One 64-row block of a substitution in place on y: LOWER (unit diagonal, columns left of
// the block) or upper (diagonal of U, columns right of it).  32 warps form the off-diagonal
// dot products of the block's rows, then warp 0 solves the 64 x 64 triangle.
template <class T, bool LOWER>
__global__ void __launch_bounds__(1024) k_trsv_block(const T* __restrict__ D, long long ldd, int n, int b0, int bs,
                                                     T* __restrict__ y) {
  __shared__ T s[kPanel];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c_lo = LOWER ? 0 : b0 + bs, c_hi = LOWER ? b0 : n;
  for (int r = warp; r < bs; r += 32) {
    const T* row = D + (long long)(b0 + r) * ldd;
    T acc = T(0);
    for (int cc = c_lo + lane; cc < c_hi; cc += 32) acc += row[cc] * y[cc];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s[r] = y[b0 + r] - acc;
  }
  __syncthreads();
  if (warp != 0) return;
  // the triangle: lanes own rows lane and lane + 32 of the block
  T v0 = lane < bs ? s[lane] : T(0), v1 = lane + 32 < bs ? s[lane + 32] : T(0);
  if (LOWER) {
    for (int i = 0; i < bs; ++i) {
      const T xi = __shfl_sync(0xffffffffu, i < 32 ? v0 : v1, i & 31);
      const int r0 = lane, r1 = lane + 32;
      if (r0 > i && r0 < bs) v0 -= D[(long long)(b0 + r0) * ldd + b0 + i] * xi;
      if (r1 > i && r1 < bs) v1 -= D[(long long)(b0 + r1) * ldd + b0 + i] * xi;
    }
  } else {
    for (int i = bs - 1; i >= 0; --i) {
      T xi = __shfl_sync(0xffffffffu, i < 32 ? v0 : v1, i & 31);
      xi = xi / D[(long long)(b0 + i) * ldd + b0 + i];
      if (lane == (i & 31)) { if (i < 32) v0 = xi; else v1 = xi; }
      const int r0 = lane, r1 = lane + 32;
      if (r0 < i) v0 -= D[(long long)(b0 + r0) * ldd + b0 + i] * xi;
      if (r1 < i) v1 -= D[(long long)(b0 + r1) * ldd + b0 + i] * xi;
    }
  }
  if (lane < bs) y[b0 + lane] = v0;
  if (lane + 32 < bs) y[b0 + lane + 32] = v1;
}

template <class T>
cudaError_t lu_factor(sc_ctx* c, T* D, long long ldd, int n, int* piv, bool tc) {
  double* pval = nullptr;
  int* prow = nullptr;
  cudaError_t e = cudaMalloc(&pval, kPivBlocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&prow, kPivBlocks * sizeof(int));
  for (int k0 = 0; k0 < n && e == cudaSuccess; k0 += kPanel) {
    const int kb = std::min(kPanel, n - k0), jend = k0 + kb;
    for (int j = k0; j < jend && e == cudaSuccess; ++j) {
      const int rows = n - j;
      const int pb = std::min<int>(kPivBlocks, (int)cdivu(rows, 256));
      count_launch(c, 4);
      k_piv_partial<T><<<pb, 256, 0, c->stream>>>(D, ldd, n, j, pval, prow);
      k_piv_final<<<1, 32, 0, c->stream>>>(pb, pval, prow, j, piv, c->d_status);
      k_swap_rows<T><<<std::min<unsigned>(cdivu(n, 256), 1024), 256, 0, c->stream>>>(D, ldd, n, j, piv);
      k_panel_col<T><<<std::min<unsigned>(cdivu(rows, 256), 4 * 152), 256, 0, c->stream>>>(D, ldd, n, j, jend);
      e = cudaGetLastError();
    }
    const int rest = n - jend;
    if (rest <= 0 || e != cudaSuccess) continue;
    count_launch(c);
    e = cudaFuncSetAttribute(k_trsm_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem<T>());
    if (e != cudaSuccess) break;
    k_trsm_panel<T><<<cdivu(rest, 32), 256, trsm_smem<T>(), c->stream>>>(D, ldd, n, k0, kb);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    T* A21 = D + (long long)jend * ldd + k0;
    const T* U12 = D + (long long)k0 * ldd + jend;
    T* A22 = D + (long long)jend * ldd + jend;
    if constexpr (std::is_same<T, float>::value) {
      if (tc) {
        count_launch(c);
        e = sc::gemm_tf32(c->stream, rest, rest, kb, -1.0f, A21, 0, (int)ldd, false, U12, 0, (int)ldd, false, 1.0f, A22,
                          0, (int)ldd, 1, c->d_status);
        continue;
      }
    }
    e = sc::gemm_update<T>(c, rest, rest, kb, A21, (int)ldd, U12, (int)ldd, A22, (int)ldd);
  }
  cudaFree(pval);
  cudaFree(prow);
  return e;
}

// x = A^-1 b with the factors (row interchanges piv applied through perm); y: n scratch.
template <class T>
cudaError_t lu_solve_dense(sc_ctx* c, const T* D, long long ldd, int n, const int* perm, const double* b, T* y,
                           double* x) {
  count_launch(c);
  k_permute_in<T><<<cdivu(n, 256), 256, 0, c->stream>>>(n, perm, b, y);
  for (int b0 = 0; b0 < n; b0 += kPanel) {
    count_launch(c);
    k_trsv_block<T, true><<<1, 1024, 0, c->stream>>>(D, ldd, n, b0, std::min(kPanel, n - b0), y);
  }
  const int last = ((n - 1) / kPanel) * kPanel;
  for (int b0 = last; b0 >= 0; b0 -= kPanel) {
    count_launch(c);
    k_trsv_block<T, false><<<1, 1024, 0, c->stream>>>(D, ldd, n, b0, std::min(kPanel, n - b0), y);
  }
  count_launch(c);
  k_to_double<T><<<cdivu(n, 256), 256, 0, c->stream>>>(n, y, x);
  return cudaGetLastError();
}

void free_direct(sc_ctx* c) {
  if (c->Dlu) cudaFree(c->Dlu);
  if (c->d_dpiv) cudaFree(c->d_dpiv);
  if (c->Dcorr) cudaFree(c->Dcorr);
  c->Dlu = nullptr;
  c->d_dpiv = nullptr;
  c->Dcorr = nullptr;
  c->direct_valid = false;
  c->direct_n = c->direct_ld = 0;
  c->direct_which = -1;
}

template <class T>
sc_status direct_factor_t(sc_ctx* c, int which, double* ms_form, double* ms_factor) {
  const Geo& G = c->G;
  const int n = which == SC_DIRECT_GLOBAL ? G.K * G.ne : G.K * G.nb;
  const long long ldd = (n + 3) & ~3;  // 16-byte aligned rows for the tensor-core update
  free_direct(c);
  if ((double)n * ldd * sizeof(T) > 64e9) {
    c->err = "direct: the dense matrix would exceed 64 GB";
    return SC_ERR_ARG;
  }
  DC_CUDA(cudaMalloc(&c->Dlu, (size_t)n * ldd * sizeof(T)));
  DC_CUDA(cudaMalloc(&c->d_dpiv, (size_t)n * sizeof(int)));
  DC_CUDA(cudaMalloc(&c->Dcorr, (size_t)G.K * G.ne * sizeof(double)));  // a sweep's correction
  T* D = static_cast<T*>(c->Dlu);
  cudaEvent_t ev[3];
  for (auto& x : ev) DC_CUDA(cudaEventCreate(&x));
  struct Evs { cudaEvent_t* v; ~Evs() { for (int i = 0; i < 3; ++i) cudaEventDestroy(v[i]); } } evg{ev};
  const int minus1 = -1;
  DC_CUDA(cudaMemcpyAsync(c->d_status, &minus1, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  DC_CUDA(cudaEventRecord(ev[0], c->stream));
  DC_CUDA(cudaMemsetAsync(D, 0, (size_t)n * ldd * sizeof(T), c->stream));
  if (which == SC_DIRECT_GLOBAL) {
    count_launch(c, 2);
    const long long nown = (long long)G.K * G.ne * G.ne, ncross = (long long)G.K * G.NP * 25;
    k_dense_own<T><<<cdivu(nown, 256), 256, 0, c->stream>>>(G, c->Aown, c->d_perm, D, ldd);
    k_dense_cross<T><<<cdivu(ncross, 256), 256, 0, c->stream>>>(G, c->X, c->d_nbr, c->d_prow, c->d_pslot, c->d_pcol,
                                                                 D, ldd);
    DC_CUDA(cudaGetLastError());
  } else {
    // S e_j through the condensed operator, the system the condensation forms
    double* xb = c->Xfull;  // K ne >= n doubles of scratch
    double* col = c->Rfull;
    DC_CUDA(cudaMemsetAsync(xb, 0, (size_t)n * sizeof(double), c->stream));
    for (int j = 0; j < n; ++j) {
      count_launch(c);
      k_unit_vec<<<1, 32, 0, c->stream>>>(xb, j, j - 1);
      if (c->cfg.precision == SC_PREC_MIXED) {
        DC_CUDA(sc::vec_to_float(c, c->Xbf, xb, (size_t)n));
        DC_CUDA(sc::cond_interior32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf));
        DC_CUDA(sc::cond_boundary32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf, col));
      } else {
        DC_CUDA(sc::cond_interior(c, xb, 1.0, nullptr, 0.0, c->Ui));
        DC_CUDA(sc::cond_boundary(c, xb, 1.0, nullptr, 0.0, c->Ui, col));
      }
      count_launch(c);
      k_put_column<T><<<cdivu(n, 256), 256, 0, c->stream>>>(col, n, j, D, ldd);
    }
    DC_CUDA(cudaGetLastError());
  }
  DC_CUDA(cudaEventRecord(ev[1], c->stream));
  DC_CUDA(lu_factor<T>(c, D, ldd, n, c->d_dpiv, c->cfg.precision == SC_PREC_MIXED && c->cfg.tensor_cores));
  DC_CUDA(cudaEventRecord(ev[2], c->stream));
  int bad = -1;
  DC_CUDA(cudaMemcpyAsync(&bad, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DC_CUDA(cudaStreamSynchronize(c->stream));
  float t01 = 0.f, t12 = 0.f;
  DC_CUDA(cudaEventElapsedTime(&t01, ev[0], ev[1]));
  DC_CUDA(cudaEventElapsedTime(&t12, ev[1], ev[2]));
  if (ms_form) *ms_form = t01;
  if (ms_factor) *ms_factor = t12;
  if (bad == SC_TC_TIMEOUT) { c->err = "direct: tensor-core wait timed out"; return SC_ERR_CUDA; }
  if (bad >= 0) { c->err = "direct: zero pivot in column " + std::to_string(bad); return SC_ERR_SINGULAR_BLOCK; }
  // the interchanges as one permutation (row i of P b is b[perm[i]])
  std::vector<int> piv(n), perm(n);
  DC_CUDA(cudaMemcpy(piv.data(), c->d_dpiv, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int j = 0; j < n; ++j) std::swap(perm[j], perm[piv[j]]);
  DC_CUDA(cudaMemcpy(c->d_dpiv, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice));
  c->direct_n = n;
  c->direct_ld = (int)ldd;
  c->direct_which = which;
  c->direct_valid = true;
  return SC_OK;
}

// d = A^-1 r with the dense factors (global, or condensed rhs + LU(S) + back-substitution).
template <class T>
sc_status direct_apply_t(sc_ctx* c, const double* r, double* d, float* ms_lu, float* ms_cond) {
  const Geo& G = c->G;
  const int n = c->direct_n;
  const T* D = static_cast<const T*>(c->Dlu);
  const bool mixed = c->cfg.precision == SC_PREC_MIXED;
  T* y = nullptr;
  DC_CUDA(cudaMalloc(&y, (size_t)n * sizeof(T)));
  struct Free { void* p; ~Free() { cudaFree(p); } } fy{y};
  cudaEvent_t ev[4];
  for (auto& x : ev) DC_CUDA(cudaEventCreate(&x));
  struct Evs { cudaEvent_t* v; ~Evs() { for (int i = 0; i < 4; ++i) cudaEventDestroy(v[i]); } } evg{ev};
  DC_CUDA(cudaEventRecord(ev[0], c->stream));
  if (c->direct_which == SC_DIRECT_GLOBAL) {
    DC_CUDA(cudaEventRecord(ev[1], c->stream));
    DC_CUDA(lu_solve_dense<T>(c, D, c->direct_ld, n, c->d_dpiv, r, y, d));
    DC_CUDA(cudaEventRecord(ev[2], c->stream));
    DC_CUDA(cudaEventRecord(ev[3], c->stream));
  } else {
    if (mixed) {  // g = B_b - A_bi A_ii^-1 B_i (eq. SC_step1)
      DC_CUDA(sc::cond_interior32(c, nullptr, 0.0, r, 1.0, c->Uf));
      DC_CUDA(sc::cond_boundary32(c, nullptr, 0.0, r, 1.0, c->Uf, c->Gb));
    } else {
      DC_CUDA(sc::cond_interior(c, nullptr, 0.0, r, 1.0, c->Ui));
      DC_CUDA(sc::cond_boundary(c, nullptr, 0.0, r, 1.0, c->Ui, c->Gb));
    }
    DC_CUDA(cudaEventRecord(ev[1], c->stream));
    DC_CUDA(lu_solve_dense<T>(c, D, c->direct_ld, n, c->d_dpiv, c->Gb, y, c->Xb));
    DC_CUDA(cudaEventRecord(ev[2], c->stream));
    if (mixed) {  // Q_i = A_ii^-1 (B_i - A_ib Q_b) (eq. SC_step2)
      DC_CUDA(sc::vec_to_float(c, c->Xbf, c->Xb, (size_t)n));
      DC_CUDA(sc::cond_interior32(c, c->Xbf, -1.0, r, 1.0, c->Uf));
      DC_CUDA(sc::scatter_solution32(c, c->Xb, c->Uf, d));
    } else {
      DC_CUDA(sc::cond_interior(c, c->Xb, -1.0, r, 1.0, c->Ui));
      DC_CUDA(sc::scatter_solution(c, c->Xb, c->Ui, d));
    }
    DC_CUDA(cudaEventRecord(ev[3], c->stream));
  }
  DC_CUDA(cudaEventSynchronize(ev[3]));
  float a = 0.f, b = 0.f, cc = 0.f;
  DC_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
  DC_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
  DC_CUDA(cudaEventElapsedTime(&cc, ev[2], ev[3]));
  *ms_lu += b;
  *ms_cond += a + cc;
  (void)G;
  return SC_OK;
}

double dnorm(sc_ctx* c, const double* v, size_t n) {
  double* const hs = c->Hd + 2 * (c->restart_alloc + 1) + 2;
  sc::multidot(c, v, 1, n, v, hs);
  double h = 0.0;
  cudaMemcpyAsync(&h, hs, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return std::sqrt(h);
}

}  // namespace

namespace sc {
void free_direct_factors(sc_ctx* c) { free_direct(c); }
}  // namespace sc

extern "C" {

sc_status sc_direct_factor(sc_ctx* c, int which, double* ms_form, double* ms_factor) {
  if (!c || (which != SC_DIRECT_GLOBAL && which != SC_DIRECT_CONDENSED)) return SC_ERR_ARG;
  if (which == SC_DIRECT_GLOBAL && !c->assembled) { c->err = "direct_factor before assemble"; return SC_ERR_STATE; }
  if (which == SC_DIRECT_CONDENSED && !c->condensed) { c->err = "direct_factor before condense"; return SC_ERR_STATE; }
  if (c->cfg.precision == SC_PREC_MIXED) return direct_factor_t<float>(c, which, ms_form, ms_factor);
  return direct_factor_t<double>(c, which, ms_form, ms_factor);
}

sc_status sc_direct_solve(sc_ctx* c, double* dQ, int on_device, sc_solve_stats* st) {
  if (!c || !dQ) return SC_ERR_ARG;
  if (!c->direct_valid || !c->assembled || (c->direct_which == SC_DIRECT_CONDENSED && !c->condensed)) {
    c->err = "direct_solve without factors of the assembled system";
    return SC_ERR_STATE;
  }
  const Geo& G = c->G;
  const size_t dofs = (size_t)G.K * G.ne;
  const bool mixed = c->cfg.precision == SC_PREC_MIXED;
  double* x = on_device ? dQ : c->Xfull;
  sc_solve_stats S{};
  S.first_bad_element = -1;
  float ms_lu = 0.f, ms_cond = 0.f;
  const double bnorm = dnorm(c, c->B, dofs);
  const double target = c->cfg.rel_tol * bnorm;
  DC_CUDA(cudaMemsetAsync(x, 0, dofs * sizeof(double), c->stream));
  DC_CUDA(cudaMemcpyAsync(c->Rfull, c->B, dofs * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  double rn = bnorm;
  int sweeps = 0;
  const int max_sweeps = mixed ? std::max(1, c->cfg.max_refine) : 2;
  // x += A^-1 r, r = B - A x (FP64): one sweep on the FP64 arm (a second if rounding left the
  // residual above rel_tol), FP64 refinement of the FP32 factors on the mixed arm
  while (rn > target && sweeps < max_sweeps) {
    sc_status s = mixed ? direct_apply_t<float>(c, c->Rfull, c->Dcorr, &ms_lu, &ms_cond)
                        : direct_apply_t<double>(c, c->Rfull, c->Dcorr, &ms_lu, &ms_cond);
    if (s != SC_OK) return s;
    DC_CUDA(sc::vec_axpby(c, x, 1.0, c->Dcorr, 1.0, dofs));
    DC_CUDA(sc::global_apply(c, x, c->Rfull));
    DC_CUDA(sc::vec_axpby(c, c->Rfull, 1.0, c->B, -1.0, dofs));
    rn = dnorm(c, c->Rfull, dofs);
    ++sweeps;
    if (!std::isfinite(rn)) { c->err = "direct: non-finite residual"; return SC_ERR_NONFINITE; }
  }
  if (!on_device) DC_CUDA(cudaMemcpyAsync(dQ, x, dofs * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  DC_CUDA(cudaStreamSynchronize(c->stream));
  S.refinements = sweeps;
  S.rel_residual = bnorm > 0 ? rn / bnorm : 0.0;
  S.ms_gmres = ms_lu;   // the dense triangular solves
  S.ms_rhs = ms_cond;   // condensed right-hand sides and back-substitutions
  if (st) *st = S;
  if (S.rel_residual > c->cfg.rel_tol * 1.0000001 && bnorm > 0.0) {
    c->err = "direct: relative residual " + std::to_string(S.rel_residual) + " above tolerance";
    return SC_ERR_NOT_CONVERGED;
  }
  return SC_OK;
}

}  // extern "C"
