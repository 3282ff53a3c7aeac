// Condensed-operator application and Krylov vector kernels.
//
// The condensed operator (Sec. 2.2 eq. SC_step1, Sec. 3.2) is applied without ever
// forming S:  S x_b = A_bb x_b - A_bi (A_ii^-1 (A_ib x_b)).  Two element-parallel
// passes do it:
//   interior pass   u_e = A_ii,e^-1 ( alpha B_i,e + beta (A_ib x_b)_e )
//   boundary pass   y_e = gamma B_b,e + delta (A_bb x_b)_e - (A_bi u)_e
// where the own-element parts are dense row-major GEMVs on the stored element block and
// the neighbour parts run over the structured coupling list.  The same two passes give
// the condensed right-hand side (x_b = 0) and the back-substitution of eq. SC_step2.
#include "sc_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double s) {
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// Neighbour part of row (node j, variable k): sum over couplings of X * vec(neighbour).
// want_b / want_i select couplings whose column node is a boundary / interior node of
// the neighbour; vb / vi hold boundary / interior vectors (element-major).
__device__ __forceinline__ double cross_row(const Geo& G, int e, int j, int k, const double* __restrict__ X,
                                            const int* __restrict__ nbr, const int* __restrict__ pptr,
                                            const int* __restrict__ pids, const int* __restrict__ pslot,
                                            const int* __restrict__ pcol, const int* __restrict__ perm,
                                            const double* __restrict__ vb, const double* __restrict__ vi,
                                            int lane) {
  double s = 0.0;
  const int b = pptr[j], en = pptr[j + 1];
  for (int q = b + lane; q < en; q += 32) {
    const int pr = pids[q];
    const int nb = nbr[e * 18 + pslot[pr]];
    const int pos = perm[pcol[pr]];
    const double* xv;
    if (pos >= G.nin) {
      if (!vb) continue;
      xv = vb + (size_t)nb * G.nb + 5 * (pos - G.nin);
    } else {
      if (!vi) continue;
      xv = vi + (size_t)nb * G.ni + 5 * pos;
    }
    const double* blk = X + ((size_t)e * G.NP + pr) * 25 + k * 5;
    for (int l = 0; l < 5; ++l) s = fma(blk[l], xv[l], s);
  }
  return s;
}

__global__ void __launch_bounds__(256) k_cond_interior(Geo G, const double* __restrict__ Aown,
    const double* __restrict__ X, const double* __restrict__ Ainv, const int* __restrict__ nbr,
    const int* __restrict__ pptr, const int* __restrict__ pids, const int* __restrict__ pslot,
    const int* __restrict__ pcol, const int* __restrict__ perm, const int* __restrict__ iperm,
    const double* __restrict__ xb, double beta, const double* __restrict__ Bfull, double alpha,
    double* __restrict__ u) {
  extern __shared__ double sm[];
  double* t = sm;  // ni
  const int e = blockIdx.x, ni = G.ni, nb = G.nb, ne = G.ne;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const double* Ae = Aown + (size_t)e * ne * ne;
  for (int ri = warp; ri < ni; ri += nw) {
    const int j = iperm[ri / 5], k = ri % 5;
    double s = 0.0;
    if (xb) {
      const double* row = Ae + (size_t)ri * ne + ni;
      const double* xe = xb + (size_t)e * nb;
      for (int cc = lane; cc < nb; cc += 32) s = fma(row[cc], xe[cc], s);
      s += cross_row(G, e, j, k, X, nbr, pptr, pids, pslot, pcol, perm, xb, nullptr, lane);
      s = warp_sum(s);
    }
    if (lane == 0) {
      double v = beta * s;
      if (Bfull) v += alpha * Bfull[((size_t)e * G.nn + j) * 5 + k];
      t[ri] = v;
    }
  }
  __syncthreads();
  const double* Ie = Ainv + (size_t)e * ni * ni;
  for (int ri = warp; ri < ni; ri += nw) {
    double s = 0.0;
    for (int cc = lane; cc < ni; cc += 32) s = fma(Ie[(size_t)ri * ni + cc], t[cc], s);
    s = warp_sum(s);
    if (lane == 0) u[(size_t)e * ni + ri] = s;
  }
}

__global__ void __launch_bounds__(256) k_cond_boundary(Geo G, const double* __restrict__ Aown,
    const double* __restrict__ X, const int* __restrict__ nbr,
    const int* __restrict__ pptr, const int* __restrict__ pids, const int* __restrict__ pslot,
    const int* __restrict__ pcol, const int* __restrict__ perm, const int* __restrict__ iperm,
    const double* __restrict__ xb, double delta, const double* __restrict__ Bfull, double gamma_,
    const double* __restrict__ u, double* __restrict__ y) {
  const int e = blockIdx.x, ni = G.ni, nb = G.nb, ne = G.ne;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const double* Ae = Aown + (size_t)e * ne * ne;
  for (int rb = warp; rb < nb; rb += nw) {
    const int ri = ni + rb;
    const int j = iperm[ri / 5], k = ri % 5;
    const double* row = Ae + (size_t)ri * ne;
    double sb = 0.0, si = 0.0;
    if (xb) {
      const double* xe = xb + (size_t)e * nb;
      for (int cc = lane; cc < nb; cc += 32) sb = fma(row[ni + cc], xe[cc], sb);
      sb += cross_row(G, e, j, k, X, nbr, pptr, pids, pslot, pcol, perm, xb, nullptr, lane);
    }
    if (u) {
      const double* ue = u + (size_t)e * ni;
      for (int cc = lane; cc < ni; cc += 32) si = fma(row[cc], ue[cc], si);
      si += cross_row(G, e, j, k, X, nbr, pptr, pids, pslot, pcol, perm, nullptr, u, lane);
    }
    const double s = warp_sum(delta * sb - si);
    if (lane == 0) {
      double v = s;
      if (Bfull) v += gamma_ * Bfull[((size_t)e * G.nn + j) * 5 + k];
      y[(size_t)e * nb + rb] = v;
    }
  }
}

// y = A x on the full system, natural global dof order.
__global__ void __launch_bounds__(256) k_global_apply(Geo G, const double* __restrict__ Aown,
    const double* __restrict__ X, const int* __restrict__ nbr, const int* __restrict__ pptr,
    const int* __restrict__ pids, const int* __restrict__ pslot, const int* __restrict__ pcol,
    const int* __restrict__ iperm, const double* __restrict__ x, double* __restrict__ y) {
  extern __shared__ double sm[];
  double* xe = sm;  // ne, permuted order
  const int e = blockIdx.x, ne = G.ne, nn = G.nn;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  for (int t = threadIdx.x; t < ne; t += blockDim.x) {
    const int pos = t / 5, k = t % 5;
    xe[t] = x[((size_t)e * nn + iperm[pos]) * 5 + k];
  }
  __syncthreads();
  const double* Ae = Aown + (size_t)e * ne * ne;
  for (int ri = warp; ri < ne; ri += nw) {
    const int j = iperm[ri / 5], k = ri % 5;
    const double* row = Ae + (size_t)ri * ne;
    double s = 0.0;
    for (int cc = lane; cc < ne; cc += 32) s = fma(row[cc], xe[cc], s);
    const int b = pptr[j], en = pptr[j + 1];
    for (int q = b + lane; q < en; q += 32) {
      const int pr = pids[q];
      const int nbe = nbr[e * 18 + pslot[pr]];
      const double* xv = x + ((size_t)nbe * nn + pcol[pr]) * 5;
      const double* blk = X + ((size_t)e * G.NP + pr) * 25 + k * 5;
      for (int l = 0; l < 5; ++l) s = fma(blk[l], xv[l], s);
    }
    s = warp_sum(s);
    if (lane == 0) y[((size_t)e * nn + j) * 5 + k] = s;
  }
}

__global__ void k_scatter(Geo G, const int* __restrict__ iperm, const double* __restrict__ xb,
                          const double* __restrict__ xi, double* __restrict__ x) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)G.K * G.ne) return;
  const int e = (int)(t / G.ne), r = (int)(t % G.ne);
  const int pos = r / 5, k = r % 5;
  const double v = pos < G.nin ? xi[(size_t)e * G.ni + r] : xb[(size_t)e * G.nb + r - G.ni];
  x[((size_t)e * G.nn + iperm[pos]) * 5 + k] = v;
}

// Partial dot products of nvec vectors V[i] (stride n) with w: partial[block][i].
__global__ void k_multidot_partial(const double* __restrict__ V, int nvec, size_t n,
                                   const double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double red[64][8];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  double acc[64];
  for (int i = 0; i < nvec; ++i) acc[i] = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double wt = w[t];
    for (int i = 0; i < nvec; ++i) acc[i] = fma(V[(size_t)i * n + t], wt, acc[i]);
  }
  for (int i = 0; i < nvec; ++i) {
    const double s = warp_sum(acc[i]);
    if (lane == 0) red[i][warp] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) s += red[i][k];
    partial[(size_t)blockIdx.x * 64 + i] = s;
  }
}

__global__ void k_multidot_final(const double* __restrict__ partial, int nblocks, int nvec, double* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= nvec) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * 64 + i];
  out[i] = s;
}

__global__ void k_vec_update(double* __restrict__ w, const double* __restrict__ V, int nvec, size_t n,
                             const double* __restrict__ coef, double sign) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < nvec; ++i) s = fma(coef[i], V[(size_t)i * n + t], s);
    w[t] = fma(sign, s, w[t]);
  }
}

__global__ void k_scale_copy(double* __restrict__ dst, const double* __restrict__ src, size_t n,
                             const double* __restrict__ scal, int invert) {
  const double a = invert ? 1.0 / scal[0] : scal[0];
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    dst[t] = a * src[t];
}

__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = a * x[t] + b * y[t];
}

constexpr int kDotBlocks = 608;  // 4 x 152 SMs

}  // namespace

namespace sc {

cudaError_t cond_interior(sc_ctx* c, const double* xb, double beta, const double* Bfull, double alpha, double* u) {
  const Geo& G = c->G;
  if (G.ni == 0) return cudaSuccess;
  k_cond_interior<<<G.K, 256, G.ni * sizeof(double), c->stream>>>(G, c->Aown, c->X, c->Ainv, c->d_nbr, c->d_pptr,
      c->d_pids, c->d_pslot, c->d_pcol, c->d_perm, c->d_iperm, xb, beta, Bfull, alpha, u);
  return cudaGetLastError();
}

cudaError_t cond_boundary(sc_ctx* c, const double* xb, double delta, const double* Bfull, double gamma_,
                          const double* u, double* y) {
  const Geo& G = c->G;
  k_cond_boundary<<<G.K, 256, 0, c->stream>>>(G, c->Aown, c->X, c->d_nbr, c->d_pptr, c->d_pids, c->d_pslot,
      c->d_pcol, c->d_perm, c->d_iperm, xb, delta, Bfull, gamma_, G.ni ? u : nullptr, y);
  return cudaGetLastError();
}

cudaError_t global_apply(sc_ctx* c, const double* x, double* y) {
  const Geo& G = c->G;
  const size_t smem = (size_t)G.ne * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(k_global_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_global_apply<<<G.K, 256, smem, c->stream>>>(G, c->Aown, c->X, c->d_nbr, c->d_pptr, c->d_pids, c->d_pslot,
                                                c->d_pcol, c->d_iperm, x, y);
  return cudaGetLastError();
}

cudaError_t scatter_solution(sc_ctx* c, const double* xb, const double* xi, double* x) {
  const Geo& G = c->G;
  const size_t n = (size_t)G.K * G.ne;
  k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(G, c->d_iperm, xb, xi, x);
  return cudaGetLastError();
}

cudaError_t multidot(sc_ctx* c, const double* V, int nvec, size_t n, const double* w, double* out_dev) {
  if (nvec > 64) return cudaErrorInvalidValue;
  k_multidot_partial<<<kDotBlocks, 256, 0, c->stream>>>(V, nvec, n, w, c->partial);
  k_multidot_final<<<1, 64, 0, c->stream>>>(c->partial, kDotBlocks, nvec, out_dev);
  return cudaGetLastError();
}

cudaError_t vec_update(sc_ctx* c, double* w, const double* V, int nvec, size_t n, const double* coef_dev,
                       double sign) {
  k_vec_update<<<kDotBlocks, 256, 0, c->stream>>>(w, V, nvec, n, coef_dev, sign);
  return cudaGetLastError();
}

cudaError_t vec_scale_copy(sc_ctx* c, double* dst, const double* src, size_t n, const double* scal_dev, int invert) {
  k_scale_copy<<<kDotBlocks, 256, 0, c->stream>>>(dst, src, n, scal_dev, invert);
  return cudaGetLastError();
}

cudaError_t vec_axpby(sc_ctx* c, double* y, double a, const double* x, double b, size_t n) {
  k_axpby<<<kDotBlocks, 256, 0, c->stream>>>(y, a, x, b, n);
  return cudaGetLastError();
}

}  // namespace sc
