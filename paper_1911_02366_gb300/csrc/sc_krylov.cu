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

// 16-byte vector type of each storage precision.
template <class T> struct Vec16;
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };

__device__ __forceinline__ void fma16(const double2& a, const double2& b, double& s0, double& s1) {
  s0 = fma(a.x, b.x, s0); s1 = fma(a.y, b.y, s1);
}
__device__ __forceinline__ void fma16(const float4& a, const float4& b, float& s0, float& s1) {
  s0 = fmaf(a.x, b.x, s0); s1 = fmaf(a.y, b.y, s1); s0 = fmaf(a.z, b.z, s0); s1 = fmaf(a.w, b.w, s1);
}

// Dot product of a row segment (global, 16-byte aligned) with a vector in shared memory
// (16-byte aligned), one warp, 16-byte loads, arithmetic in the storage precision T;
// returns this lane's partial sum.
template <class T>
__device__ __forceinline__ T warp_dot(const T* __restrict__ row, const T* v, int len, int lane) {
  using V = typename Vec16<T>::type;
  constexpr int W = Vec16<T>::n;
  const V* r = reinterpret_cast<const V*>(row);
  const V* x = reinterpret_cast<const V*>(v);
  const int nv = len / W;
  T s0 = T(0), s1 = T(0);
#pragma unroll 4
  for (int i = lane; i < nv; i += 32) fma16(__ldg(r + i), x[i], s0, s1);
  for (int i = nv * W + lane; i < len; i += 32) s0 = fma(__ldg(row + i), v[i], s0);
  return s0 + s1;
}

__device__ __forceinline__ float warp_sum(float s) {
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

// Two row dots at once (independent loads in flight): lane partial sums of
// rowA . v and rowB . v over len entries.
template <class T>
__device__ __forceinline__ void warp_dot2(const T* __restrict__ rowA, const T* __restrict__ rowB, const T* v, int len,
                                          int lane, T& sa, T& sb) {
  using V = typename Vec16<T>::type;
  constexpr int W = Vec16<T>::n;
  const V* ra = reinterpret_cast<const V*>(rowA);
  const V* rb = reinterpret_cast<const V*>(rowB);
  const V* x = reinterpret_cast<const V*>(v);
  const int nv = len / W;
  T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
#pragma unroll 2
  for (int i = lane; i < nv; i += 32) {
    const V xa = x[i];
    fma16(__ldg(ra + i), xa, a0, a1);
    fma16(__ldg(rb + i), xa, b0, b1);
  }
  for (int i = nv * W + lane; i < len; i += 32) { a0 = fma(__ldg(rowA + i), v[i], a0); b0 = fma(__ldg(rowB + i), v[i], b0); }
  sa = a0 + a1; sb = b0 + b1;
}

// Neighbour couplings of row (node j, variable k) of element e.  The couplings of one
// row are contiguous in X (layout X[e][k][pair][l]); vb / vi are the condensed
// boundary / interior vectors of all elements in the storage precision T (either may
// be null), scaled by cb / ci.
template <class T>
__device__ __forceinline__ T cross_row(const Geo& G, int e, int j, int k, const T* __restrict__ X,
                                       const int* nbr_s, const int* __restrict__ pptr,
                                       const int* __restrict__ pinfo, const T* __restrict__ vb, T cb,
                                       const T* __restrict__ vi, T ci, int lane) {
  const int q0 = __ldg(pptr + j), q1 = __ldg(pptr + j + 1);
  const T* Xr = X + (((size_t)e * 5 + k) * G.NP + q0) * 5;
  T s = T(0);
  for (int f = lane; f < 5 * (q1 - q0); f += 32) {
    const int q = q0 + f / 5, l = f % 5;
    const int info = __ldg(pinfo + q);
    const int nb = nbr_s[pinfo_slot(info)];
    const int off = pinfo_offset(info) + l;
    T xv;
    if (pinfo_interior(info)) {
      if (!vi) continue;
      xv = ci * vi[(size_t)nb * G.ni + off];
    } else {
      if (!vb) continue;
      xv = cb * vb[(size_t)nb * G.nb + off];
    }
    s = fma(__ldg(Xr + f), xv, s);
  }
  return s;
}

// Neighbour couplings of a set of rows, one thread per (element, row): rows are the
// permuted positions [row0, row0 + nrows) of every element; out[e][r - row0] =
// sum over the row's couplings of X * (cb x_b or ci v_i) of the neighbour.
template <class T>
__global__ void __launch_bounds__(256) k_cross_rows(Geo G, const T* __restrict__ X, const int* __restrict__ nbr,
    const int* __restrict__ pptr, const int* __restrict__ pinfo, const int* __restrict__ iperm, int row0, int nrows,
    const T* __restrict__ vb, T cb, const T* __restrict__ vi, T ci, T* __restrict__ out) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)G.K * nrows) return;
  const int e = (int)(t / nrows), r = row0 + (int)(t % nrows);
  const int j = __ldg(iperm + r / 5), k = r % 5;
  const int q0 = __ldg(pptr + j), q1 = __ldg(pptr + j + 1);
  const T* Xr = X + (((size_t)e * 5 + k) * G.NP + q0) * 5;
  const int* nb_e = nbr + e * 18;
  T s = T(0);
  for (int q = q0; q < q1; ++q) {
    const int info = __ldg(pinfo + q);
    const int nb = __ldg(nb_e + pinfo_slot(info));
    const int off = pinfo_offset(info);
    const T* vec;
    T coef;
    if (pinfo_interior(info)) { vec = vi ? vi + (size_t)nb * G.ni + off : nullptr; coef = ci; }
    else { vec = vb ? vb + (size_t)nb * G.nb + off : nullptr; coef = cb; }
    if (!vec) continue;
    const T* xq = Xr + (q - q0) * 5;
    T a = T(0);
#pragma unroll
    for (int l = 0; l < 5; ++l) a = fma(__ldg(xq + l), vec[l], a);
    s = fma(coef, a, s);
  }
  out[t] = s;
}

// Interior pass: u_e = A_ii,e^-1 (alpha B_i,e + beta (A_ib x_b)_e).  Matrices and the
// vectors x_b, u in precision T; the full right-hand side B in double.
template <class T>
__global__ void __launch_bounds__(256) k_cond_interior(Geo G, const T* __restrict__ Aown,
    const T* __restrict__ X, const T* __restrict__ Ainv, const int* __restrict__ nbr,
    const int* __restrict__ pptr, const int* __restrict__ pinfo, const int* __restrict__ iperm,
    const T* __restrict__ xb, double beta, const double* __restrict__ Bfull, double alpha,
    T* __restrict__ u, const T* __restrict__ cross) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int e = blockIdx.x, ni = G.ni, nb = G.nb;
  T* v = reinterpret_cast<T*>(smem_raw);  // nb: x_e
  T* t = v + ((nb + 3) & ~3);             // ldi: right-hand side of the interior solve, zero padded,
                                          // 16-byte aligned for the vector loads of warp_dot
  __shared__ int nbr_s[18];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  if (threadIdx.x < 18) nbr_s[threadIdx.x] = nbr[e * 18 + threadIdx.x];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[i] = xb ? xb[(size_t)e * nb + i] : T(0);
  for (int i = ni + threadIdx.x; i < G.ldi; i += blockDim.x) t[i] = T(0);
  __syncthreads();
  const T* Ae = Aown + (size_t)e * own_stride(G);
  for (int ri = warp; ri < ni; ri += nw) {
    const int j = __ldg(iperm + ri / 5), k = ri % 5;
    T s = T(0);
    if (xb) {
      s = warp_dot(Ae + (size_t)ri * G.lda + G.cb0, v, nb, lane);
      if (!cross) s += cross_row(G, e, j, k, X, nbr_s, pptr, pinfo, xb, T(1), (const T*)nullptr, T(0), lane);
      s = warp_sum(s);
      if (cross) s += cross[(size_t)e * ni + ri];
    }
    if (lane == 0) {
      T val = T(beta) * s;
      if (Bfull) val += T(alpha * Bfull[((size_t)e * G.nn + j) * 5 + k]);
      t[ri] = val;
    }
  }
  __syncthreads();
  const T* Ie = Ainv + (size_t)e * ni * G.ldi;
  for (int ri = 2 * warp; ri < ni; ri += 2 * nw) {
    const bool two = ri + 1 < ni;
    T sa, sb;
    warp_dot2(Ie + (size_t)ri * G.ldi, Ie + (size_t)(two ? ri + 1 : ri) * G.ldi, t, G.ldi, lane, sa, sb);
    sa = warp_sum(sa); sb = warp_sum(sb);
    if (lane == 0) {
      u[(size_t)e * ni + ri] = sa;
      if (two) u[(size_t)e * ni + ri + 1] = sb;
    }
  }
}

// Boundary pass: y_e = gamma B_b,e + delta (A_bb x_b)_e - (A_bi u)_e.  Matrices and x_b, u
// in precision T; B and y in double.
template <class T>
__global__ void __launch_bounds__(256) k_cond_boundary(Geo G, const T* __restrict__ Aown,
    const T* __restrict__ X, const int* __restrict__ nbr,
    const int* __restrict__ pptr, const int* __restrict__ pinfo, const int* __restrict__ iperm,
    const T* __restrict__ xb, double delta, const double* __restrict__ Bfull, double gamma_,
    const T* __restrict__ u, double* __restrict__ y, const T* __restrict__ cross) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int e = blockIdx.x, ni = G.ni, nb = G.nb, ne = G.ne, lda = G.lda, cb0 = G.cb0;
  T* v = reinterpret_cast<T*>(smem_raw);  // lda: [-u_e | 0 | delta x_e | 0] in own-column order
  __shared__ int nbr_s[18];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const T dT = T(delta);
  if (threadIdx.x < 18) nbr_s[threadIdx.x] = nbr[e * 18 + threadIdx.x];
  for (int i = threadIdx.x; i < lda; i += blockDim.x) {
    T val = T(0);
    if (i < ni) { if (u) val = -u[(size_t)e * ni + i]; }
    else if (i >= cb0 && i < cb0 + nb) { if (xb) val = dT * xb[(size_t)e * nb + i - cb0]; }
    v[i] = val;
  }
  __syncthreads();
  const T* Ae = Aown + (size_t)e * own_stride(G);
  const int c0 = u ? 0 : cb0;                 // skip the A_bi columns when u is absent
  const int len = (xb ? cb0 + nb : ni) - c0;  // and the A_bb columns when x_b is absent
  for (int ra = ni + 2 * warp; ra < ne; ra += 2 * nw) {
    const int rb2 = ra + 1 < ne ? ra + 1 : ra;
    T sa = T(0), sb = T(0);
    if (xb || u) warp_dot2(Ae + (size_t)ra * lda + c0, Ae + (size_t)rb2 * lda + c0, v + c0, len, lane, sa, sb);
    if (!cross) {
      sa += cross_row(G, e, __ldg(iperm + ra / 5), ra % 5, X, nbr_s, pptr, pinfo, xb, dT, u, T(-1), lane);
      sb += cross_row(G, e, __ldg(iperm + rb2 / 5), rb2 % 5, X, nbr_s, pptr, pinfo, xb, dT, u, T(-1), lane);
    }
    sa = warp_sum(sa); sb = warp_sum(sb);
    if (cross) { sa += cross[(size_t)e * nb + ra - ni]; sb += cross[(size_t)e * nb + rb2 - ni]; }
    if (lane == 0) {
      double va = (double)sa, vb = (double)sb;
      if (Bfull) {
        va += gamma_ * Bfull[((size_t)e * G.nn + __ldg(iperm + ra / 5)) * 5 + ra % 5];
        vb += gamma_ * Bfull[((size_t)e * G.nn + __ldg(iperm + rb2 / 5)) * 5 + rb2 % 5];
      }
      y[(size_t)e * nb + ra - ni] = va;
      if (rb2 != ra) y[(size_t)e * nb + rb2 - ni] = vb;
    }
  }
}

// y = A x on the full system, natural global dof order.
__global__ void __launch_bounds__(256) k_global_apply(Geo G, const double* __restrict__ Aown,
    const double* __restrict__ X, const int* __restrict__ nbr, const int* __restrict__ pptr,
    const int* __restrict__ pinfo, const int* __restrict__ pcol, const int* __restrict__ iperm,
    const double* __restrict__ x, double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* v = reinterpret_cast<double*>(smem_raw);  // lda, own-column order
  __shared__ int nbr_s[18];
  const int e = blockIdx.x, ne = G.ne, nn = G.nn, lda = G.lda;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  if (threadIdx.x < 18) nbr_s[threadIdx.x] = nbr[e * 18 + threadIdx.x];
  for (int i = threadIdx.x; i < lda; i += blockDim.x) v[i] = 0.0;
  __syncthreads();
  for (int t = threadIdx.x; t < ne; t += blockDim.x) {
    const int pos = t / 5, k = t % 5;
    v[own_col(G, pos, k)] = x[((size_t)e * nn + iperm[pos]) * 5 + k];
  }
  __syncthreads();
  const double* Ae = Aown + (size_t)e * own_stride(G);
  for (int ri = warp; ri < ne; ri += nw) {
    const int j = __ldg(iperm + ri / 5), k = ri % 5;
    double s = warp_dot(Ae + (size_t)ri * lda, v, lda, lane);
    const int q0 = __ldg(pptr + j), q1 = __ldg(pptr + j + 1);
    const double* Xr = X + (((size_t)e * 5 + k) * G.NP + q0) * 5;
    for (int f = lane; f < 5 * (q1 - q0); f += 32) {
      const int q = q0 + f / 5, l = f % 5;
      const int nbe = nbr_s[pinfo_slot(__ldg(pinfo + q))];
      s = fma(__ldg(Xr + f), x[((size_t)nbe * nn + __ldg(pcol + q)) * 5 + l], s);
    }
    s = warp_sum(s);
    if (lane == 0) y[((size_t)e * nn + j) * 5 + k] = s;
  }
}

template <class TI>
__global__ void k_scatter(Geo G, const int* __restrict__ iperm, const double* __restrict__ xb,
                          const TI* __restrict__ xi, double* __restrict__ x) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)G.K * G.ne) return;
  const int e = (int)(t / G.ne), r = (int)(t % G.ne);
  const int pos = r / 5, k = r % 5;
  const double v = pos < G.nin ? (double)xi[(size_t)e * G.ni + r] : xb[(size_t)e * G.nb + r - G.ni];
  x[((size_t)e * G.nn + iperm[pos]) * 5 + k] = v;
}

// Partial dot products <V[i], w> over a slice of the vectors: grid (chunks, nvec);
// partial[i * gridDim.x + chunk].
// Partial dot products w . v_i over the chunk of block x, one vector per block row y.  With
// vec2 (n even, both pointers 16-byte aligned) the loads are double2, two chains per thread.
__global__ void __launch_bounds__(256) k_multidot_partial(const double* __restrict__ V, size_t n,
                                                          const double* __restrict__ w,
                                                          double* __restrict__ partial, int vec2) {
  __shared__ double red[8];
  const int i = blockIdx.y;
  const double* v = V + (size_t)i * n;
  double s = 0.0, s2 = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if (vec2) {
    const double2* v2 = reinterpret_cast<const double2*>(v);
    const double2* w2 = reinterpret_cast<const double2*>(w);
    const size_t n2 = n / 2;
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; t + stride < n2; t += 2 * stride) {
      const double2 a = __ldg(v2 + t), b = __ldg(w2 + t), c = __ldg(v2 + t + stride), d = __ldg(w2 + t + stride);
      s = fma(a.x, b.x, s); s2 = fma(a.y, b.y, s2);
      s = fma(c.x, d.x, s); s2 = fma(c.y, d.y, s2);
    }
    if (t < n2) {
      const double2 a = __ldg(v2 + t), b = __ldg(w2 + t);
      s = fma(a.x, b.x, s); s2 = fma(a.y, b.y, s2);
    }
  } else {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += stride) s = fma(v[t], w[t], s);
  }
  s = warp_sum(s + s2);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) r += red[k];
    partial[(size_t)i * gridDim.x + blockIdx.x] = r;
  }
}

__global__ void k_multidot_final(const double* __restrict__ partial, int nchunks, int nvec, double* __restrict__ out) {
  const int i = blockIdx.x;
  if (i >= nvec) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nchunks; b += blockDim.x) s += partial[(size_t)i * nchunks + b];
  s = warp_sum(s);
  __shared__ double red[8];
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) r += red[k];
    out[i] = r;
  }
}

// w -= or += sum_i coef[i] v_i (sign); with vec2 (n even, pointers 16-byte aligned) double2
// accesses and the vectors taken four at a time into independent accumulators.
__global__ void __launch_bounds__(256) k_vec_update(double* __restrict__ w, const double* __restrict__ V, int nvec,
                                                    size_t n, const double* __restrict__ coef, double sign,
                                                    int vec2) {
  __shared__ double cs[64];
  for (int i = threadIdx.x; i < nvec && i < 64; i += blockDim.x) cs[i] = coef[i];
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if (vec2 && nvec <= 64) {
    const size_t n2 = n / 2;
    double2* w2 = reinterpret_cast<double2*>(w);
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n2; t += stride) {
      double2 a0 = make_double2(0.0, 0.0), a1 = a0, a2 = a0, a3 = a0;
      int i = 0;
      for (; i + 4 <= nvec; i += 4) {
        const double2 v0 = __ldg(reinterpret_cast<const double2*>(V + (size_t)i * n) + t);
        const double2 v1 = __ldg(reinterpret_cast<const double2*>(V + (size_t)(i + 1) * n) + t);
        const double2 v2 = __ldg(reinterpret_cast<const double2*>(V + (size_t)(i + 2) * n) + t);
        const double2 v3 = __ldg(reinterpret_cast<const double2*>(V + (size_t)(i + 3) * n) + t);
        a0.x = fma(cs[i], v0.x, a0.x); a0.y = fma(cs[i], v0.y, a0.y);
        a1.x = fma(cs[i + 1], v1.x, a1.x); a1.y = fma(cs[i + 1], v1.y, a1.y);
        a2.x = fma(cs[i + 2], v2.x, a2.x); a2.y = fma(cs[i + 2], v2.y, a2.y);
        a3.x = fma(cs[i + 3], v3.x, a3.x); a3.y = fma(cs[i + 3], v3.y, a3.y);
      }
      for (; i < nvec; ++i) {
        const double2 v0 = __ldg(reinterpret_cast<const double2*>(V + (size_t)i * n) + t);
        a0.x = fma(cs[i], v0.x, a0.x); a0.y = fma(cs[i], v0.y, a0.y);
      }
      double2 o = w2[t];
      o.x = fma(sign, (a0.x + a1.x) + (a2.x + a3.x), o.x);
      o.y = fma(sign, (a0.y + a1.y) + (a2.y + a3.y), o.y);
      w2[t] = o;
    }
    return;
  }
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += stride) {
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

__global__ void k_vec_to_float(float* __restrict__ y, const double* __restrict__ x, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}

// y = a x + b y; with b = 0 y is not read (it may hold anything, NaN included, e.g. a fresh
// Krylov basis vector in memory another context used before).
__global__ void k_axpby(double* __restrict__ y, double a, const double* __restrict__ x, double b, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = b == 0.0 ? a * x[t] : a * x[t] + b * y[t];
}

constexpr int kDotBlocks = 608;  // 4 x 152 SMs
constexpr int kDotChunks = 152;

}  // namespace

namespace sc {

// The condensed operator's passes: fused kernels on the pattern-packed blocks once the
// condensation has packed them, otherwise a coupling pass followed by the dense kernels.
template <class T>
cudaError_t cond_interior_t(sc_ctx* c, const T* Aown, const T* Apk, const T* X, const T* Ainv, T* crossbuf,
                            const T* xb, double beta, const double* Bfull, double alpha, T* u) {
  const Geo& G = c->G;
  if (G.ni == 0) return cudaSuccess;
  if (Apk) {
    ProfScope ps(c, SCK_COND_INTERIOR);
    return cond_interior_pk<T>(c, Apk, X, Ainv, xb, beta, Bfull, alpha, u, 0);
  }
  if (xb) {
    count_launch(c);
    const size_t rows = (size_t)G.K * G.ni;
    k_cross_rows<T><<<(unsigned)((rows + 255) / 256), 256, 0, c->stream>>>(G, X, c->d_nbr, c->d_pptr, c->d_pinfo,
        c->d_iperm, 0, G.ni, xb, T(1), (const T*)nullptr, T(0), crossbuf);
  }
  ProfScope ps(c, SCK_COND_INTERIOR);
  const size_t smem = (size_t)(((G.nb + 3) & ~3) + G.ldi) * sizeof(T);
  k_cond_interior<T><<<G.K, 256, smem, c->stream>>>(G, Aown, X, Ainv, c->d_nbr, c->d_pptr, c->d_pinfo, c->d_iperm,
                                                    xb, beta, Bfull, alpha, u, xb ? crossbuf : (const T*)nullptr);
  return cudaGetLastError();
}

template <class T>
cudaError_t cond_boundary_t(sc_ctx* c, const T* Aown, const T* Apk, const T* X, T* crossbuf, const T* xb,
                            double delta, const double* Bfull, double gamma_, const T* u, double* y) {
  const Geo& G = c->G;
  if (G.ni == 0) u = nullptr;
  if (Apk) {
    ProfScope ps(c, SCK_COND_BOUNDARY);
    return cond_boundary_pk<T>(c, Apk, X, xb, delta, Bfull, gamma_, u, y);
  }
  const bool need = xb || u;
  if (need) {
    count_launch(c);
    const size_t rows = (size_t)G.K * G.nb;
    k_cross_rows<T><<<(unsigned)((rows + 255) / 256), 256, 0, c->stream>>>(G, X, c->d_nbr, c->d_pptr, c->d_pinfo,
        c->d_iperm, G.ni, G.nb, xb, T(delta), u, T(-1), crossbuf);
  }
  ProfScope ps(c, SCK_COND_BOUNDARY);
  const size_t smem = (size_t)G.lda * sizeof(T);
  k_cond_boundary<T><<<G.K, 256, smem, c->stream>>>(G, Aown, X, c->d_nbr, c->d_pptr, c->d_pinfo, c->d_iperm, xb,
                                                    delta, Bfull, gamma_, u, y, need ? crossbuf : (const T*)nullptr);
  return cudaGetLastError();
}

cudaError_t cond_interior(sc_ctx* c, const double* xb, double beta, const double* Bfull, double alpha, double* u) {
  return cond_interior_t<double>(c, c->Aown, c->packed ? c->Apk : nullptr, c->X, c->Ainv, c->Cross, xb, beta, Bfull,
                                 alpha, u);
}

cudaError_t cond_boundary(sc_ctx* c, const double* xb, double delta, const double* Bfull, double gamma_,
                          const double* u, double* y) {
  return cond_boundary_t<double>(c, c->Aown, c->packed ? c->Apk : nullptr, c->X, c->Cross, xb, delta, Bfull, gamma_,
                                 u, y);
}

cudaError_t cond_interior32(sc_ctx* c, const float* xb, double beta, const double* Bfull, double alpha, float* u) {
  return cond_interior_t<float>(c, c->Aown32, c->packed ? c->Apk32 : nullptr, c->X32, c->Ainv32, c->Cross32, xb, beta,
                                Bfull, alpha, u);
}

// Interior pass of the red-black sweep: u = A_ii^-1 (A_ib x_b) with x_b zero on the black
// elements, whose own part is then skipped (packed blocks; otherwise the general pass).
cudaError_t cond_interior_sweep(sc_ctx* c, const double* xb, double* u) {
  if (!c->packed || c->G.ni == 0) return cond_interior(c, xb, 1.0, nullptr, 0.0, u);
  ProfScope ps(c, SCK_COND_INTERIOR);
  return cond_interior_pk<double>(c, c->Apk, c->X, c->Ainv, xb, 1.0, nullptr, 0.0, u, 1);
}

cudaError_t cond_interior_sweep32(sc_ctx* c, const float* xb, float* u) {
  if (!c->packed || c->G.ni == 0) return cond_interior32(c, xb, 1.0, nullptr, 0.0, u);
  ProfScope ps(c, SCK_COND_INTERIOR);
  return cond_interior_pk<float>(c, c->Apk32, c->X32, c->Ainv32, xb, 1.0, nullptr, 0.0, u, 1);
}

cudaError_t cond_boundary32(sc_ctx* c, const float* xb, double delta, const double* Bfull, double gamma_,
                            const float* u, double* y) {
  return cond_boundary_t<float>(c, c->Aown32, c->packed ? c->Apk32 : nullptr, c->X32, c->Cross32, xb, delta, Bfull,
                                gamma_, u, y);
}

cudaError_t global_apply(sc_ctx* c, const double* x, double* y) {
  const Geo& G = c->G;
  const size_t smem = (size_t)G.lda * sizeof(double);
  ProfScope ps(c, SCK_GLOBAL_APPLY);
  k_global_apply<<<G.K, 256, smem, c->stream>>>(G, c->Aown, c->X, c->d_nbr, c->d_pptr, c->d_pinfo, c->d_pcol,
                                                c->d_iperm, x, y);
  return cudaGetLastError();
}

cudaError_t scatter_solution(sc_ctx* c, const double* xb, const double* xi, double* x) {
  const Geo& G = c->G;
  const size_t n = (size_t)G.K * G.ne;
  count_launch(c);
  k_scatter<double><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(G, c->d_iperm, xb, xi, x);
  return cudaGetLastError();
}

cudaError_t scatter_solution32(sc_ctx* c, const double* xb, const float* xi, double* x) {
  const Geo& G = c->G;
  const size_t n = (size_t)G.K * G.ne;
  count_launch(c);
  k_scatter<float><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(G, c->d_iperm, xb, xi, x);
  return cudaGetLastError();
}

cudaError_t multidot(sc_ctx* c, const double* V, int nvec, size_t n, const double* w, double* out_dev) {
  if (nvec < 1 || nvec > c->restart_alloc + 1) return cudaErrorInvalidValue;
  const int chunks = kDotChunks;
  count_launch(c, 2);
  const int vec2 = n % 2 == 0 && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  k_multidot_partial<<<dim3(chunks, nvec), 256, 0, c->stream>>>(V, n, w, c->partial, vec2);
  k_multidot_final<<<nvec, 256, 0, c->stream>>>(c->partial, chunks, nvec, out_dev);
  return cudaGetLastError();
}

cudaError_t vec_update(sc_ctx* c, double* w, const double* V, int nvec, size_t n, const double* coef_dev,
                       double sign) {
  count_launch(c);
  const int vec2 = n % 2 == 0 && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
  k_vec_update<<<kDotBlocks, 256, 0, c->stream>>>(w, V, nvec, n, coef_dev, sign, vec2);
  return cudaGetLastError();
}

cudaError_t vec_scale_copy(sc_ctx* c, double* dst, const double* src, size_t n, const double* scal_dev, int invert) {
  count_launch(c);
  k_scale_copy<<<kDotBlocks, 256, 0, c->stream>>>(dst, src, n, scal_dev, invert);
  return cudaGetLastError();
}

cudaError_t vec_to_float(sc_ctx* c, float* y, const double* x, size_t n) {
  count_launch(c);
  k_vec_to_float<<<kDotBlocks, 256, 0, c->stream>>>(y, x, n);
  return cudaGetLastError();
}

cudaError_t vec_axpby(sc_ctx* c, double* y, double a, const double* x, double b, size_t n) {
  count_launch(c);
  k_axpby<<<kDotBlocks, 256, 0, c->stream>>>(y, a, x, b, n);
  return cudaGetLastError();
}

}  // namespace sc

// ---------------------------------------------------------------------------------
// Allocation-free condensed operator.
//
// sc_condensed_matvec_static applies S with the same operator passes as
// sc_condensed_matvec, but the vectors that link its passes (the interior vector
// u = A_ii^-1 A_ib x_b, and on the mixed arm also the FP32 copy of x_b) live in the static
// device array below instead of context-owned memory, so the call itself never
// allocates.  The array holds 8 MiB on every GPU that loads this library, for the life
// of the process.
// ---------------------------------------------------------------------------------
namespace {
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
}  // namespace

static __device__ __align__(256) unsigned char g_condensed_scratch[kStaticScratchBytes];

namespace {
// Device address of the scratch array on the current device.  Looked up on every call
// with that device current: the lookup allocates nothing, and it stays valid across a
// cudaDeviceReset, which reloads the module at a possibly different address.
cudaError_t static_scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_condensed_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}
}  // namespace

extern "C" sc_status sc_condensed_matvec_static(sc_ctx* c, const double* xb, double* yb) {
  if (!c || !xb || !yb) return SC_ERR_ARG;
  if (!c->has_mesh) {
    c->err = "condensed_matvec_static before set_mesh";
    return SC_ERR_STATE;
  }
  const Geo& G = c->G;
  const bool mixed = c->cfg.precision == SC_PREC_MIXED;
  const bool expl = mixed && c->cfg.explicit_schur;
  const size_t n1 = (size_t)G.K * G.nb, nint = (size_t)G.K * G.ni;
  // FP64 arm: u in doubles; mixed arm: the FP32 copy of x_b (aligned to 256 bytes), then u
  // in floats (the explicit operator needs no u)
  const size_t xf_bytes = mixed ? ((n1 * sizeof(float) + 255) & ~size_t(255)) : 0;
  const size_t need = mixed ? xf_bytes + (expl ? 0 : nint * sizeof(float)) : nint * sizeof(double);
  if (need > kStaticScratchBytes) {
    c->err = "condensed_matvec_static: this mesh needs " + std::to_string(need) +
             " bytes of scratch (FP64 arm: 8 x elements x interior dofs; mixed arm: 4 x elements x"
             " (boundary + interior dofs)), more than the " + std::to_string(kStaticScratchBytes) +
             " bytes of the static buffer; use sc_condensed_matvec";
    return SC_ERR_ARG;
  }
  if (!c->condensed) {
    c->err = "condensed_matvec_static before condense";
    return SC_ERR_STATE;
  }
  unsigned char* scratch = nullptr;
  cudaError_t e = static_scratch_address(&scratch);
  if (e != cudaSuccess) {
    c->err = std::string("condensed_matvec_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return SC_ERR_CUDA;
  }
  // Every pass writes the entries it later reads (x_b's FP32 copy, then u) before reading
  // them, so nothing left in the array by an earlier call is ever read.
  if (mixed) {
    float* xf = reinterpret_cast<float*>(scratch);
    float* uf = reinterpret_cast<float*>(scratch + xf_bytes);
    e = sc::vec_to_float(c, xf, xb, n1);
    if (e == cudaSuccess) {
      if (expl) {
        e = sc::explicit_matvec32(c, xf, yb);
      } else {
        e = sc::cond_interior32(c, xf, 1.0, nullptr, 0.0, uf);
        if (e == cudaSuccess) e = sc::cond_boundary32(c, xf, 1.0, nullptr, 0.0, uf, yb);
      }
    }
  } else {
    double* u = reinterpret_cast<double*>(scratch);
    e = sc::cond_interior(c, xb, 1.0, nullptr, 0.0, u);
    if (e == cudaSuccess) e = sc::cond_boundary(c, xb, 1.0, nullptr, 0.0, u, yb);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("condensed_matvec_static: ") + cudaGetErrorString(e);
    return SC_ERR_CUDA;
  }
  return SC_OK;
}
