// Pattern-packed element blocks for the condensed operator (Sec. 2.2, eq. SC_step1 with
// the implicit Schur product; Sec. 3.1 on the sparsity of the element blocks).
//
// On a tensor-product GL element the own block couples node j only to the nodes that
// share at least one of its three GL indices: the inviscid volume terms run along the
// three grid lines through j, and the BR1 viscous terms differentiate a lifted gradient
// that itself runs along lines, so they reach the three planes through j.  The operator
// passes need A_ib (interior rows, boundary columns) and [A_bi A_bb] (boundary rows): of
// these dense blocks only 43-50 % of the 5 x 5 node blocks can be nonzero.
//
// Packed layout, per element and shared by all elements: row r of the own block keeps
// the entries of its node's column list (the column nodes sharing an index, interior
// columns first, in own-column order), 5 per column node, padded to a multiple of 4
// entries so that every row starts on 16 bytes.  The packing kernel also checks that
// every entry left out is exactly zero and reports the element otherwise.
#include "sc_internal.cuh"

namespace {

// Resident CTAs per SM asked of the operator passes: the FP32 passes are latency-bound at
// their natural 64 registers (4 CTAs); capping them at 40 (6 CTAs) measured 14 % (boundary)
// and 29 % (interior) faster at 16^3, N = 4.  The FP64 passes are FP64-ALU bound and keep
// their natural allocation (3 CTAs allow the 71-80 registers they use).
template <class T> struct PkOcc { static constexpr int v = 3; };
template <> struct PkOcc<float> { static constexpr int v = 6; };

template <class T> struct PkVec;
template <> struct PkVec<float> { using type = float4; static constexpr int n = 4; };
template <> struct PkVec<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The 5 rows of node p (variables k = 0..4) against the own-column-ordered vector v in
// shared memory: row k of the node starts at P0 + k * rs and holds n packed entries;
// entry j belongs to column node j / 5 of the node's list `cols`, variable j % 5.  The
// column decode and the gather from v are shared by the five rows.
template <class T>
__device__ __forceinline__ void own_node5(const T* __restrict__ P0, int rs, int n, const int* __restrict__ cols,
                                          const T* __restrict__ v, int lane, T acc[5]) {
  using V = typename PkVec<T>::type;
  constexpr int W = PkVec<T>::n;
#pragma unroll 2
  for (int j0 = lane * W; j0 < n; j0 += 32 * W) {
    V a[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) a[k] = __ldg(reinterpret_cast<const V*>(P0 + (size_t)k * rs + j0));
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int j = j0 + w;
      if (j < n) {
        const int q = j / 5, l = j - 5 * q;
        const T xv = v[__ldg(cols + q) + l];
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] = fma(reinterpret_cast<const T*>(&a[k])[w], xv, acc[k]);
      }
    }
  }
}

// Neighbour couplings of the 5 rows of one node: row k's pairs are the m = 5 * npairs
// consecutive entries X0[k * ks + idx] (pair idx / 5, variable idx % 5); each pair's
// packed info names the neighbour slot and the offset of its 5 entries in that
// neighbour's boundary (vb, coefficient cb) or interior (vi, coefficient ci) vector.
template <class T>
__device__ __forceinline__ void cross_node5(const T* __restrict__ X0, long long ks, int m,
                                            const int* __restrict__ info, const int* nbr_s, int nb, int ni,
                                            const T* __restrict__ vb, T cb, const T* __restrict__ vi, T ci,
                                            int lane, T acc[5]) {
#pragma unroll 2
  for (int idx = lane; idx < m; idx += 32) {
    const int q = idx / 5, l = idx - 5 * q;
    const int f = __ldg(info + q);
    const int nbe = nbr_s[pinfo_slot(f)], off = pinfo_offset(f);
    T g;
    if (pinfo_interior(f)) {
      if (!vi) continue;
      g = ci * vi[(size_t)nbe * ni + off + l];
    } else {
      if (!vb) continue;
      g = cb * vb[(size_t)nbe * nb + off + l];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] = fma(__ldg(X0 + (size_t)k * ks + idx), g, acc[k]);
  }
}

template <class T>
__device__ __forceinline__ T pick5(const T acc[5], int k) {
  return k == 0 ? acc[0] : k == 1 ? acc[1] : k == 2 ? acc[2] : k == 3 ? acc[3] : acc[4];
}

// Dense FP64 own blocks -> packed blocks of type T; entries outside the pattern must be
// zero (status <- SC_PACK_VIOLATION).  One warp per row.
// With dense32 non-null (mixed arm) the same pass also writes the FP32 copy of the whole
// dense block (padding included) that the condensation products read.
template <class T>
__global__ void __launch_bounds__(256) k_pack(Geo G, const double* __restrict__ Aown, const int* __restrict__ row_off,
                                              const int* __restrict__ pos, T* __restrict__ Apk, long long pstride,
                                              int* __restrict__ status, float* __restrict__ dense32) {
  const int e = blockIdx.x, lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const double* Ae = Aown + (size_t)e * own_stride(G);
  T* Pe = Apk + (size_t)e * pstride;
  bool bad = false;
  for (int r = warp; r < G.ne; r += nw) {
    const int p = r / 5;
    const int* posr = pos + (size_t)p * G.nn;
    T* prow = Pe + __ldg(row_off + r);
    for (int cidx = lane; cidx < G.lda; cidx += 32) {
      const double val = Ae[(size_t)r * G.lda + cidx];
      if (dense32) dense32[(size_t)e * own_stride(G) + (size_t)r * G.lda + cidx] = (float)val;
      int q, l;
      if (cidx < G.ni) { q = cidx / 5; l = cidx - 5 * q; }
      else if (cidx >= G.cb0 && cidx < G.cb0 + G.nb) { const int t = cidx - G.cb0; q = G.nin + t / 5; l = t - 5 * (t / 5); }
      else continue;  // alignment padding
      const int b = __ldg(posr + q);
      if (b >= 0) prow[5 * b + l] = (T)val;
      else if (b == -1 && val != 0.0) bad = true;
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(status, -1, SC_PACK_VIOLATION);
}

// Interior pass: u_e = A_ii,e^-1 (alpha B_i,e + beta (A_ib x_b)_e), A_ib from the packed
// own block and the neighbour couplings; one warp per interior node (its 5 rows).
template <class T>
__global__ void __launch_bounds__(256, PkOcc<T>::v) k_cond_interior_pk(Geo G, const T* __restrict__ Apk, long long pstride,
    const int* __restrict__ row_off, const int* __restrict__ lptr, const int* __restrict__ list,
    const T* __restrict__ X, const int* __restrict__ nbr, const int* __restrict__ pptr,
    const int* __restrict__ pinfo, const T* __restrict__ Ainv, const int* __restrict__ iperm,
    const T* __restrict__ xb, double beta, const double* __restrict__ Bfull, double alpha, T* __restrict__ u,
    int black_zero) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int e = blockIdx.x, ni = G.ni, nb = G.nb, lda = G.lda, ldi = G.ldi;
  // black_zero: x_b is zero on the black elements (the red-black sweep), so their own A_ib x_b
  // part is skipped and only the neighbour couplings feed their interior solve
  const bool own = !(black_zero && ((e % G.n + (e / G.n) % G.n + e / (G.n * G.n)) & 1));
  T* v = reinterpret_cast<T*>(smem_raw);  // lda: x_e at the boundary columns
  T* t = v + lda;                         // ldi: right-hand side of the interior solve
  __shared__ int nbr_s[18];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  if (threadIdx.x < 18) nbr_s[threadIdx.x] = nbr[e * 18 + threadIdx.x];
  for (int i = threadIdx.x; i < lda; i += blockDim.x) {
    T val = T(0);
    if (xb && i >= G.cb0 && i < G.cb0 + nb) val = xb[(size_t)e * nb + i - G.cb0];
    v[i] = val;
  }
  for (int i = ni + threadIdx.x; i < ldi; i += blockDim.x) t[i] = T(0);
  __syncthreads();
  const T* Pe = Apk + (size_t)e * pstride;
  const long long ks = (long long)G.NP * 5;
  for (int p = warp; p < G.nin; p += nw) {
    const int j = __ldg(iperm + p);
    T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (xb) {
      if (own) {
        const int l0 = __ldg(lptr + p), n = 5 * (__ldg(lptr + p + 1) - l0);
        own_node5(Pe + __ldg(row_off + 5 * p), (n + 3) & ~3, n, list + l0, v, lane, acc);
      }
      const int q0 = __ldg(pptr + j), q1 = __ldg(pptr + j + 1);
      cross_node5(X + ((size_t)e * 5 * G.NP + q0) * 5, ks, 5 * (q1 - q0), pinfo + q0, nbr_s, nb, ni, xb, T(1),
                  (const T*)nullptr, T(0), lane, acc);
#pragma unroll
      for (int k = 0; k < 5; ++k) acc[k] = wsum(acc[k]);
    }
    if (lane < 5) {
      T val = T(beta) * pick5(acc, lane);
      if (Bfull) val += T(alpha * Bfull[((size_t)e * G.nn + j) * 5 + lane]);
      t[5 * p + lane] = val;
    }
  }
  __syncthreads();
  using V = typename PkVec<T>::type;
  constexpr int W = PkVec<T>::n;
  const T* Ie = Ainv + (size_t)e * ni * ldi;
  for (int ra = 2 * warp; ra < ni; ra += 2 * nw) {
    const int rb = ra + 1 < ni ? ra + 1 : ra;
    const T* ia = Ie + (size_t)ra * ldi;
    const T* ib = Ie + (size_t)rb * ldi;
    T sa = T(0), sb = T(0);
    for (int j0 = lane * W; j0 < ldi; j0 += 32 * W) {
      const V a = __ldg(reinterpret_cast<const V*>(ia + j0));
      const V b = __ldg(reinterpret_cast<const V*>(ib + j0));
      const T* av = reinterpret_cast<const T*>(&a);
      const T* bv = reinterpret_cast<const T*>(&b);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        sa = fma(av[w], t[j0 + w], sa);
        sb = fma(bv[w], t[j0 + w], sb);
      }
    }
    sa = wsum(sa); sb = wsum(sb);
    if (lane == 0) {
      u[(size_t)e * ni + ra] = sa;
      if (rb != ra) u[(size_t)e * ni + rb] = sb;
    }
  }
}

// Boundary pass: y_e = gamma B_b,e + delta (A_bb x_b)_e - (A_bi u)_e from the packed own
// block and the neighbour couplings (delta x_b of boundary neighbours, -u of interior
// ones); one warp per boundary node (its 5 rows).
template <class T>
__global__ void __launch_bounds__(256, PkOcc<T>::v) k_cond_boundary_pk(Geo G, const T* __restrict__ Apk, long long pstride,
    const int* __restrict__ row_off, const int* __restrict__ lptr, const int* __restrict__ list,
    const T* __restrict__ X, const int* __restrict__ nbr, const int* __restrict__ pptr,
    const int* __restrict__ pinfo, const int* __restrict__ iperm, const T* __restrict__ xb, double delta,
    const double* __restrict__ Bfull, double gamma_, const T* __restrict__ u, double* __restrict__ y,
    const int* __restrict__ elist, const int* __restrict__ nint) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // CTA i serves element elist[i] (one colour of the red-black sweep), or element i
  const int e = elist ? __ldg(elist + blockIdx.x) : blockIdx.x, ni = G.ni, nb = G.nb, lda = G.lda, cb0 = G.cb0;
  T* v = reinterpret_cast<T*>(smem_raw);  // lda: [-u_e | 0 | delta x_e | 0]
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
  const T* Pe = Apk + (size_t)e * pstride;
  const long long ks = (long long)G.NP * 5;
  const bool need = xb || u;
  for (int p = G.nin + warp; p < G.nn; p += nw) {
    const int j = __ldg(iperm + p);
    T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (need) {
      const int l0 = __ldg(lptr + p), n = 5 * (__ldg(lptr + p + 1) - l0);
      // with nint: the element's own boundary values are zero, only the interior columns count
      own_node5(Pe + __ldg(row_off + 5 * p), (n + 3) & ~3, nint ? __ldg(nint + p) : n, list + l0, v, lane, acc);
      const int q0 = __ldg(pptr + j), q1 = __ldg(pptr + j + 1);
      cross_node5(X + ((size_t)e * 5 * G.NP + q0) * 5, ks, 5 * (q1 - q0), pinfo + q0, nbr_s, nb, ni, xb, dT, u,
                  T(-1), lane, acc);
#pragma unroll
      for (int k = 0; k < 5; ++k) acc[k] = wsum(acc[k]);
    }
    if (lane < 5) {
      double val = (double)pick5(acc, lane);
      if (Bfull) val += gamma_ * Bfull[((size_t)e * G.nn + j) * 5 + lane];
      y[(size_t)e * nb + 5 * (p - G.nin) + lane] = val;
    }
  }
}

}  // namespace

namespace sc {

// Host tables of the packed layout (per mesh): column lists per node slot, row offsets,
// and the slot-pair position table used by the packing kernel.
void build_packed_pattern(sc_ctx* c) {
  const Geo& G = c->G;
  const int nn = G.nn, p1 = G.p;
  c->pk_lptr.assign(nn + 1, 0);
  c->pk_list.clear();
  c->pk_pos.assign((size_t)nn * nn, -1);
  auto nat = [&](int slot, int d) {
    const int m = c->iperm[slot];
    return d == 0 ? m % p1 : d == 1 ? (m / p1) % p1 : m / (p1 * p1);
  };
  for (int p = 0; p < nn; ++p) {
    int len = 0;
    for (int q = 0; q < nn; ++q) {
      if (p < G.nin && q < G.nin) { c->pk_pos[(size_t)p * nn + q] = -2; continue; }  // A_ii: not packed
      const bool share = nat(p, 0) == nat(q, 0) || nat(p, 1) == nat(q, 1) || nat(p, 2) == nat(q, 2);
      if (!share) continue;
      c->pk_pos[(size_t)p * nn + q] = len++;
      c->pk_list.push_back(own_col(G, q, 0));
    }
    c->pk_lptr[p + 1] = c->pk_lptr[p] + len;
  }
  c->pk_nint.assign(nn, 0);
  for (int p = 0; p < nn; ++p)
    for (int i = c->pk_lptr[p]; i < c->pk_lptr[p + 1]; ++i) c->pk_nint[p] += c->pk_list[i] < G.ni ? 5 : 0;
  c->pk_row_off.assign(G.ne + 1, 0);
  c->pk_nnz_int = c->pk_nnz_bnd = 0;
  for (int r = 0; r < G.ne; ++r) {
    const int p = r / 5, n = 5 * (c->pk_lptr[p + 1] - c->pk_lptr[p]);
    c->pk_row_off[r + 1] = c->pk_row_off[r] + ((n + 3) & ~3);
    (r < G.ni ? c->pk_nnz_int : c->pk_nnz_bnd) += n;
  }
  c->pk_stride = c->pk_row_off[G.ne];
}

cudaError_t upload_packed_pattern(sc_ctx* c) {
  cudaError_t e = cudaMemcpy(c->d_pk_lptr, c->pk_lptr.data(), c->pk_lptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_pk_list, c->pk_list.data(), c->pk_list.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_pk_row_off, c->pk_row_off.data(), c->pk_row_off.size() * sizeof(int),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_pk_pos, c->pk_pos.data(), c->pk_pos.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_pk_nint, c->pk_nint.data(), c->pk_nint.size() * sizeof(int), cudaMemcpyHostToDevice);
  return e;
}

// Pack the FP64 own blocks into the operator's precision (mixed arm: and write their
// dense FP32 copy).
cudaError_t pack_own(sc_ctx* c) {
  const Geo& G = c->G;
  count_launch(c);
  if (c->cfg.precision == SC_PREC_MIXED)
    k_pack<float><<<G.K, 256, 0, c->stream>>>(G, c->Aown, c->d_pk_row_off, c->d_pk_pos, c->Apk32, c->pk_stride,
                                              c->d_status, c->Aown32);
  else
    k_pack<double><<<G.K, 256, 0, c->stream>>>(G, c->Aown, c->d_pk_row_off, c->d_pk_pos, c->Apk, c->pk_stride,
                                               c->d_status, nullptr);
  return cudaGetLastError();
}

template <class T>
cudaError_t cond_interior_pk(sc_ctx* c, const T* Apk, const T* X, const T* Ainv, const T* xb, double beta,
                             const double* Bfull, double alpha, T* u, int black_zero) {
  const Geo& G = c->G;
  const size_t smem = (size_t)(G.lda + G.ldi) * sizeof(T);
  k_cond_interior_pk<T><<<G.K, 256, smem, c->stream>>>(G, Apk, c->pk_stride, c->d_pk_row_off, c->d_pk_lptr,
                                                       c->d_pk_list, X, c->d_nbr, c->d_pptr, c->d_pinfo, Ainv,
                                                       c->d_iperm, xb, beta, Bfull, alpha, u, black_zero);
  return cudaGetLastError();
}

template <class T>
cudaError_t cond_boundary_pk(sc_ctx* c, const T* Apk, const T* X, const T* xb, double delta, const double* Bfull,
                             double gamma_, const T* u, double* y) {
  const Geo& G = c->G;
  const size_t smem = (size_t)G.lda * sizeof(T);
  k_cond_boundary_pk<T><<<G.K, 256, smem, c->stream>>>(G, Apk, c->pk_stride, c->d_pk_row_off, c->d_pk_lptr,
                                                       c->d_pk_list, X, c->d_nbr, c->d_pptr, c->d_pinfo, c->d_iperm,
                                                       xb, delta, Bfull, gamma_, u, y, nullptr, nullptr);
  return cudaGetLastError();
}

// y_e = (A_bb x_b)_e - (A_bi u)_e for the elements of a list only (rows of one colour), whose
// own boundary values in x_b are zero (the black elements in the red-black sweep): their packed
// rows are read in the interior columns only (a quarter of the own-block bytes at N = 4).
template <class T>
cudaError_t cond_boundary_pk_list(sc_ctx* c, const T* Apk, const T* X, const T* xb, const T* u, double* y,
                                  const int* elist, int nlist) {
  const Geo& G = c->G;
  if (nlist <= 0) return cudaSuccess;
  const size_t smem = (size_t)G.lda * sizeof(T);
  ProfScope ps(c, SCK_COND_BOUNDARY, nlist);
  k_cond_boundary_pk<T><<<nlist, 256, smem, c->stream>>>(G, Apk, c->pk_stride, c->d_pk_row_off, c->d_pk_lptr,
                                                         c->d_pk_list, X, c->d_nbr, c->d_pptr, c->d_pinfo,
                                                         c->d_iperm, xb, 1.0, nullptr, 0.0, G.ni ? u : nullptr, y,
                                                         elist, c->d_pk_nint);
  return cudaGetLastError();
}
template cudaError_t cond_boundary_pk_list<float>(sc_ctx*, const float*, const float*, const float*, const float*,
                                                  double*, const int*, int);
template cudaError_t cond_boundary_pk_list<double>(sc_ctx*, const double*, const double*, const double*,
                                                   const double*, double*, const int*, int);

template cudaError_t cond_interior_pk<float>(sc_ctx*, const float*, const float*, const float*, const float*, double,
                                             const double*, double, float*, int);
template cudaError_t cond_interior_pk<double>(sc_ctx*, const double*, const double*, const double*, const double*,
                                              double, const double*, double, double*, int);
template cudaError_t cond_boundary_pk<float>(sc_ctx*, const float*, const float*, const float*, double, const double*,
                                             double, const float*, double*);
template cudaError_t cond_boundary_pk<double>(sc_ctx*, const double*, const double*, const double*, double,
                                              const double*, double, const double*, double*);

}  // namespace sc
