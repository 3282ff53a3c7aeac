// Learned correction of the red-black block sweep of the condensed system (not in the
// paper; its GMRES runs on S x_b = g of Sec. 2.2, eq. SC_step1).  For boundary node k of a
// black element b (checkerboard colouring, ex + ey + ez odd), with f the lowest-index face of
// b containing k (order -x, +x, -y, +y, -z, +z), n the neighbour across f and k' the node of n
// at the same point:
//   features (128): q_k over free-stream scales | [S_bb]_kk, S_(k,k'), S_(k',k''), [S_nn]_(k'k'),
//                  each over its Frobenius norm (k'' the co-located node across the lowest face
//                  of n containing k', k itself on a single face) | (Ma, Re / 1000, dt c_inf / h,
//                  N) | (faces of b containing k) / 3 | the norms of the three coupling /
//                  neighbour blocks over that of [S_bb]_kk | 0 x 15
//   correction    C_k = net(features) ||[S_bb]_kk||_F, added to the diagonal node block k of
//                  S_bb before it is factorised for the black half of the sweep
//   target        C*_k / ||[S_bb]_kk||_F with C*_k = -(1/2) sum_{red m} [S_bm S_mm^-1 S_mb]_kk:
//                  half the node-diagonal part of what eliminating the red neighbours adds to
//                  the black block (the whole of it over-corrects: the off-diagonal node
//                  blocks it leaves out would have balanced it).
// The coupling block of S between k and k' has three parts (no other element reaches a
// boundary row of b through its interior):
//   S_(k,k') = A_bb[k,k'] - A_bi,e[k,:] A_ii,e^-1 A_ib[e_int, k'] - A_bi[k, n_int] Y_n[:, k']
// with Y_n = A_ii,n^-1 A_ib,n (kept transposed by the mixed condensation).
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "sc_internal.cuh"

namespace {

// 5 x 5 diagonal node blocks of the S_ee blocks (before factorisation).
__global__ void k_extract_sdiag(int nb, const float* __restrict__ See, long long sS, int lds,
                                float* __restrict__ out, int nsmp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsmp * 25) return;
  const int s = t / 25, r = (t / 5) % 5, cc = t % 5;
  const int nbn = nb / 5, e = s / nbn, a = s % nbn;
  out[t] = See[(long long)e * sS + (long long)(5 * a + r) * lds + 5 * a + cc];
}

// S_(k,k') for every (element, boundary node): one warp per sample.
__global__ void __launch_bounds__(256) k_learned_coupling(Geo G, const float* __restrict__ Aown, const float* __restrict__ Ainv,
    const float* __restrict__ X, const int* __restrict__ pptr, const int* __restrict__ pinfo,
    const int* __restrict__ iperm, const int* __restrict__ nbr, const int* __restrict__ lface,
    const int* __restrict__ lmirror, const float* __restrict__ Y, int y_transposed, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int nbn = G.nbn, ni = G.ni, nb = G.nb;
  const int smp = blockIdx.x * (blockDim.x / 32) + warp;
  if (smp >= G.K * nbn) return;
  const int e = smp / nbn, a = smp % nbn;
  const int f = __ldg(lface + a), am = __ldg(lmirror + a);
  const int n = __ldg(nbr + e * 18 + f);
  float* t = reinterpret_cast<float*>(smem_raw) + (size_t)warp * (ni * 5 + 32);  // [ni][5] = A_ii^-1 A_ib[:, k']
  int* hits = reinterpret_cast<int*>(t + ni * 5);                                 // up to 32 (node, pair) hits
  for (int i = lane; i < ni * 5; i += 32) t[i] = 0.f;
  __shared__ int nhit_s[8];
  if (lane == 0) nhit_s[warp] = 0;
  __syncwarp();
  // pairs of e's interior nodes with the neighbour dof k' (boundary column 5 am of n)
  for (int pi = 0; pi < G.nin; ++pi) {
    const int j = __ldg(iperm + pi), q0 = __ldg(pptr + j), q1 = __ldg(pptr + j + 1);
    for (int q = q0 + lane; q < q1; q += 32) {
      const int info = __ldg(pinfo + q);
      if (pinfo_slot(info) == f && !pinfo_interior(info) && pinfo_offset(info) == 5 * am) {
        const int h = atomicAdd(&nhit_s[warp], 1);
        if (h < 16) { hits[2 * h] = pi; hits[2 * h + 1] = q; }
      }
    }
  }
  __syncwarp();
  const int nh = min(nhit_s[warp], 16);
  const float* Ie = Ainv + (size_t)e * ni * G.ldi;
  const size_t xs = (size_t)G.NP * 5;  // X stride between row variables
  for (int h = 0; h < nh; ++h) {
    const int pi = hits[2 * h], q = hits[2 * h + 1];
    const float* Xq = X + ((size_t)e * 5 * G.NP + q) * 5;
    for (int r = lane; r < ni; r += 32) {
#pragma unroll
      for (int kv = 0; kv < 5; ++kv) {
        const float av = Ie[(size_t)r * G.ldi + 5 * pi + kv];
#pragma unroll
        for (int l = 0; l < 5; ++l) t[r * 5 + l] = fmaf(av, __ldg(Xq + kv * xs + l), t[r * 5 + l]);
      }
    }
  }
  __syncwarp();
  // term 2: A_bi,e[k, :] t  (rows of node a in the own block, interior columns)
  float acc[25];
#pragma unroll
  for (int i = 0; i < 25; ++i) acc[i] = 0.f;
  const float* Ae = Aown + (size_t)e * own_stride(G) + (size_t)(ni + 5 * a) * G.lda;
  for (int r = lane; r < ni; r += 32) {
#pragma unroll
    for (int kv = 0; kv < 5; ++kv) {
      const float rv = Ae[(size_t)kv * G.lda + r];
#pragma unroll
      for (int l = 0; l < 5; ++l) acc[kv * 5 + l] = fmaf(-rv, t[r * 5 + l], acc[kv * 5 + l]);
    }
  }
  // terms 1 and 3 from the pairs of node a itself
  const int ja = __ldg(iperm + G.nin + a), q0 = __ldg(pptr + ja), q1 = __ldg(pptr + ja + 1);
  const float* Yn = Y + (size_t)n * nb * G.ldi;
  for (int q = q0 + lane; q < q1; q += 32) {
    const int info = __ldg(pinfo + q);
    if (pinfo_slot(info) != f) continue;
    const int off = pinfo_offset(info);
    const float* Xq = X + ((size_t)e * 5 * G.NP + q) * 5;
    if (!pinfo_interior(info)) {
      if (off == 5 * am)
#pragma unroll
        for (int kv = 0; kv < 5; ++kv)
#pragma unroll
          for (int l = 0; l < 5; ++l) acc[kv * 5 + l] += __ldg(Xq + kv * xs + l);
    } else {
      // - A_bi[k, n_int(off..off+4)] Y_n[off.., k']
#pragma unroll
      for (int l = 0; l < 5; ++l)
#pragma unroll
        for (int kk = 0; kk < 5; ++kk) {
          const float yv = y_transposed ? Yn[(size_t)(5 * am + kk) * G.ldi + off + l]
                                        : Y[(size_t)n * ni * nb + (size_t)(off + l) * nb + 5 * am + kk];
#pragma unroll
          for (int kv = 0; kv < 5; ++kv) acc[kv * 5 + kk] = fmaf(-__ldg(Xq + kv * xs + l), yv, acc[kv * 5 + kk]);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 25; ++i) {
    float v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[(size_t)smp * 25 + i] = v;
  }
}

__device__ __forceinline__ void put_unit(float* dst, const float* src, float* norm_out) {
  float s = 0.f;
  for (int i = 0; i < 25; ++i) s = fmaf(src[i], src[i], s);
  const float nrm = sqrtf(s);
  const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
  for (int i = 0; i < 25; ++i) dst[i] = src[i] * inv;
  if (norm_out) *norm_out = nrm;
}

__global__ void k_learned_features(Geo G, const double* __restrict__ Q, const int* __restrict__ iperm,
                                   const float* __restrict__ Sdiag, const float* __restrict__ Cpl, float4 scal,
                                   float e_inf, const int* __restrict__ nfaces, const int* __restrict__ nbr,
                                   const int* __restrict__ lface, const int* __restrict__ lmirror,
                                   float* __restrict__ F, float* __restrict__ snorm) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= G.K * G.nbn) return;
  const int e = s / G.nbn, a = s % G.nbn;
  const int j = __ldg(iperm + G.nin + a);
  // the neighbour's own sample at the co-located node k'
  const int sm = __ldg(nbr + e * 18 + __ldg(lface + a)) * G.nbn + __ldg(lmirror + a);
  float* f = F + (size_t)s * 128;
  const double* q = Q + ((size_t)e * G.nn + j) * 5;
  f[0] = (float)q[0]; f[1] = (float)q[1]; f[2] = (float)q[2]; f[3] = (float)q[3]; f[4] = (float)(q[4] / e_inf);
  float nk = 0.f, n1 = 0.f, n2 = 0.f, n3 = 0.f;
  put_unit(f + 5, Sdiag + (size_t)s * 25, &nk);
  put_unit(f + 30, Cpl + (size_t)s * 25, &n1);
  put_unit(f + 55, Cpl + (size_t)sm * 25, &n2);
  put_unit(f + 80, Sdiag + (size_t)sm * 25, &n3);
  f[105] = scal.x; f[106] = scal.y; f[107] = scal.z; f[108] = scal.w;
  f[109] = (float)__ldg(nfaces + a) * (1.0f / 3.0f);
  const float ik = nk > 0.f ? 1.f / nk : 0.f;
  f[110] = n1 * ik; f[111] = n2 * ik; f[112] = n3 * ik;
  for (int i = 113; i < 128; ++i) f[i] = 0.f;
  snorm[s] = nk;
}

__global__ void k_set_unit(double* x, size_t n, long long on, long long off) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t == 0 && off >= 0) x[off] = 0.0;
  if (t == 0 && on >= 0) x[on] = 1.0;
  (void)n;
}

// Share of the node-diagonal Schur correction the target keeps.
constexpr float kLearnedDamping = 0.5f;

// T[s] = -kLearnedDamping sum_{pairs p of b} [S_bm X_p]_(k,k) / ||[S_bb]_kk||_F for every sample
// s = (black element b, boundary node a); red samples get zero.  X_p = S_mm^-1 S_mb with
// column j contiguous (k_solve_cols); S column by column with n1 rows.
__global__ void k_black_targets(int nb, int nbn, long long n1, const double* __restrict__ Scm,
                                const float* __restrict__ X, const int* __restrict__ bidx,
                                const int* __restrict__ pptr, const int* __restrict__ pm,
                                const float* __restrict__ snorm, int nsmp, float* __restrict__ T) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nsmp * 25) return;
  const int smp = (int)(t / 25), r = (int)((t / 5) % 5), l = (int)(t % 5);
  const int e = smp / nbn, a = smp % nbn;
  const int bi = __ldg(bidx + e);
  if (bi < 0) { T[t] = 0.f; return; }
  const long long row = (long long)e * nb + 5 * a + r;
  double acc = 0.0;
  for (int p = __ldg(pptr + bi); p < __ldg(pptr + bi + 1); ++p) {
    const long long m0 = (long long)__ldg(pm + p) * nb;
    const float* xc = X + ((long long)p * nb + 5 * a + l) * nb;
    for (int i = 0; i < nb; ++i) acc += Scm[(m0 + i) * n1 + row] * (double)xc[i];
  }
  const float sn = snorm[smp];
  T[t] = sn > 0.f ? (float)(-(double)kLearnedDamping * acc) / sn : 0.f;
}

// C_k = y_k ||[S_ee]_kk||_F (the network works on blocks scaled by the node's own block)
__global__ void k_scale_correction(int nsmp, const float* __restrict__ Y, const float* __restrict__ snorm,
                                   float* __restrict__ Ck) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsmp * 25) return;
  Ck[t] = Y[t] * snorm[t / 25];
}

}  // namespace

namespace sc {

// Per boundary position: lowest-index face containing the node and the boundary position
// of the co-located node of the neighbour across it.
void build_learned_tables(sc_ctx* c) {
  const Geo& G = c->G;
  const int p = G.p, N = G.N;
  c->l_face.assign(G.nbn, 0);
  c->l_mirror.assign(G.nbn, 0);
  c->l_nfaces.assign(G.nbn, 0);
  for (int a = 0; a < G.nbn; ++a) {
    const int m = c->iperm[G.nin + a];
    int cc[3] = {m % p, (m / p) % p, m / (p * p)};
    int f = -1;
    for (int d = 0; d < 3 && f < 0; ++d) {
      if (cc[d] == 0) f = 2 * d;
      else if (cc[d] == N) f = 2 * d + 1;
    }
    c->l_face[a] = f;
    c->l_nfaces[a] = (cc[0] == 0 || cc[0] == N) + (cc[1] == 0 || cc[1] == N) + (cc[2] == 0 || cc[2] == N);
    cc[f / 2] = N - cc[f / 2];
    const int mm = cc[0] + p * (cc[1] + p * cc[2]);
    c->l_mirror[a] = c->perm[mm] - G.nin;
  }
}

cudaError_t extract_sdiag(sc_ctx* c, const float* See) {
  const Geo& G = c->G;
  const int nsmp = G.K * G.nbn;
  count_launch(c);
  k_extract_sdiag<<<(nsmp * 25 + 255) / 256, 256, 0, c->stream>>>(G.nb, See, (long long)G.nb * G.lds, G.lds,
                                                                   c->Sdiag, nsmp);
  return cudaGetLastError();
}

// Features of every (element, boundary node) of the current condensed system.
cudaError_t learned_features(sc_ctx* c, float* F, float* snorm) {
  const Geo& G = c->G;
  const int nsmp = G.K * G.nbn;
  const size_t smem = (size_t)8 * (G.ni * 5 + 32) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_learned_coupling, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch(c, 2);
  k_learned_coupling<<<(nsmp + 7) / 8, 256, smem, c->stream>>>(G, c->Aown32, c->Ainv32, c->X32, c->d_pptr,
      c->d_pinfo, c->d_iperm, c->d_nbr, c->d_lface, c->d_lmirror, c->Y32, c->cfg.tensor_cores ? 1 : 0, c->Cpl);
  const double Ma = c->cfg.Ma, gamma = c->cfg.gamma;
  const double p_inf = 1.0 / (gamma * Ma * Ma);
  const float e_inf = (float)(p_inf / (gamma - 1.0) + 0.5);
  const float4 scal = make_float4((float)Ma, (float)(c->cfg.Re / 1000.0), (float)(G.dt * (1.0 / Ma) / G.h),
                                  (float)G.N);
  k_learned_features<<<(nsmp + 255) / 256, 256, 0, c->stream>>>(G, c->Q, c->d_iperm, c->Sdiag, c->Cpl, scal, e_inf,
                                                                c->d_lnfaces, c->d_nbr, c->d_lface, c->d_lmirror, F,
                                                                snorm);
  return cudaGetLastError();
}

// Network on the features, scaled into the per-node corrections C_k.
cudaError_t learned_correction(sc_ctx* c) {
  const Geo& G = c->G;
  const int nsmp = G.K * G.nbn;
  cudaError_t e = learned_features(c, c->Feat, c->Snorm);
  if (e == cudaSuccess)
    e = mlp_forward(c->stream, c->Wbf16, c->Wbias, c->Feat, nsmp, c->Ynet, c->Hbuf, c->Hbuf + (size_t)nsmp * 256);
  if (e != cudaSuccess) return e;
  count_launch(c, 4);
  k_scale_correction<<<(nsmp * 25 + 255) / 256, 256, 0, c->stream>>>(nsmp, c->Ynet, c->Snorm, c->Ck);
  return cudaGetLastError();
}

}  // namespace sc

extern "C" {

sc_status sc_learned_features(sc_ctx* c, float* F, float* snorm) {
  if (!c || !F || !snorm) return SC_ERR_ARG;
  if (!c->condensed || c->cfg.precision != SC_PREC_MIXED || !c->Sdiag_valid)
    return SC_ERR_STATE;
  if (sc::learned_features(c, F, snorm) != cudaSuccess) return SC_ERR_CUDA;
  return cudaStreamSynchronize(c->stream) == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

sc_status sc_learned_targets(sc_ctx* c, float* T) {
  if (!c || !T) return SC_ERR_ARG;
  if (!c->condensed || c->cfg.precision != SC_PREC_MIXED || !c->Sdiag_valid) return SC_ERR_STATE;
  const Geo& G = c->G;
  const long long n1 = (long long)G.K * G.nb;
  const int nsmp = G.K * G.nbn;
  if ((double)n1 * n1 * 8.0 > 40e9) return SC_ERR_ARG;  // training meshes only
  // pairs (black element, distinct red neighbour), grouped by black element
  std::vector<int> hb, hm, hptr(1, 0), hbidx(G.K, -1);
  for (int i = c->n_red; i < G.K; ++i) {
    const int b = c->colour_list[i];
    hbidx[b] = i - c->n_red;
    std::vector<int> seen;
    for (int sl = 0; sl < 18; ++sl) {
      const int m = c->nbr[(size_t)b * 18 + sl];
      const int ex = m % G.n, ey = (m / G.n) % G.n, ez = m / (G.n * G.n);
      if (((ex + ey + ez) & 1) != 0 || std::find(seen.begin(), seen.end(), m) != seen.end()) continue;
      seen.push_back(m);
      hb.push_back(b); hm.push_back(m);
    }
    hptr.push_back((int)hb.size());
  }
  const int npairs = (int)hb.size();
  cudaStream_t st = c->stream;
  double* Scm = nullptr;
  float *X = nullptr, *F = nullptr, *sn = nullptr;
  int *pb = nullptr, *pm = nullptr, *pptr = nullptr, *bidx = nullptr;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(cudaMalloc(&Scm, (size_t)n1 * n1 * sizeof(double)));
  A(cudaMalloc(&X, (size_t)std::max(npairs, 1) * G.nb * G.nb * sizeof(float)));
  A(cudaMalloc(&F, (size_t)nsmp * 128 * sizeof(float)));
  A(cudaMalloc(&sn, (size_t)nsmp * sizeof(float)));
  A(cudaMalloc(&pb, std::max(npairs, 1) * sizeof(int))); A(cudaMalloc(&pm, std::max(npairs, 1) * sizeof(int)));
  A(cudaMalloc(&pptr, hptr.size() * sizeof(int))); A(cudaMalloc(&bidx, G.K * sizeof(int)));
  sc_status status = SC_OK;
  if (e != cudaSuccess) { status = SC_ERR_OOM; goto done; }
  {
    // S column by column through the condensed operator (the system the method forms)
    double* xb = c->Xfull;  // K ne >= n1 doubles of scratch
    A(cudaMemsetAsync(xb, 0, (size_t)n1 * sizeof(double), st));
    for (long long jcol = 0; jcol < n1 && e == cudaSuccess; ++jcol) {
      k_set_unit<<<1, 32, 0, st>>>(xb, (size_t)n1, jcol, jcol - 1);
      A(sc::vec_to_float(c, c->Xbf, xb, (size_t)n1));
      A(sc::cond_interior32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf));
      A(sc::cond_boundary32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf, Scm + jcol * n1));
    }
    if (npairs > 0) {
      A(cudaMemcpyAsync(pb, hb.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, st));
      A(cudaMemcpyAsync(pm, hm.data(), npairs * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    A(cudaMemcpyAsync(pptr, hptr.data(), hptr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    A(cudaMemcpyAsync(bidx, hbidx.data(), G.K * sizeof(int), cudaMemcpyHostToDevice, st));
    if (npairs > 0) A(sc::solve_columns32(c, Scm, n1, pb, pm, npairs, X));
    A(sc::learned_features(c, F, sn));
    if (e == cudaSuccess) {
      count_launch(c);
      const long long nt = (long long)nsmp * 25;
      k_black_targets<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(G.nb, G.nbn, n1, Scm, X, bidx, pptr, pm, sn,
                                                                    nsmp, T);
      A(cudaGetLastError());
    }
    A(cudaStreamSynchronize(st));
    if (e != cudaSuccess) status = SC_ERR_CUDA;
  }
done:
  cudaFree(Scm); cudaFree(X); cudaFree(F); cudaFree(sn); cudaFree(pb); cudaFree(pm); cudaFree(pptr); cudaFree(bidx);
  return status;
}

sc_status sc_set_learned_correction(sc_ctx* c, const float* Ck, float scale) {
  if (!c || !Ck) return SC_ERR_ARG;
  if (!c->condensed || !c->SeeB) return SC_ERR_STATE;
  if (sc::learned_black_factor(c, Ck, scale) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
    return SC_ERR_CUDA;
  c->weights_set = true;  // the corrected black factors are in place; the next sc_solve uses them
  return SC_OK;
}

sc_status sc_set_learned_weights(sc_ctx* c, const uint16_t* Wbf16, const float* bias) {
  if (!c || !Wbf16 || !bias) return SC_ERR_ARG;
  if (!c->Wbf16) return SC_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(c->Wbf16, Wbf16, (size_t)sc::kMlpWeights * sizeof(uint16_t),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->Wbias, bias, (size_t)sc::kMlpBiases * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return SC_ERR_CUDA;
  c->weights_set = true;
  return SC_OK;
}

sc_status sc_load_mlp(sc_ctx* c, const char* path) {
  if (!c || !path) return SC_ERR_ARG;
  if (!c->Wbf16) return SC_ERR_STATE;
  float *W = nullptr, *b = nullptr;
  uint16_t* Wh = nullptr;
  cudaError_t e = cudaMalloc(&W, (size_t)sc::kMlpWeights * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b, (size_t)sc::kMlpBiases * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&Wh, (size_t)sc::kMlpWeights * sizeof(uint16_t));
  sc_status s = e == cudaSuccess ? sc_mlp_load(path, W, Wh, b) : SC_ERR_OOM;
  if (s == SC_OK) s = sc_set_learned_weights(c, Wh, b);
  else c->err = "load_mlp: cannot read a network from the file";
  cudaFree(W); cudaFree(b); cudaFree(Wh);
  return s;
}

}  // extern "C"
