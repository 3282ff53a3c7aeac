// Learned correction of the red-black sweep of the condensed system (not in the paper; its
// GMRES runs on S x_b = g of Sec. 2.2, eq. SC_step1, preconditioned there by point Jacobi).
//
// The black half of the sweep solves with D_b = S_bb + C_b; C_b is block diagonal over the
// 5 x 5 node blocks, one per boundary node k of the black element b:
//   C_k = -(1/2) sum over the faces f of b containing k of S_(k,k'_f) Z_(k'_f) S_(k'_f,k),
// k'_f the node at the same point in the (red) neighbour n_f across f and Z_(k') the diagonal
// node block of the inverse of that neighbour's face block, [S_nn^-1]_(k'k'): the co-located
// part of the Schur correction that eliminating the red neighbours adds to S_bb, halved (the
// off-diagonal node blocks it leaves out would balance it).  Z is what the network provides:
// it predicts, from local features of node k' of element n, the correction of the inverse of
// the node block, Z = [S_nn]_(k'k')^-1 + y / ||[S_nn]_(k'k')||_F (the exact Z needs n_b unit
// solves per element; the network one forward pass per node).  In the solver the output
// enters at half weight (kNetworkDamping).
//   features (128): q_k over free-stream scales | [S_ee]_kk, S_(k,k'), S_(k',k), [S_nn]_(k'k'),
//                  each over its Frobenius norm (k' across the lowest face of e containing k) |
//                  (Ma, Re / 1000, dt c_inf / h, N) | (faces of e containing k) / 3 | the norms
//                  of the last three over that of [S_ee]_kk | 0 x 15
//   target        ([S_ee^-1]_kk - [S_ee]_kk^-1) ||[S_ee]_kk||_F, every element of either colour
// The coupling block of S between k and k'_f has three parts (no other element reaches a
// boundary row of e through its interior):
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
    const int* __restrict__ iperm, const int* __restrict__ nbr, const int* __restrict__ lface3,
    const int* __restrict__ lmirror3, const int* __restrict__ nfaces, const float* __restrict__ Y, int y_transposed,
    float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int nbn = G.nbn, ni = G.ni, nb = G.nb;
  const int w = blockIdx.x * (blockDim.x / 32) + warp;  // (sample, i-th face of its node)
  if (w >= G.K * nbn * 3) return;
  const int smp = w / 3, slot = w % 3;
  const int e = smp / nbn, a = smp % nbn;
  if (slot >= __ldg(nfaces + a)) {  // the node lies on fewer faces: the slot stays zero
    if (lane < 25) out[(size_t)w * 25 + lane] = 0.f;
    return;
  }
  const int f = __ldg(lface3 + 3 * a + slot), am = __ldg(lmirror3 + 3 * a + slot);
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
    if (lane == 0) out[(size_t)w * 25 + i] = v;
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
                                   const int* __restrict__ lface3, const int* __restrict__ lmirror3,
                                   const int* __restrict__ lrslot3, float* __restrict__ F, float* __restrict__ snorm) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= G.K * G.nbn) return;
  const int e = s / G.nbn, a = s % G.nbn;
  const int j = __ldg(iperm + G.nin + a);
  // the neighbour's sample at the co-located node k' across the lowest face of e containing k
  const int sm = __ldg(nbr + e * 18 + __ldg(lface3 + 3 * a)) * G.nbn + __ldg(lmirror3 + 3 * a);
  float* f = F + (size_t)s * 128;
  const double* q = Q + ((size_t)e * G.nn + j) * 5;
  f[0] = (float)q[0]; f[1] = (float)q[1]; f[2] = (float)q[2]; f[3] = (float)q[3]; f[4] = (float)(q[4] / e_inf);
  float nk = 0.f, n1 = 0.f, n2 = 0.f, n3 = 0.f;
  put_unit(f + 5, Sdiag + (size_t)s * 25, &nk);
  put_unit(f + 30, Cpl + (size_t)s * 75, &n1);                                   // S_(k,k')
  put_unit(f + 55, Cpl + ((size_t)sm * 3 + __ldg(lrslot3 + 3 * a)) * 25, &n2);  // S_(k',k)
  put_unit(f + 80, Sdiag + (size_t)sm * 25, &n3);                                // [S_nn]_(k'k')
  f[105] = scal.x; f[106] = scal.y; f[107] = scal.z; f[108] = scal.w;
  f[109] = (float)__ldg(nfaces + a) * (1.0f / 3.0f);
  const float ik = nk > 0.f ? 1.f / nk : 0.f;
  f[110] = n1 * ik; f[111] = n2 * ik; f[112] = n3 * ik;
  for (int i = 113; i < 128; ++i) f[i] = 0.f;
  snorm[s] = nk;
}

// Inverse of a 5 x 5 matrix (row-major) by Gauss-Jordan elimination with partial pivoting;
// false (and B untouched) when a pivot vanishes.
__device__ bool inv5(const float* A, float* B) {
  float M[5][10];
  for (int r = 0; r < 5; ++r)
    for (int cc = 0; cc < 5; ++cc) { M[r][cc] = A[5 * r + cc]; M[r][5 + cc] = r == cc ? 1.f : 0.f; }
  for (int k = 0; k < 5; ++k) {
    int p = k;
    for (int r = k + 1; r < 5; ++r)
      if (fabsf(M[r][k]) > fabsf(M[p][k])) p = r;
    if (M[p][k] == 0.f) return false;
    if (p != k)
      for (int cc = 0; cc < 10; ++cc) { const float t = M[k][cc]; M[k][cc] = M[p][cc]; M[p][cc] = t; }
    const float ip = 1.f / M[k][k];
    for (int cc = 0; cc < 10; ++cc) M[k][cc] *= ip;
    for (int r = 0; r < 5; ++r) {
      if (r == k) continue;
      const float fct = M[r][k];
      if (fct != 0.f)
        for (int cc = 0; cc < 10; ++cc) M[r][cc] -= fct * M[k][cc];
    }
  }
  for (int r = 0; r < 5; ++r)
    for (int cc = 0; cc < 5; ++cc) B[5 * r + cc] = M[r][5 + cc];
  return true;
}

// Targets T[s] = ([S_ee^-1]_kk - [S_ee]_kk^-1) ||[S_ee]_kk||_F for every sample.
__global__ void k_inverse_targets(int nsmp, const float* __restrict__ Zex, const float* __restrict__ Sdiag,
                                  float* __restrict__ T) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsmp) return;
  float B[25], nk = 0.f;
  for (int i = 0; i < 25; ++i) nk = fmaf(Sdiag[(size_t)s * 25 + i], Sdiag[(size_t)s * 25 + i], nk);
  nk = sqrtf(nk);
  if (!inv5(Sdiag + (size_t)s * 25, B))
    for (int i = 0; i < 25; ++i) B[i] = 0.f;
  for (int i = 0; i < 25; ++i) T[(size_t)s * 25 + i] = (Zex[(size_t)s * 25 + i] - B[i]) * nk;
}

// C_k = -(1/2) sum_f S_(k,k'_f) Z_(k'_f) S_(k'_f,k) for the samples of black elements (zero for
// red ones), Z_(k') = [S_nn]_(k'k')^-1 + scale y_(k') / ||[S_nn]_(k'k')||_F.
__global__ void k_assemble_correction(Geo G, const float* __restrict__ Y, float scale,
                                      const float* __restrict__ Sdiag, const float* __restrict__ Cpl,
                                      const int* __restrict__ nbr, const int* __restrict__ nfaces,
                                      const int* __restrict__ lface3, const int* __restrict__ lmirror3,
                                      const int* __restrict__ lrslot3, float* __restrict__ C) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= G.K * G.nbn) return;
  const int e = s / G.nbn, a = s % G.nbn;
  float acc[25];
  for (int i = 0; i < 25; ++i) acc[i] = 0.f;
  const int ex = e % G.n, ey = (e / G.n) % G.n, ez = e / (G.n * G.n);
  if (((ex + ey + ez) & 1) == 1) {
    for (int i = 0; i < __ldg(nfaces + a); ++i) {
      const int sm = __ldg(nbr + e * 18 + __ldg(lface3 + 3 * a + i)) * G.nbn + __ldg(lmirror3 + 3 * a + i);
      const float* Sd = Sdiag + (size_t)sm * 25;
      float Z[25], nk = 0.f;
      for (int t = 0; t < 25; ++t) nk = fmaf(Sd[t], Sd[t], nk);
      nk = sqrtf(nk);
      if (!inv5(Sd, Z)) continue;
      const float sc = nk > 0.f ? scale / nk : 0.f;
      for (int t = 0; t < 25; ++t) Z[t] = fmaf(sc, Y[(size_t)sm * 25 + t], Z[t]);
      const float* Skc = Cpl + ((size_t)s * 3 + i) * 25;                            // S_(k,k')
      const float* Sck = Cpl + ((size_t)sm * 3 + __ldg(lrslot3 + 3 * a + i)) * 25;  // S_(k',k)
      float ZS[25];
      for (int r = 0; r < 5; ++r)
        for (int cc = 0; cc < 5; ++cc) {
          float v = 0.f;
          for (int t = 0; t < 5; ++t) v = fmaf(Z[5 * r + t], Sck[5 * t + cc], v);
          ZS[5 * r + cc] = v;
        }
      for (int r = 0; r < 5; ++r)
        for (int cc = 0; cc < 5; ++cc) {
          float v = 0.f;
          for (int t = 0; t < 5; ++t) v = fmaf(Skc[5 * r + t], ZS[5 * t + cc], v);
          acc[5 * r + cc] -= 0.5f * v;
        }
    }
  }
  for (int i = 0; i < 25; ++i) C[(size_t)s * 25 + i] = acc[i];
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
  c->l_face3.assign(3 * G.nbn, 0);
  c->l_mirror3.assign(3 * G.nbn, 0);
  c->l_rslot3.assign(3 * G.nbn, 0);
  auto faces_of = [&](int m, int out[3]) {
    const int cc[3] = {m % p, (m / p) % p, m / (p * p)};
    int k = 0;
    for (int d = 0; d < 3; ++d) {
      if (cc[d] == 0) out[k++] = 2 * d;
      else if (cc[d] == N) out[k++] = 2 * d + 1;
    }
    return k;
  };
  for (int a = 0; a < G.nbn; ++a) {
    const int m = c->iperm[G.nin + a];
    int fl[3];
    const int nf = faces_of(m, fl);
    c->l_nfaces[a] = nf;
    for (int i = 0; i < nf; ++i) {
      const int f = fl[i];
      int cc[3] = {m % p, (m / p) % p, m / (p * p)};
      cc[f / 2] = N - cc[f / 2];
      const int mm = cc[0] + p * (cc[1] + p * cc[2]);
      int fr[3];
      const int nr = faces_of(mm, fr);
      int rs = 0;
      for (int t = 0; t < nr; ++t)
        if (fr[t] == (f ^ 1)) rs = t;  // the mirrored node's slot of the face back to e
      c->l_face3[3 * a + i] = f;
      c->l_mirror3[3 * a + i] = c->perm[mm] - G.nin;
      c->l_rslot3[3 * a + i] = rs;
    }
    c->l_face[a] = c->l_face3[3 * a];
    c->l_mirror[a] = c->l_mirror3[3 * a];
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

// Couplings S_(k,k'_f) of every (element, boundary node, face of the node) into Cpl.
cudaError_t learned_couplings(sc_ctx* c) {
  const Geo& G = c->G;
  const int nsmp = G.K * G.nbn;
  const size_t smem = (size_t)8 * (G.ni * 5 + 32) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_learned_coupling, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launch(c);
  k_learned_coupling<<<(3 * nsmp + 7) / 8, 256, smem, c->stream>>>(G, c->Aown32, c->Ainv32, c->X32, c->d_pptr,
      c->d_pinfo, c->d_iperm, c->d_nbr, c->d_lface3, c->d_lmirror3, c->d_lnfaces, c->Y32,
      c->cfg.tensor_cores ? 1 : 0, c->Cpl);
  return cudaGetLastError();
}

// Features of every (element, boundary node) of the current condensed system.
cudaError_t learned_features(sc_ctx* c, float* F, float* snorm) {
  const Geo& G = c->G;
  const int nsmp = G.K * G.nbn;
  cudaError_t e = learned_couplings(c);
  if (e != cudaSuccess) return e;
  count_launch(c);
  const double Ma = c->cfg.Ma, gamma = c->cfg.gamma;
  const double p_inf = 1.0 / (gamma * Ma * Ma);
  const float e_inf = (float)(p_inf / (gamma - 1.0) + 0.5);
  const float4 scal = make_float4((float)Ma, (float)(c->cfg.Re / 1000.0), (float)(G.dt * (1.0 / Ma) / G.h),
                                  (float)G.N);
  k_learned_features<<<(nsmp + 255) / 256, 256, 0, c->stream>>>(G, c->Q, c->d_iperm, c->Sdiag, c->Cpl, scal, e_inf,
                                                                c->d_lnfaces, c->d_nbr, c->d_lface3, c->d_lmirror3,
                                                                c->d_lrslot3, F, snorm);
  return cudaGetLastError();
}

// The black blocks' corrections C from network outputs Y (per sample, target form) into c->Ck;
// the couplings of every face come from the last learned_features.
cudaError_t assemble_correction(sc_ctx* c, const float* Y, float scale) {
  const Geo& G = c->G;
  const int nsmp = G.K * G.nbn;
  count_launch(c);
  k_assemble_correction<<<(nsmp + 127) / 128, 128, 0, c->stream>>>(G, Y, scale, c->Sdiag, c->Cpl, c->d_nbr,
                                                                   c->d_lnfaces, c->d_lface3, c->d_lmirror3,
                                                                   c->d_lrslot3, c->Ck);
  return cudaGetLastError();
}

// Network on the features, its outputs assembled into the black blocks' corrections C_k.
// The predicted corrections of the inverse node blocks enter halved (kNetworkDamping),
// shrunk towards the closed form Z = [S_nn]_(k'k')^-1: the corrected black blocks amplify
// errors in Z, and a network whose median relative error is 0.14 on the 16^3, N = 4 systems
// gave 575 GMRES iterations at full weight, 152 at half weight (closed form 170).
constexpr float kNetworkDamping = 0.5f;

cudaError_t learned_correction(sc_ctx* c) {
  const Geo& G = c->G;
  const int nsmp = G.K * G.nbn;
  cudaError_t e = learned_features(c, c->Feat, c->Snorm);
  if (e == cudaSuccess)
    e = mlp_forward(c->stream, c->Wbf16, c->Wbias, c->Feat, nsmp, c->Ynet, c->Hbuf, c->Hbuf + (size_t)nsmp * 256);
  if (e == cudaSuccess) e = assemble_correction(c, c->Ynet, kNetworkDamping);
  return e;
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
  const int nsmp = G.K * G.nbn;
  float* Zex = nullptr;
  if (cudaMalloc(&Zex, (size_t)nsmp * 25 * sizeof(float)) != cudaSuccess) return SC_ERR_OOM;
  cudaError_t e = sc::inverse_node_blocks32(c, Zex);
  if (e == cudaSuccess) {
    count_launch(c);
    k_inverse_targets<<<(nsmp + 127) / 128, 128, 0, c->stream>>>(nsmp, Zex, c->Sdiag, T);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(Zex);
  return e == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

sc_status sc_set_learned_correction(sc_ctx* c, const float* Y, float scale) {
  if (!c || !Y) return SC_ERR_ARG;
  if (!c->condensed || !c->SeeB || !c->Ck || !c->Feat) return SC_ERR_STATE;
  cudaError_t e = sc::learned_features(c, c->Feat, c->Snorm);  // the couplings of every face
  if (e == cudaSuccess) e = sc::assemble_correction(c, Y, scale);
  if (e == cudaSuccess) e = sc::learned_black_factor(c, c->Ck, 1.0f);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return SC_ERR_CUDA;
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
