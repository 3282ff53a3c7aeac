// Explicit Schur complement over the extended boundary sets (Sec. 2.2, eq.
// StaticCondBlock; Sec. 3.2): for every element e,
//   Y_e = A_ii,e^-1 A_ib[e_int, E_e]      (ni x m)
//   W_e = A_bi[E_e, e_int] Y_e            (m x m)
//   S   = A_bb - sum_e P_e^T W_e P_e
// where E_e holds e's own boundary dofs (nb) followed, face by face (-x, +x, -y, +y, -z,
// +z), by the dofs of the face neighbour that sit on the shared face ((N+1)^2 nodes, 5
// variables each): m = nb + 30 (N+1)^2 (1240 at N = 4).  Interior rows of e couple to
// neighbours only through those face dofs, and a neighbour's boundary rows reach e's
// interior only from that face, so W_e carries every Schur term of e.
//
// The explicit operator, y = A_bb x - sum_e P_e^T (W_e (P_e x)), is an alternative to the
// implicit one the solver uses: it reads the m^2 entries of W_e per element per product
// instead of the packed element blocks.  The mixed arm forms it with the TF32 tensor-core
// products (or FP32 CUDA cores) and applies it in FP32.
#include "sc_internal.cuh"

namespace {

// A_ib[e_int, E_e] (ni x ldm) and A_bi[E_e, e_int] (m x ldi) from the own block and the
// neighbour couplings.  Buffers are zero on entry.
__global__ void __launch_bounds__(256) k_gather_ext(Geo G, const float* __restrict__ Aown, const float* __restrict__ X,
    const int* __restrict__ nbr, const int* __restrict__ pptr, const int* __restrict__ pinfo,
    const int* __restrict__ iperm, const int* __restrict__ ex_nbpos, const int* __restrict__ ex_face_idx, int F,
    int ldm, float* __restrict__ Aib, float* __restrict__ Abi, int* __restrict__ status) {
  const int e = blockIdx.x, ni = G.ni, nb = G.nb, nbn = G.nbn;
  const float* Ae = Aown + (size_t)e * own_stride(G);
  float* Ib = Aib + (size_t)e * ni * ldm;
  const int m = nb + 30 * F;
  float* Bi = Abi + (size_t)e * m * G.ldi;
  const size_t xs = (size_t)G.NP * 5;
  // own parts
  for (int t = threadIdx.x; t < ni * nb; t += blockDim.x) {
    const int r = t / nb, cc = t % nb;
    Ib[(size_t)r * ldm + cc] = Ae[(size_t)r * G.lda + G.cb0 + cc];
  }
  for (int t = threadIdx.x; t < nb * ni; t += blockDim.x) {
    const int r = t / ni, cc = t % ni;
    Bi[(size_t)r * G.ldi + cc] = Ae[(size_t)(ni + r) * G.lda + cc];
  }
  // interior rows of e -> face dofs of the neighbours
  for (int pi = 0; pi < G.nin; ++pi) {
    const int j = __ldg(iperm + pi), q0 = __ldg(pptr + j), q1 = __ldg(pptr + j + 1);
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
      const int info = __ldg(pinfo + q), slot = pinfo_slot(info);
      if (pinfo_interior(info)) continue;
      int i = -1;
      if (slot < 6) i = __ldg(ex_face_idx + slot * nbn + pinfo_offset(info) / 5);
      if (i < 0) { atomicCAS(status, -1, SC_EXPLICIT_PATTERN); continue; }
      const float* Xq = X + ((size_t)e * 5 * G.NP + q) * 5;
      for (int kv = 0; kv < 5; ++kv)
        for (int l = 0; l < 5; ++l)
          Ib[(size_t)(5 * pi + kv) * ldm + nb + slot * 5 * F + 5 * i + l] = __ldg(Xq + kv * xs + l);
    }
  }
  // face dofs of each neighbour -> interior of e (from the neighbour's couplings)
  for (int f = 0; f < 6; ++f) {
    const int n = __ldg(nbr + e * 18 + f), fb = f ^ 1;
    for (int i = 0; i < F; ++i) {
      const int ap = __ldg(ex_nbpos + f * F + i);
      const int mm = __ldg(iperm + G.nin + ap), q0 = __ldg(pptr + mm), q1 = __ldg(pptr + mm + 1);
      for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        const int info = __ldg(pinfo + q);
        if (!pinfo_interior(info) || pinfo_slot(info) != fb) continue;
        const int off = pinfo_offset(info);
        const float* Xq = X + ((size_t)n * 5 * G.NP + q) * 5;
        for (int kv = 0; kv < 5; ++kv)
          for (int l = 0; l < 5; ++l)
            Bi[(size_t)(nb + f * 5 * F + 5 * i + kv) * G.ldi + off + l] = __ldg(Xq + kv * xs + l);
      }
    }
  }
}

// y -= P_e^T (W_e (P_e x)) for every element; one CTA per element, two rows per warp.
__global__ void __launch_bounds__(256) k_explicit_w(Geo G, const float* __restrict__ W, int ldm,
    const int* __restrict__ nbr, const int* __restrict__ ex_nbpos, int F, const float* __restrict__ x,
    double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* xe = reinterpret_cast<float*>(smem_raw);
  const int e = blockIdx.x, nb = G.nb, m = nb + 30 * F;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  __shared__ int nb_s[6];
  if (threadIdx.x < 6) nb_s[threadIdx.x] = nbr[e * 18 + threadIdx.x];
  __syncthreads();
  for (int c = threadIdx.x; c < ldm; c += blockDim.x) {
    float v = 0.f;
    if (c < nb) {
      v = x[(size_t)e * nb + c];
    } else if (c < m) {
      const int t = c - nb, f = t / (5 * F), i = (t % (5 * F)) / 5, l = t % 5;
      v = x[(size_t)nb_s[f] * nb + 5 * __ldg(ex_nbpos + f * F + i) + l];
    }
    xe[c] = v;
  }
  __syncthreads();
  const float* We = W + (size_t)e * m * ldm;
  for (int ra = 2 * warp; ra < m; ra += 2 * nw) {
    const int rb = ra + 1 < m ? ra + 1 : ra;
    const float4* wa = reinterpret_cast<const float4*>(We + (size_t)ra * ldm);
    const float4* wb = reinterpret_cast<const float4*>(We + (size_t)rb * ldm);
    const float4* xv = reinterpret_cast<const float4*>(xe);
    float sa = 0.f, sb = 0.f;
#pragma unroll 4
    for (int c4 = lane; c4 < ldm / 4; c4 += 32) {
      const float4 a = __ldg(wa + c4), b = __ldg(wb + c4), v = xv[c4];
      sa = fmaf(a.x, v.x, fmaf(a.y, v.y, fmaf(a.z, v.z, fmaf(a.w, v.w, sa))));
      sb = fmaf(b.x, v.x, fmaf(b.y, v.y, fmaf(b.z, v.z, fmaf(b.w, v.w, sb))));
    }
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (lane < 2 && (lane == 0 || rb != ra)) {
      const int r = lane == 0 ? ra : rb;
      const float s = lane == 0 ? sa : sb;
      size_t dst;
      if (r < nb) {
        dst = (size_t)e * nb + r;
      } else {
        const int t = r - nb, f = t / (5 * F), i = (t % (5 * F)) / 5, kv = t % 5;
        dst = (size_t)nb_s[f] * nb + 5 * __ldg(ex_nbpos + f * F + i) + kv;
      }
      atomicAdd(y + dst, -(double)s);
    }
  }
}

}  // namespace

namespace sc {

// Face node tables of the extended boundary set: for face f and its i-th node (natural
// order), the boundary position of the neighbour's co-located node, and the inverse map.
void build_explicit_tables(sc_ctx* c) {
  const Geo& G = c->G;
  const int p = G.p, N = G.N, F = p * p;
  c->ex_F = F;
  c->ex_m = G.nb + 30 * F;
  c->ex_ldm = (c->ex_m + 3) & ~3;
  c->ex_nbpos.assign(6 * F, 0);
  c->ex_face_idx.assign((size_t)6 * G.nbn, -1);
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, side = f % 2 ? N : 0;
    int i = 0;
    for (int mnat = 0; mnat < G.nn; ++mnat) {
      int cc[3] = {mnat % p, (mnat / p) % p, mnat / (p * p)};
      if (cc[d] != side) continue;
      cc[d] = N - cc[d];
      const int mm = cc[0] + p * (cc[1] + p * cc[2]);
      const int ap = c->perm[mm] - G.nin;
      c->ex_nbpos[f * F + i] = ap;
      c->ex_face_idx[(size_t)f * G.nbn + ap] = i;
      ++i;
    }
  }
}

cudaError_t upload_explicit_tables(sc_ctx* c) {
  cudaError_t e = cudaMemcpy(c->d_ex_nbpos, c->ex_nbpos.data(), c->ex_nbpos.size() * sizeof(int),
                             cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_ex_face_idx, c->ex_face_idx.data(), c->ex_face_idx.size() * sizeof(int),
                   cudaMemcpyHostToDevice);
  return e;
}

size_t explicit_elems_W(const Geo& G, const sc_ctx* c) { return (size_t)G.K * c->ex_m * c->ex_ldm; }

// Y_e and W_e for every element (after the FP32 element blocks and A_ii^-1 exist).
cudaError_t explicit_build(sc_ctx* c) {
  const Geo& G = c->G;
  const int m = c->ex_m, ldm = c->ex_ldm, ni = G.ni, K = G.K;
  cudaError_t e = cudaMemsetAsync(c->ExIb, 0, (size_t)K * ni * ldm * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ExBi, 0, (size_t)K * m * G.ldi * sizeof(float), c->stream);
  if (e != cudaSuccess) return e;
  count_launch(c);
  k_gather_ext<<<K, 256, 0, c->stream>>>(G, c->Aown32, c->X32, c->d_nbr, c->d_pptr, c->d_pinfo, c->d_iperm,
                                         c->d_ex_nbpos, c->d_ex_face_idx, c->ex_F, ldm, c->ExIb, c->ExBi,
                                         c->d_status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ProfScope ps(c, SCK_EXPLICIT_GEMM);
  count_launch(c);
  if (c->cfg.tensor_cores) {
    e = gemm_tf32(c->stream, ni, m, ni, 1.0f, c->Ainv32, (long long)ni * G.ldi, G.ldi, false, c->ExIb,
                  (long long)ni * ldm, ldm, false, 0.0f, c->ExY, (long long)ni * ldm, ldm, K, c->d_status);
    if (e == cudaSuccess)
      e = gemm_tf32(c->stream, m, m, ni, 1.0f, c->ExBi, (long long)m * G.ldi, G.ldi, false, c->ExY,
                    (long long)ni * ldm, ldm, false, 0.0f, c->ExW, (long long)m * ldm, ldm, K, c->d_status);
  } else {
    e = gemm_fp32(c, ni, m, ni, c->Ainv32, (long long)ni * G.ldi, G.ldi, c->ExIb, (long long)ni * ldm, ldm, c->ExY,
                  (long long)ni * ldm, ldm, K);
    if (e == cudaSuccess)
      e = gemm_fp32(c, m, m, ni, c->ExBi, (long long)m * G.ldi, G.ldi, c->ExY, (long long)ni * ldm, ldm, c->ExW,
                    (long long)m * ldm, ldm, K);
  }
  return e;
}

// y = S x with the explicit Schur blocks: the packed A_bb pass (own and neighbour
// couplings), then the W_e products subtracted at the extended dofs.
cudaError_t explicit_matvec32(sc_ctx* c, const float* x, double* y) {
  const Geo& G = c->G;
  cudaError_t e = cond_boundary_pk<float>(c, c->Apk32, c->X32, x, 1.0, nullptr, 0.0, nullptr, y);
  if (e != cudaSuccess) return e;
  ProfScope ps(c, SCK_EXPLICIT_APPLY);
  const size_t smem = (size_t)c->ex_ldm * sizeof(float);
  k_explicit_w<<<G.K, 256, smem, c->stream>>>(G, c->ExW, c->ex_ldm, c->d_nbr, c->d_ex_nbpos, c->ex_F, x, y);
  return cudaGetLastError();
}

}  // namespace sc
