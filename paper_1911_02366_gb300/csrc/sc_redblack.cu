// Red-black block Gauss-Seidel preconditioner of the condensed system S x_b = g
// (Sec. 2.2, eq. SC_step1), and the learned correction of its black face blocks.
//
// Not in the paper, whose GMRES on the condensed system uses point Jacobi (Sec. 4).  The
// elements are coloured like a checkerboard (ex + ey + ez even: red, odd: black), so that
// every face neighbour of a red element is black and vice versa (edge neighbours share the
// colour; on meshes with an odd n the periodic wrap also joins some face neighbours of one
// colour).  One application z = P v of the preconditioner is one forward block sweep:
//   z_r = S_rr^-1 v_r                          for every red element r,
//   z_b = D_b^-1 (v_b - sum_{red n} S_bn z_n)  for every black element b,
// with D_b = S_bb (SC_PC_RED_BLACK) or S_bb + C_b (SC_PC_LEARNED).  The couplings
// sum S_bn z_n are the black rows of S z for z zero on the black elements, which the
// implicit operator passes give: the interior pass over every element, then the boundary
// pass over the black elements only.
//
// C_b approximates the node-diagonal 5 x 5 blocks of the Schur correction that eliminating
// the red face neighbours would add to the black block, -sum_n [S_bn S_nn^-1 S_nb]_kk: a
// network predicts it from local features (the block-ILU view of the sweep: with this
// correction the black blocks carry what the red elements do to them).
#include "sc_internal.cuh"

namespace {

// dst[i] = src[list[i]] for nb x lds FP32 blocks.
__global__ void k_gather_blocks(int nb, int lds, const float* __restrict__ src, const int* __restrict__ list,
                                float* __restrict__ dst) {
  const long long per = (long long)nb * lds;
  const int i = blockIdx.y;
  const float* s = src + (long long)__ldg(list + i) * per;
  float* d = dst + (long long)i * per;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per; t += (long long)gridDim.x * blockDim.x)
    d[t] = s[t];
}

// SeeL[i] += scale C_k on the diagonal node blocks of black element list[i]; C per sample
// (element e, boundary node a) in the condensed order, 25 floats row-major.
__global__ void k_add_node_blocks(int nbn, int lds, int nlist, const int* __restrict__ list,
                                  const float* __restrict__ Ck, float scale, float* __restrict__ SeeL) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nlist * nbn * 25) return;
  const int i = (int)(t / ((long long)nbn * 25)), rem = (int)(t % ((long long)nbn * 25));
  const int a = rem / 25, r = (rem / 5) % 5, l = rem % 5;
  const int e = __ldg(list + i);
  const int nb = 5 * nbn;
  SeeL[(long long)i * nb * lds + (long long)(5 * a + r) * lds + 5 * a + l] +=
      scale * Ck[((long long)e * nbn + a) * 25 + 5 * r + l];
}

}  // namespace

namespace sc {

void build_colours(sc_ctx* c) {
  const Geo& G = c->G;
  const int n = G.n;
  c->colour_list.clear();
  for (int colour = 0; colour < 2; ++colour)
    for (int e = 0; e < G.K; ++e) {
      const int ex = e % n, ey = (e / n) % n, ez = e / (n * n);
      if (((ex + ey + ez) & 1) == colour) c->colour_list.push_back(e);
    }
  c->n_red = 0;
  for (int e = 0; e < G.K; ++e) c->n_red += ((e % n + (e / n) % n + e / (n * n)) & 1) == 0;
  c->n_black = G.K - c->n_red;
}

bool rb_active(const sc_ctx* c) {
  if (!c->d_colour) return false;
  if (c->cfg.precond == SC_PC_RED_BLACK) return true;
  return c->cfg.precond == SC_PC_LEARNED && c->learned_on && c->blackL_valid;
}

// FP64 arm: z = P v (z must not alias v).
cudaError_t precond_rb(sc_ctx* c, const double* v, double* z) {
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb;
  cudaError_t e = cudaMemsetAsync(z, 0, n1 * sizeof(double), c->stream);
  if (e == cudaSuccess) e = lu_solve_list(c, c->Sls, c->rowperm, 0, c->d_colour, c->n_red, v, nullptr, z);
  if (e == cudaSuccess) e = cond_interior(c, z, 1.0, nullptr, 0.0, c->Ui);
  if (e == cudaSuccess)
    e = cond_boundary_pk_list<double>(c, c->Apk, c->X, z, c->Ui, c->Trb, c->d_colour + c->n_red, c->n_black);
  if (e == cudaSuccess)
    e = lu_solve_list(c, c->Sls, c->rowperm, 0, c->d_colour + c->n_red, c->n_black, v, c->Trb, z);
  return e;
}

// Mixed arm (FP32 factors and operator): z (double) and / or zf (float) = P v.
cudaError_t precond_rb32(sc_ctx* c, const double* v, double* z, float* zf) {
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb;
  float* zt = zf ? zf : c->Zrb;
  const bool learned = c->cfg.precond == SC_PC_LEARNED && c->learned_on && c->blackL_valid;
  const int* black = c->d_colour + c->n_red;
  cudaError_t e = cudaMemsetAsync(zt, 0, n1 * sizeof(float), c->stream);
  if (e == cudaSuccess) e = lu_solve_list32(c, c->Sls32, c->rowperm, 0, c->d_colour, c->n_red, v, nullptr, z, zt);
  if (e == cudaSuccess) e = cond_interior32(c, zt, 1.0, nullptr, 0.0, c->Uf);
  if (e == cudaSuccess) e = cond_boundary_pk_list<float>(c, c->Apk32, c->X32, zt, c->Uf, c->Trb, black, c->n_black);
  if (e == cudaSuccess) {
    if (learned)
      e = lu_solve_list32(c, c->SlsL, c->rowpermL, 1, black, c->n_black, v, c->Trb, z, zt);
    else
      e = lu_solve_list32(c, c->Sls32, c->rowperm, 0, black, c->n_black, v, c->Trb, z, zt);
  }
  return e;
}

// Copy of the black elements' S_ee blocks before their factorisation (condensation).
cudaError_t gather_black_see(sc_ctx* c, const float* See) {
  const Geo& G = c->G;
  if (!c->SeeB || c->n_black == 0) return cudaSuccess;
  count_launch(c);
  k_gather_blocks<<<dim3(64, c->n_black), 256, 0, c->stream>>>(G.nb, G.lds, See, c->d_colour + c->n_red, c->SeeB);
  return cudaGetLastError();
}

// Corrected black blocks S_bb + scale C (C per sample, K nbn x 25; null: no correction),
// factorised into the compact black solve layout.
cudaError_t learned_black_factor(sc_ctx* c, const float* Ck, float scale) {
  const Geo& G = c->G;
  c->blackL_valid = false;
  if (!c->SeeB || c->n_black == 0) return cudaSuccess;
  const size_t per = (size_t)G.nb * G.lds;
  cudaError_t e = cudaMemcpyAsync(c->SeeL, c->SeeB, (size_t)c->n_black * per * sizeof(float),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return e;
  if (Ck) {
    const long long nt = (long long)c->n_black * G.nbn * 25;
    count_launch(c);
    k_add_node_blocks<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(G.nbn, G.lds, c->n_black,
                                                                          c->d_colour + c->n_red, Ck, scale, c->SeeL);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  e = factor_batch32(c, c->SeeL, G.nb, G.lds, (long long)per, c->n_black, c->pivL, c->rowpermL, c->SlsL,
                     c->d_status);
  if (e == cudaSuccess) c->blackL_valid = true;
  return e;
}

}  // namespace sc
