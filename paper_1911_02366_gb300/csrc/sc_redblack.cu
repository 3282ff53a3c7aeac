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
// with D_b = S_bb (SC_PC_RED_BLACK) or S_bb + C_b (SC_PC_LEARNED, SC_PC_RB_SCHUR).  The couplings
// sum S_bn z_n are the black rows of S z for z zero on the black elements, which the
// implicit operator passes give: the interior pass over every element, then the boundary
// pass over the black elements only.
//
// Eliminating the red unknowns leaves the black Schur complement
// Sigma = S_bb - S_br S_rr^-1 S_rb, and the sweep's preconditioned operator has the spectrum
// of D^-1 Sigma (plus ones): the best block-diagonal D is the block diagonal of Sigma.
// SC_PC_RB_SCHUR forms it through the co-located couplings of each shared face,
//   C_b[k,l] = -sum_f S_(k,k'_f) [S_mm^-1]_(k'_f,l'_f) S_(l'_f,l)      (k, l on face f of b),
// from the red neighbour's explicit inverse; SC_PC_LEARNED keeps the node-diagonal blocks
// of a correction assembled from the network's inverse node blocks.
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

// D_i -= sum over the faces f of black element b = list[i], over the node pairs (k, l) on f:
// S_(k,k') [S_mm^-1]_(k',l') S_(l',l), m the neighbour across f (skipped when it is black, on
// meshes with an odd n), k', l' the nodes of m at the points of k, l.  Cpl holds S_(k,k'_f) per
// (sample, face slot); Zinv the red inverses column-major.  One CTA per black element, faces
// in turn (the pairs of one face write distinct entries; an edge node's pairs meet again on
// its other faces).
__global__ void __launch_bounds__(256) k_face_schur(Geo G, const int* __restrict__ list, const int* __restrict__ redidx,
                                                    const float* __restrict__ Zinv, const float* __restrict__ Cpl,
                                                    const int* __restrict__ nbr, const int* __restrict__ ftab,
                                                    const int* __restrict__ lmirror3, const int* __restrict__ lrslot3,
                                                    float* __restrict__ SeeL) {
  const int i = blockIdx.x, b = __ldg(list + i);
  const int P2 = (G.N + 1) * (G.N + 1), nb = G.nb, nbn = G.nbn;
  float* D = SeeL + (long long)i * nb * G.lds;
  for (int f = 0; f < 6; ++f) {
    const int m = __ldg(nbr + (long long)b * 18 + f);
    const int ri = __ldg(redidx + m);
    if (ri >= 0) {
      const float* Z = Zinv + (long long)ri * nb * nb;
      const int* fa = ftab + 2 * f * P2;
      const int* fs = fa + P2;
      for (int p = threadIdx.x; p < P2 * P2; p += blockDim.x) {
        const int ia = p % P2, ib = p / P2;
        const int a = __ldg(fa + ia), sa = __ldg(fs + ia), bb = __ldg(fa + ib), sb = __ldg(fs + ib);
        const int am = __ldg(lmirror3 + 3 * a + sa), bm = __ldg(lmirror3 + 3 * bb + sb);
        const float* Skc = Cpl + ((long long)(b * nbn + a) * 3 + sa) * 25;                           // S_(k,k')
        const float* Sck = Cpl + ((long long)(m * nbn + bm) * 3 + __ldg(lrslot3 + 3 * bb + sb)) * 25;  // S_(l',l)
        float T[25];  // [S_mm^-1]_(k',l') S_(l',l)
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
          for (int cc = 0; cc < 5; ++cc) T[5 * r + cc] = 0.f;
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          const float* zc = Z + (long long)(5 * bm + t) * nb + 5 * am;  // column 5 l' + t, rows of k'
          float zr[5], sr[5];
#pragma unroll
          for (int r = 0; r < 5; ++r) zr[r] = __ldg(zc + r);
#pragma unroll
          for (int cc = 0; cc < 5; ++cc) sr[cc] = __ldg(Sck + 5 * t + cc);
#pragma unroll
          for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int cc = 0; cc < 5; ++cc) T[5 * r + cc] = fmaf(zr[r], sr[cc], T[5 * r + cc]);
        }
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          float u[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int t = 0; t < 5; ++t) {
            const float k = __ldg(Skc + 5 * r + t);
#pragma unroll
            for (int cc = 0; cc < 5; ++cc) u[cc] = fmaf(k, T[5 * t + cc], u[cc]);
          }
          float* drow = D + (long long)(5 * a + r) * G.lds + 5 * bb;
#pragma unroll
          for (int cc = 0; cc < 5; ++cc) drow[cc] -= u[cc];
        }
      }
    }
    __syncthreads();
  }
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
  c->red_index.assign(G.K, -1);
  for (int i = 0; i < c->n_red; ++i) c->red_index[c->colour_list[i]] = i;
}

// face_tab: per face f the boundary nodes on f (condensed order) and the slot of f in each
// node's face list (the learned tables l_face3 hold the faces of every boundary node).
void build_face_tables(sc_ctx* c) {
  const Geo& G = c->G;
  const int P2 = (G.N + 1) * (G.N + 1);
  c->face_tab.assign(12 * (size_t)P2, 0);
  for (int f = 0; f < 6; ++f) {
    int t = 0;
    for (int a = 0; a < G.nbn; ++a)
      for (int i = 0; i < c->l_nfaces[a]; ++i)
        if (c->l_face3[3 * a + i] == f && t < P2) {  // (N+1)^2 boundary nodes on every face
          c->face_tab[2 * f * P2 + t] = a;
          c->face_tab[(2 * f + 1) * P2 + t] = i;
          ++t;
        }
  }
}

bool rb_active(const sc_ctx* c) {
  if (!c->d_colour) return false;
  if (c->cfg.precond == SC_PC_RED_BLACK || c->cfg.precond == SC_PC_RB_SCHUR) return true;
  return c->cfg.precond == SC_PC_LEARNED && c->learned_on && c->blackL_valid;
}

// FP64 arm: z = P v (z must not alias v).
cudaError_t precond_rb(sc_ctx* c, const double* v, double* z) {
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb;
  cudaError_t e = cudaMemsetAsync(z, 0, n1 * sizeof(double), c->stream);
  if (e == cudaSuccess) e = lu_solve_list(c, c->Sls, c->rowperm, 0, c->d_colour, c->n_red, v, nullptr, z);
  if (e == cudaSuccess) e = cond_interior_sweep(c, z, c->Ui);
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
  const bool corrected = c->blackL_valid && ((c->cfg.precond == SC_PC_LEARNED && c->learned_on) ||
                                             c->cfg.precond == SC_PC_RB_SCHUR);
  const int* black = c->d_colour + c->n_red;
  cudaError_t e = cudaMemsetAsync(zt, 0, n1 * sizeof(float), c->stream);
  if (e == cudaSuccess)
    e = lu_solve_list32(c, c->Sls32, c->rowperm, c->red_compact ? 1 : 0, c->d_colour, c->n_red, v, nullptr, z, zt);
  if (e == cudaSuccess) e = cond_interior_sweep32(c, zt, c->Uf);
  if (e == cudaSuccess) e = cond_boundary_pk_list<float>(c, c->Apk32, c->X32, zt, c->Uf, c->Trb, black, c->n_black);
  if (e == cudaSuccess) {
    if (corrected)
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

// Corrected black blocks S_bb + scale C (C per sample, K nbn x 25; null: no correction), plus
// the face-block Schur correction when face_schur is set (couplings in Cpl and the red
// inverses in Zinv already formed), factorised into the compact black solve layout.
static cudaError_t black_factor(sc_ctx* c, const float* Ck, float scale, bool face_schur) {
  const Geo& G = c->G;
  c->blackL_valid = false;
  if (!c->SeeB || c->n_black == 0) return cudaSuccess;
  const size_t per = (size_t)G.nb * G.lds;
  cudaError_t e = cudaMemcpyAsync(c->SeeL, c->SeeB, (size_t)c->n_black * per * sizeof(float),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return e;
  if (face_schur) {
    count_launch(c);
    k_face_schur<<<c->n_black, 256, 0, c->stream>>>(G, c->d_colour + c->n_red, c->d_redidx, c->Zinv, c->Cpl, c->d_nbr,
                                                    c->d_face_tab, c->d_lmirror3, c->d_lrslot3, c->SeeL);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (Ck) {
    const long long nt = (long long)c->n_black * G.nbn * 25;
    count_launch(c);
    k_add_node_blocks<<<(unsigned)((nt + 255) / 256), 256, 0, c->stream>>>(G.nbn, G.lds, c->n_black,
                                                                          c->d_colour + c->n_red, Ck, scale, c->SeeL);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  e = factor_batch32(c, c->SeeL, G.nb, G.lds, (long long)per, c->n_black, c->pivL, c->rowpermL, c->SlsL,
                     c->d_status + 2);
  if (e == cudaSuccess) c->blackL_valid = true;
  return e;
}

cudaError_t learned_black_factor(sc_ctx* c, const float* Ck, float scale) { return black_factor(c, Ck, scale, false); }

// SC_PC_RB_SCHUR after the condensation: couplings, red inverses, corrected black factors.
cudaError_t schur_black_factor(sc_ctx* c) {
  if (!c->Zinv || !c->SeeB || c->n_black == 0) {
    c->blackL_valid = false;
    return cudaSuccess;
  }
  cudaError_t e = learned_couplings(c);
  if (e == cudaSuccess) e = inverse_columns32(c, c->red_compact ? nullptr : c->d_colour, c->n_red, c->Zinv);
  if (e == cudaSuccess) e = black_factor(c, nullptr, 0.f, true);
  return e;
}

// The red blocks alone (SC_PC_RB_SCHUR): gathered into SeeL (free until the black correction)
// and factorised into the first n_red entries of the solve layout and of rowperm.
cudaError_t red_factor32(sc_ctx* c, const float* See) {
  const Geo& G = c->G;
  if (c->n_red == 0) return cudaSuccess;
  count_launch(c);
  k_gather_blocks<<<dim3(64, c->n_red), 256, 0, c->stream>>>(G.nb, G.lds, See, c->d_colour, c->SeeL);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t per = (size_t)G.nb * G.lds;
  return factor_batch32(c, c->SeeL, G.nb, G.lds, (long long)per, c->n_red, c->piv, c->rowperm, c->Sls32,
                        c->d_status);
}

// The plain black blocks into SlsL: the Schur-corrected sweep's fallback when a corrected
// block is singular (its red factors are compact, so the plain sweep takes its black factors
// from here as well).
cudaError_t plain_black_factor(sc_ctx* c) { return black_factor(c, nullptr, 0.f, false); }

}  // namespace sc
