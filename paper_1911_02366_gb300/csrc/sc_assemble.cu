// Residual and Jacobian assembly of the GL-DGSEM Newton system on the GPU.
//
// Residual (Sec. 2.1, eq. DGSEMsystem, in the strong form that summation by parts
// gives on Gauss-Lobatto nodes):
//   g_a(m) = (2/h) [ sum_b D[m_a][b] q(m with coord a = b)
//                    + (1/w_N) (1/2)(q_nb - q_m)  on the +a face, - on the -a face ]   (BR1)
//   R_j = c0 J W_j (q_j - q_hist)/dt + Jf W_j sum_a sum_b D[j_a][b] F_a(m_b)
//         + sum_{faces f of j} Jf W^f_j [ fhat_f(j) - s_f F_{d_f}(j) ]
// with F = f^a - f^nu, fhat = Roe(q+, q-) - (1/2) s (f^nu_d(+) + f^nu_d(-)), J = (h/2)^3,
// Jf = (h/2)^2, W_j the tensor GL weight.  With the symmetric interior penalty (the paper's
// experiment, Sec. 4) the face flux takes f^nu at each side's own unlifted gradient
// Dq = (2/h) sum_b D[m_a][b] q(...) instead of the lifted one and adds sigma (q+ - q-); the
// volume flux F keeps the lifted gradient (qhat = {{q}}), which supplies the symmetrising
// term.  The unlifted gradients depend on their own element only, so the edge-neighbour
// couplings of BR1 vanish.
//
// Jacobian (Sec. 2.1.1-2.1.2, eqs. AdvImpDG, DiffImpDGouter, GradDGImp): the point flux
// Jacobians dF_d/dq, df^nu_d/dq and df^nu_d/dg_a, and the Roe derivatives, are
// evaluated per node with a five-direction dual number; the element blocks then follow
// from the chain rule through the (linear) lifting operator, which is non-zero only
// along grid lines:
//   dR_j/dq_r = delta_jr c0 J W_j/dt
//     + sum_d sum_{m on the d-line of j} Jf W_j D[j_d][m_d] [ delta_mr dF_d/dq(m)
//                                            + sum_a L_a(m, r) dF_d/dg_a(m) ]
//     + surface terms of the faces of j (own and neighbour lifting, Roe derivatives).
// L_a(m, r) = (2/h) D[m_a][r_a] (r on the a-line of m) + 1/(h w_N) (-[m_a = N] + [m_a = 0])
// for r = m, and +- 1/(h w_N) for the neighbour node across the a-face.
#include "sc_internal.cuh"

namespace {

constexpr int NJC = 375;  // node Jacobian components: Fq(3x25) | fvq(3x25) | fvg(9x25)

SC_HD inline void node_coords(int m, int p, int c[3]) {
  c[0] = m % p; c[1] = (m / p) % p; c[2] = m / (p * p);
}
SC_HD inline int node_index(const int c[3], int p) { return c[0] + p * (c[1] + p * c[2]); }

__global__ void k_history(Geo G, const double* __restrict__ Qs, const double* __restrict__ Qsm1,
                          double* __restrict__ Qh, size_t n, int bdf) {
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  Qh[t] = (bdf == 2) ? (4.0 * Qs[t] - Qsm1[t]) / 3.0 : Qs[t];
}

// Lifted gradients, one thread per node.
SC_HD void lift_body(const Geo& G, const double* Q, const int* nbr, int t, double* grad, int lifted) {
  const int e = t / G.nn, m = t % G.nn, p = G.p, N = G.N;
  int c[3]; node_coords(m, p, c);
  const double* qe = Q + (size_t)e * G.nn * 5;
  const double* qm = qe + (size_t)m * 5;
  for (int a = 0; a < 3; ++a) {
    double acc[5] = {0, 0, 0, 0, 0};
    int cc[3] = {c[0], c[1], c[2]};
    for (int b = 0; b < p; ++b) {
      cc[a] = b;
      const double Dab = G.D[c[a]][b];
      const double* qb = qe + (size_t)node_index(cc, p) * 5;
      for (int k = 0; k < 5; ++k) acc[k] = fma(Dab, qb[k], acc[k]);
    }
    if (lifted && (c[a] == N || c[a] == 0)) {
      const int s = (c[a] == N) ? 1 : -1;
      const int nb = nbr[e * 18 + face_slot(a, s)];
      int cn[3] = {c[0], c[1], c[2]}; cn[a] = N - c[a];
      const double* qn = Q + ((size_t)nb * G.nn + node_index(cn, p)) * 5;
      const double coef = 0.5 * s / G.w[c[a]];
      for (int k = 0; k < 5; ++k) acc[k] = fma(coef, qn[k] - qm[k], acc[k]);
    }
    for (int k = 0; k < 5; ++k) grad[(size_t)t * 15 + a * 5 + k] = G.dx * acc[k];
  }
}

// lifted = 1: the BR1 lifted gradient g; 0: the element's own gradient Dq.
__global__ void k_lift(Geo G, const double* __restrict__ Q, const int* __restrict__ nbr,
                       double* __restrict__ grad, int lifted) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < G.K * G.nn) lift_body(G, Q, nbr, t, grad, lifted);
}

SC_HD inline void load_node(const double* __restrict__ Q, const double* __restrict__ grad,
                                          size_t t, double q[5], double g[3][5]) {
  for (int k = 0; k < 5; ++k) q[k] = Q[t * 5 + k];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 5; ++k) g[a][k] = grad[t * 15 + a * 5 + k];
}

// Point fluxes F_d = f^a_d - f^nu_d, one thread per node.
__global__ void k_flux(Geo G, const double* __restrict__ Q, const double* __restrict__ grad,
                       double* __restrict__ F) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.K * G.nn) return;
  double q[5], g[3][5];
  load_node(Q, grad, t, q, g);
  for (int d = 0; d < 3; ++d) {
    double fa[5], fv[5];
    flux_inviscid(G, q, d, fa);
    flux_viscous(G, q, g, d, fv);
    for (int k = 0; k < 5; ++k) F[(size_t)t * 15 + d * 5 + k] = fa[k] - fv[k];
  }
}

// Residual rows; writes B = -R.  One thread per node.
// gface: the gradients the face flux takes (lifted for BR1, unlifted for the interior penalty).
__global__ void k_resid(Geo G, const double* __restrict__ Q, const double* __restrict__ Qh,
                        const double* __restrict__ gface, const double* __restrict__ F,
                        const int* __restrict__ nbr, double* __restrict__ Bout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G.K * G.nn) return;
  const int e = t / G.nn, j = t % G.nn, p = G.p, N = G.N;
  int c[3]; node_coords(j, p, c);
  const double Wj = G.w[c[0]] * G.w[c[1]] * G.w[c[2]];
  double r[5];
  const double tcoef = G.c0 * G.Jf * 0.5 * G.h * Wj / G.dt;
  for (int k = 0; k < 5; ++k) r[k] = tcoef * (Q[(size_t)t * 5 + k] - Qh[(size_t)t * 5 + k]);
  const size_t e0 = (size_t)e * G.nn;
  for (int d = 0; d < 3; ++d) {
    int cc[3] = {c[0], c[1], c[2]};
    for (int b = 0; b < p; ++b) {
      cc[d] = b;
      const double coef = G.Jf * Wj * G.D[c[d]][b];
      const double* Fm = F + (e0 + node_index(cc, p)) * 15 + d * 5;
      for (int k = 0; k < 5; ++k) r[k] = fma(coef, Fm[k], r[k]);
    }
  }
  for (int d = 0; d < 3; ++d) {
    if (c[d] != 0 && c[d] != N) continue;
    const int s = (c[d] == N) ? 1 : -1;
    const int nb = nbr[e * 18 + face_slot(d, s)];
    int cn[3] = {c[0], c[1], c[2]}; cn[d] = N - c[d];
    const size_t tn = (size_t)nb * G.nn + node_index(cn, p);
    double qa[5], ga[3][5], qb[5], gb[3][5];
    load_node(Q, gface, t, qa, ga);
    load_node(Q, gface, tn, qb, gb);
    double fr[5], fva[5], fvb[5];
    flux_adv(G, qa, qb, d, s, fr);
    flux_viscous(G, qa, ga, d, fva);
    flux_viscous(G, qb, gb, d, fvb);
    const double Sf = G.Jf * Wj / G.w[c[d]];
    for (int k = 0; k < 5; ++k) {
      double fhat = fr[k] - 0.5 * s * (fva[k] + fvb[k]);
      if (G.visc_flux == 1) fhat = fma(G.sigma, qa[k] - qb[k], fhat);
      r[k] = fma(Sf, fhat - s * F[(size_t)t * 15 + d * 5 + k], r[k]);
    }
  }
  for (int k = 0; k < 5; ++k) Bout[(size_t)t * 5 + k] = -r[k];
}

// Point flux Jacobians of every node: NJ[e][comp][m].
SC_HD void nodejac_body(const Geo& G, const double* Q, const double* grad, int t, double* NJ) {
  const int e = t / G.nn, m = t % G.nn;
  double q[5], g[3][5];
  load_node(Q, grad, t, q, g);
  double* out = NJ + (size_t)e * NJC * G.nn + m;
  const size_t cs = G.nn;  // component stride
  {
    D5 qd[5], gd[3][5], fa[5], fv[3][5];
    for (int k = 0; k < 5; ++k) { qd[k] = D5(q[k]); qd[k].d[k] = 1.0; }
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 5; ++k) gd[a][k] = D5(g[a][k]);
    flux_viscous_all(G, qd, gd, fv);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      flux_inviscid(G, qd, d, fa);
      for (int k = 0; k < 5; ++k)
        for (int l = 0; l < 5; ++l) {
          out[(size_t)(d * 25 + k * 5 + l) * cs] = fa[k].d[l] - fv[d][k].d[l];
          out[(size_t)(75 + d * 25 + k * 5 + l) * cs] = fv[d][k].d[l];
        }
    }
  }
#pragma unroll
  for (int ap = 0; ap < 3; ++ap) {
    D5 qd[5], gd[3][5], fv[3][5];
    for (int k = 0; k < 5; ++k) qd[k] = D5(q[k]);
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 5; ++k) {
        gd[a][k] = D5(g[a][k]);
        if (a == ap) gd[a][k].d[k] = 1.0;
      }
    flux_viscous_all(G, qd, gd, fv);
    for (int d = 0; d < 3; ++d)
      for (int k = 0; k < 5; ++k)
        for (int l = 0; l < 5; ++l) out[(size_t)(150 + (d * 3 + ap) * 25 + k * 5 + l) * cs] = fv[d][k].d[l];
  }
}

__global__ void k_nodejac(Geo G, const double* __restrict__ Q, const double* __restrict__ grad,
                          double* __restrict__ NJ) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < G.K * G.nn) nodejac_body(G, Q, grad, t, NJ);
}

// Numerical-flux (Roe or Lax-Friedrichs) derivatives at every face node of every element: RJ[e][f][comp][fidx],
// comp < 25: d fhat/d q+, comp >= 25: d fhat/d q-; fidx = a + p*b over the in-face
// coordinates ((d+1)%3, (d+2)%3).
SC_HD void roejac_body(const Geo& G, const double* Q, const int* nbr, int t, double* RJ) {
  const int pp = G.p * G.p;
  const int e = t / (6 * pp), f = (t / pp) % 6, fidx = t % pp;
  const int d = f / 2, s = (f & 1) ? 1 : -1, N = G.N, p = G.p;
  int c[3]; c[d] = s > 0 ? N : 0; c[(d + 1) % 3] = fidx % p; c[(d + 2) % 3] = fidx / p;
  const int j = node_index(c, p);
  int cn[3] = {c[0], c[1], c[2]}; cn[d] = N - c[d];
  const int nb = nbr[e * 18 + f];
  const double* qa = Q + ((size_t)e * G.nn + j) * 5;
  const double* qb = Q + ((size_t)nb * G.nn + node_index(cn, p)) * 5;
  double* out = RJ + ((size_t)e * 6 + f) * 50 * pp + fidx;
  for (int side = 0; side < 2; ++side) {
    D5 a[5], b[5], fh[5];
    for (int k = 0; k < 5; ++k) { a[k] = D5(qa[k]); b[k] = D5(qb[k]); }
    for (int k = 0; k < 5; ++k) (side == 0 ? a : b)[k].d[k] = 1.0;
    flux_adv(G, a, b, d, s, fh);
    for (int k = 0; k < 5; ++k)
      for (int l = 0; l < 5; ++l) out[(size_t)(side * 25 + k * 5 + l) * pp] = fh[k].d[l];
  }
}

__global__ void k_roejac(Geo G, const double* __restrict__ Q, const int* __restrict__ nbr,
                         double* __restrict__ RJ) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < G.K * 6 * G.p * G.p) roejac_body(G, Q, nbr, t, RJ);
}

// ---- assembly helpers (all data of one element e) --------------------------------
struct ElemView {
  const double* nj;  // NJ of the element
  int nn;
  SC_HD inline double Fq(int d, int m, int kl) const { return nj[(size_t)(d * 25 + kl) * nn + m]; }
  SC_HD inline double fvq(int d, int m, int kl) const { return nj[(size_t)(75 + d * 25 + kl) * nn + m]; }
  SC_HD inline double fvg(int d, int a, int m, int kl) const {
    return nj[(size_t)(150 + (d * 3 + a) * 25 + kl) * nn + m];
  }
};

// Own-lifting coefficient L_a(m, r) for r on the a-line of m (same element).
SC_HD inline double lift_own(const Geo& G, const int cm[3], const int cr[3], int a, bool same) {
  double v = G.dx * G.D[cm[a]][cr[a]];
  if (same) {
    if (cm[a] == G.N) v -= G.inv_hw;
    if (cm[a] == 0) v += G.inv_hw;
  }
  return v;
}

SC_HD inline double wprod(const Geo& G, const int c[3]) { return G.w[c[0]] * G.w[c[1]] * G.w[c[2]]; }

// acc += coef * M where M is a 5x5 component set read through fn(kl)
#define ACC25(coef, EXPR)                                  \
  do {                                                     \
    const double _c = (coef);                              \
    if (_c != 0.0) {                                       \
      _Pragma("unroll") for (int kl = 0; kl < 25; ++kl)    \
        acc[kl] = fma(_c, (EXPR), acc[kl]);                \
    }                                                      \
  } while (0)

// Own element block: rows j, columns r (both in element e).  NJL: the point-flux Jacobians at
// the unlifted gradients (interior penalty only; null with BR1).
template <bool IP>
SC_HD void own_entry(const Geo& G, const double* NJ, const double* NJL, const double* RJ, const int* nbr, int e,
                     int j, int r, double acc[25]) {
  const int nn = G.nn, p = G.p, N = G.N;
  ElemView V{NJ + (size_t)e * NJC * nn, nn};
  constexpr bool ip = IP;
  ElemView VL{ip ? NJL + (size_t)e * NJC * nn : nullptr, nn};
  const int pp = p * p;
  {
    int cj[3], cr[3];
    node_coords(j, p, cj); node_coords(r, p, cr);
    int ndiff = 0, dc[3];
    for (int a = 0; a < 3; ++a) if (cj[a] != cr[a]) dc[ndiff++] = a;
#pragma unroll
    for (int kl = 0; kl < 25; ++kl) acc[kl] = 0.0;
    if (ndiff < 3) {
      const double Wj = wprod(G, cj);
      const double Dwj = G.Jf * Wj;  // Dw_d(j, m) = Dwj * D[j_d][m_d]
      if (ndiff == 0) {
        const double tc = G.c0 * G.Jf * 0.5 * G.h * Wj / G.dt;
        for (int k = 0; k < 5; ++k) acc[k * 6] += tc;
        for (int d = 0; d < 3; ++d) {
          ACC25(Dwj * G.D[cj[d]][cj[d]], V.Fq(d, j, kl));
          int cm[3] = {cj[0], cj[1], cj[2]};
          for (int b = 0; b < p; ++b) {  // (d, d): m along the d-line
            cm[d] = b;
            const int m = node_index(cm, p);
            ACC25(Dwj * G.D[cj[d]][b] * lift_own(G, cm, cj, d, b == cj[d]), -V.fvg(d, d, m, kl));
          }
          for (int a = 0; a < 3; ++a) {  // (d, a != d): m = j
            if (a == d) continue;
            ACC25(Dwj * G.D[cj[d]][cj[d]] * lift_own(G, cj, cj, a, true), -V.fvg(d, a, j, kl));
          }
        }
      } else if (ndiff == 1) {
        const int cdir = dc[0];
        ACC25(Dwj * G.D[cj[cdir]][cr[cdir]], V.Fq(cdir, r, kl));
        int cm[3] = {cj[0], cj[1], cj[2]};
        for (int b = 0; b < p; ++b) {  // (c, c): m along the c-line
          cm[cdir] = b;
          const int m = node_index(cm, p);
          ACC25(Dwj * G.D[cj[cdir]][b] * lift_own(G, cm, cr, cdir, b == cr[cdir]), -V.fvg(cdir, cdir, m, kl));
        }
        for (int a = 0; a < 3; ++a) {
          if (a == cdir) continue;
          // (c, a): m = r
          ACC25(Dwj * G.D[cj[cdir]][cr[cdir]] * lift_own(G, cr, cr, a, true), -V.fvg(cdir, a, r, kl));
          // (a, c): m = j
          ACC25(Dwj * G.D[cj[a]][cj[a]] * lift_own(G, cj, cr, cdir, false), -V.fvg(a, cdir, j, kl));
        }
      } else {  // ndiff == 2
        const int c1 = dc[0], c2 = dc[1];
        for (int o = 0; o < 2; ++o) {
          const int d = o ? c2 : c1, a = o ? c1 : c2;
          int cm[3] = {cj[0], cj[1], cj[2]}; cm[d] = cr[d];
          const int m = node_index(cm, p);
          ACC25(Dwj * G.D[cj[d]][cr[d]] * lift_own(G, cm, cr, a, false), -V.fvg(d, a, m, kl));
        }
      }
      // surface terms of the faces containing j
      if (ndiff <= 1) {
        for (int df = 0; df < 3; ++df) {
          if (cj[df] != 0 && cj[df] != N) continue;
          const int sf = (cj[df] == N) ? 1 : -1;
          const double Sf = G.Jf * Wj / G.w[cj[df]];
          if constexpr (ip) {
            // fhat - s F_d(j): the strong-form term -s F_d(j) keeps the lifted gradient at j
            // (full weight), the face average -s/2 f^nu(q_j, Dq_j) takes the unlifted one
            // (Dq_a(j) = dx D[j_a][r_a] q_r along the a-line), and sigma (q_j - q_jm) adds
            // sigma on the diagonal
            if (ndiff == 0) {
              const int f = face_slot(df, sf);
              const int fidx = cj[(df + 1) % 3] + p * cj[(df + 2) % 3];
              const double* rj = RJ + ((size_t)e * 6 + f) * 50 * pp + fidx;
              ACC25(Sf, rj[(size_t)kl * pp] - sf * V.Fq(df, j, kl) - 0.5 * sf * VL.fvq(df, j, kl)
                            + (kl % 6 == 0 ? G.sigma : 0.0));
              for (int a = 0; a < 3; ++a) {
                ACC25(Sf * sf * lift_own(G, cj, cj, a, true), V.fvg(df, a, j, kl));
                ACC25(-0.5 * Sf * sf * G.dx * G.D[cj[a]][cj[a]], VL.fvg(df, a, j, kl));
              }
            } else {
              const int a = dc[0];
              ACC25(Sf * sf * lift_own(G, cj, cr, a, false), V.fvg(df, a, j, kl));
              ACC25(-0.5 * Sf * sf * G.dx * G.D[cj[a]][cr[a]], VL.fvg(df, a, j, kl));
            }
          } else if (ndiff == 0) {
            const int f = face_slot(df, sf);
            const int fidx = cj[(df + 1) % 3] + p * cj[(df + 2) % 3];
            const double* rj = RJ + ((size_t)e * 6 + f) * 50 * pp + fidx;
            const int nb = nbr[e * 18 + f];
            int cn[3] = {cj[0], cj[1], cj[2]}; cn[df] = N - cj[df];
            ElemView Vn{NJ + (size_t)nb * NJC * nn, nn};
            const int jm = node_index(cn, p);
            ACC25(Sf, rj[(size_t)kl * pp] - sf * V.Fq(df, j, kl) - 0.5 * sf * V.fvq(df, j, kl)
                          + 0.5 * G.inv_hw * Vn.fvg(df, df, jm, kl));
            for (int a = 0; a < 3; ++a)
              ACC25(Sf * 0.5 * sf * lift_own(G, cj, cj, a, true), V.fvg(df, a, j, kl));
          } else {
            const int a = dc[0];
            ACC25(Sf * 0.5 * sf * lift_own(G, cj, cr, a, false), V.fvg(df, a, j, kl));
          }
        }
      }
    }
  }
}

// Pairs sharing no GL index are structurally zero: they are not in the pair list and keep the
// zeros written when the mesh was set.
template <bool IP>
__global__ void __launch_bounds__(256, 3) k_asm_own(Geo G, const double* __restrict__ NJ,
                                                 const double* __restrict__ NJL,
                                                 const double* __restrict__ RJ,
                                                 const int* __restrict__ nbr, const int* __restrict__ iperm,
                                                 const int* __restrict__ pairs, int npairs,
                                                 double* __restrict__ Aown) {
  const int e = blockIdx.x;
  const int lda = G.lda;
  for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
    const int code = pairs[t];
    const int pj = code >> 16, pr = code & 0xffff;
    double acc[25];
    own_entry<IP>(G, NJ, NJL, RJ, nbr, e, iperm[pj], iperm[pr], acc);
    double* out = Aown + (size_t)e * own_stride(G) + (size_t)(5 * pj) * lda + own_col(G, pr, 0);
    for (int k = 0; k < 5; ++k)
      for (int l = 0; l < 5; ++l) out[(size_t)k * lda + l] = acc[k * 5 + l];
  }
}

// Neighbour couplings: X[e][pair][5x5] = dR_{e, row}/dq_{nbr(e, slot), col}.
// With the interior penalty (NJL non-null) the neighbour enters the face rows through its
// state and its unlifted gradient only, and the edge slots stay zero.
template <bool IP>
SC_HD void cross_entry(const Geo& G, const double* NJ, const double* NJL, const double* RJ, const int* nbr, int e,
                       int j, int slot, int r, double acc[25]) {
  const int nn = G.nn, p = G.p, N = G.N, pp = p * p;
  int cj[3], cr[3];
  node_coords(j, p, cj); node_coords(r, p, cr);
  ElemView V{NJ + (size_t)e * NJC * nn, nn};
  constexpr bool ip = IP;
#pragma unroll
  for (int kl = 0; kl < 25; ++kl) acc[kl] = 0.0;
  const double Wj = wprod(G, cj);
  if (slot < 6) {
    const int df = slot / 2, sf = (slot & 1) ? 1 : -1;
    const int jend = sf > 0 ? N : 0, nend = N - jend;
    const int nb = nbr[e * 18 + slot];
    ElemView Vn{NJ + (size_t)nb * NJC * nn, nn};
    ElemView VnL{ip ? NJL + (size_t)nb * NJC * nn : nullptr, nn};
    // (V) volume rows through e's own lifted gradient at the face node m co-located with r
    if (cr[df] == nend) {
      int cm[3] = {cr[0], cr[1], cr[2]}; cm[df] = jend;
      const int m = node_index(cm, p);
      for (int d = 0; d < 3; ++d) {
        bool online = true;
        for (int a = 0; a < 3; ++a) if (a != d && cj[a] != cm[a]) online = false;
        if (!online) continue;
        ACC25(G.Jf * Wj * G.D[cj[d]][cm[d]] * sf * G.inv_hw, -V.fvg(d, df, m, kl));
      }
    }
    if (cj[df] == jend) {
      int cn[3] = {cj[0], cj[1], cj[2]}; cn[df] = nend;
      const int jm = node_index(cn, p);
      const double Sf = G.Jf * Wj / G.w[cj[df]];
      if (r == jm) {
        const int fidx = cj[(df + 1) % 3] + p * cj[(df + 2) % 3];
        const double* rj = RJ + ((size_t)e * 6 + slot) * 50 * pp + fidx;
        if (ip)                                                                  // (S1)
          ACC25(Sf, rj[(size_t)(25 + kl) * pp] - 0.5 * sf * VnL.fvq(df, jm, kl) - (kl % 6 == 0 ? G.sigma : 0.0));
        else
          ACC25(Sf, rj[(size_t)(25 + kl) * pp] - 0.5 * sf * Vn.fvq(df, jm, kl));
        // (S2) e's lifted gradient at j reaches across the face: in every face term of j,
        // at half weight (BR1 average) or at the full weight of -s F_d(j) (interior penalty)
        const double w2 = ip ? 1.0 : 0.5;
        for (int d2 = 0; d2 < 3; ++d2) {
          if (cj[d2] != 0 && cj[d2] != N) continue;
          const int s2 = (cj[d2] == N) ? 1 : -1;
          const double Sf2 = G.Jf * Wj / G.w[cj[d2]];
          ACC25(Sf2 * w2 * s2 * sf * G.inv_hw, V.fvg(d2, df, j, kl));
        }
      }
      // (S3) the neighbour's gradient at jm (lifted, or unlifted with the interior penalty),
      // along its grid lines through jm
      int nd = 0, dd = -1;
      for (int a = 0; a < 3; ++a) if (cn[a] != cr[a]) { ++nd; dd = a; }
      if (ip) {
        if (nd == 0) {
          for (int a = 0; a < 3; ++a)
            ACC25(-0.5 * sf * Sf * G.dx * G.D[cn[a]][cn[a]], VnL.fvg(df, a, jm, kl));
        } else if (nd == 1) {
          ACC25(-0.5 * sf * Sf * G.dx * G.D[cn[dd]][cr[dd]], VnL.fvg(df, dd, jm, kl));
        }
      } else if (nd == 0) {
        for (int a = 0; a < 3; ++a)
          ACC25(-0.5 * sf * Sf * lift_own(G, cn, cn, a, true), Vn.fvg(df, a, jm, kl));
      } else if (nd == 1) {
        ACC25(-0.5 * sf * Sf * lift_own(G, cn, cr, dd, false), Vn.fvg(df, dd, jm, kl));
      }
    }
  } else if (!ip) {
    const int q = slot - 6, pi = q / 4;
    const int d1 = pi == 2 ? 1 : 0, d2 = pi == 0 ? 1 : 2;
    const int s1 = (q & 2) ? 1 : -1, s2 = (q & 1) ? 1 : -1;
    const int e1 = s1 > 0 ? N : 0, e2 = s2 > 0 ? N : 0;
    if (cj[d1] == e1 && cj[d2] == e2) {
      int cx[3] = {cj[0], cj[1], cj[2]}; cx[d1] = N - e1; cx[d2] = N - e2;
      if (node_index(cx, p) == r) {
        for (int o = 0; o < 2; ++o) {
          const int da = o ? d2 : d1, sa = o ? s2 : s1, db = o ? d1 : d2, sb = o ? s1 : s2;
          const int nb = nbr[e * 18 + face_slot(da, sa)];
          ElemView Vn{NJ + (size_t)nb * NJC * nn, nn};
          int cn[3] = {cj[0], cj[1], cj[2]}; cn[da] = N - cj[da];
          const double Sfa = G.Jf * Wj / G.w[cj[da]];
          ACC25(-0.5 * sa * Sfa * sb * G.inv_hw, Vn.fvg(da, db, node_index(cn, p), kl));
        }
      }
    }
  }
}

template <bool IP>
__global__ void k_asm_cross(Geo G, const double* __restrict__ NJ, const double* __restrict__ NJL,
                            const double* __restrict__ RJ,
                            const int* __restrict__ nbr, const int* __restrict__ prow,
                            const int* __restrict__ pslot, const int* __restrict__ pcol,
                            double* __restrict__ X) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= (size_t)G.K * G.NP) return;
  const int e = (int)(t / G.NP), pr = (int)(t % G.NP);
  double acc[25];
  cross_entry<IP>(G, NJ, NJL, RJ, nbr, e, prow[pr], pslot[pr], pcol[pr], acc);
  // layout X[e][k][pair][l]: the couplings of one row variable are contiguous
  for (int k = 0; k < 5; ++k)
    for (int l = 0; l < 5; ++l) X[(((size_t)e * 5 + k) * G.NP + pr) * 5 + l] = acc[k * 5 + l];
}

inline unsigned blocks_for(size_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

namespace sc {

cudaError_t launch_residual_geo(sc_ctx* c, const Geo& G, const double* Q, const double* Qh, double* out) {
  const size_t nodes = (size_t)G.K * G.nn;
  const bool ip = G.visc_flux == 1;
  count_launch(c, ip ? 4 : 3);
  k_lift<<<blocks_for(nodes, 128), 128, 0, c->stream>>>(G, Q, c->d_nbr, c->grad, 1);
  if (ip) k_lift<<<blocks_for(nodes, 128), 128, 0, c->stream>>>(G, Q, c->d_nbr, c->gloc, 0);
  k_flux<<<blocks_for(nodes, 128), 128, 0, c->stream>>>(G, Q, c->grad, c->F);
  k_resid<<<blocks_for(nodes, 128), 128, 0, c->stream>>>(G, Q, Qh, ip ? c->gloc : c->grad, c->F, c->d_nbr, out);
  return cudaGetLastError();
}

cudaError_t launch_residual(sc_ctx* c) { return launch_residual_geo(c, c->G, c->Q, c->Qh, c->B); }

cudaError_t launch_history(sc_ctx* c, const double* Qs, const double* Qsm1) {
  const size_t n = (size_t)c->G.K * c->G.nn * 5;
  count_launch(c);
  k_history<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->G, Qs, Qsm1, c->Qh, n, c->bdf);
  return cudaGetLastError();
}

cudaError_t launch_assembly(sc_ctx* c) {
  const Geo& G = c->G;
  const size_t nodes = (size_t)G.K * G.nn;
  const bool ip = G.visc_flux == 1;
  count_launch(c, ip ? 4 : 3);
  k_nodejac<<<blocks_for(nodes, 64), 64, 0, c->stream>>>(G, c->Q, c->grad, c->NJ);
  // the unlifted gradients are those of the last residual evaluation of this state
  if (ip) k_nodejac<<<blocks_for(nodes, 64), 64, 0, c->stream>>>(G, c->Q, c->gloc, c->NJL);
  const size_t fn = (size_t)G.K * 6 * G.p * G.p;
  k_roejac<<<blocks_for(fn, 64), 64, 0, c->stream>>>(G, c->Q, c->d_nbr, c->RJ);
  {
    ProfScope ps(c, SCK_ASM_OWN);
    if (ip)
      k_asm_own<true><<<G.K, 256, 0, c->stream>>>(G, c->NJ, c->NJL, c->RJ, c->d_nbr, c->d_iperm, c->d_own_pairs,
                                                  (int)c->own_pairs.size(), c->Aown);
    else
      k_asm_own<false><<<G.K, 256, 0, c->stream>>>(G, c->NJ, nullptr, c->RJ, c->d_nbr, c->d_iperm, c->d_own_pairs,
                                                   (int)c->own_pairs.size(), c->Aown);
  }
  const size_t np = (size_t)G.K * G.NP;
  if (ip)
    k_asm_cross<true><<<blocks_for(np, 128), 128, 0, c->stream>>>(G, c->NJ, c->NJL, c->RJ, c->d_nbr, c->d_prow,
                                                                  c->d_pslot, c->d_pcol, c->X);
  else
    k_asm_cross<false><<<blocks_for(np, 128), 128, 0, c->stream>>>(G, c->NJ, nullptr, c->RJ, c->d_nbr, c->d_prow,
                                                                   c->d_pslot, c->d_pcol, c->X);
  return cudaGetLastError();
}

}  // namespace sc
