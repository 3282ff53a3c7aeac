// C-ABI entry points (include/sc.h) and host orchestration of the condensed solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <set>
#include <tuple>

#include "sc_internal.cuh"

namespace sc {
cudaError_t launch_history(sc_ctx* c, const double* Qs, const double* Qsm1);
}

namespace {

#define SC_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess) return fail(c, SC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

sc_status fail(sc_ctx* c, sc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

// Gauss-Lobatto nodes: interior nodes are the roots of q(x) = P_{N+1}(x) - P_{N-1}(x)
// found by Newton's method; weights 2 / (N (N+1) P_N(x)^2).
void legendre_q(int N, double x, double& q, double& dq, double& LN) {
  double l0 = 1.0, l1 = x, d0 = 0.0, d1 = 1.0;
  double lm1 = 1.0, dm1 = 0.0;  // P_{N-1}, P'_{N-1}
  for (int k = 1; k <= N; ++k) {
    const double l2 = ((2 * k + 1) * x * l1 - k * l0) / (k + 1);
    const double d2 = d0 + (2 * k + 1) * l1;
    if (k == N - 1) { lm1 = l1; dm1 = d1; }
    l0 = l1; l1 = l2; d0 = d1; d1 = d2;
  }
  // now l1 = P_{N+1}, l0 = P_N
  if (N == 1) { lm1 = 1.0; dm1 = 0.0; }
  q = l1 - lm1;
  dq = d1 - dm1;
  LN = l0;
}

void gauss_lobatto(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N + 1, 0.0); w.assign(N + 1, 0.0);
  x[0] = -1.0; x[N] = 1.0;
  const double pi = 3.14159265358979323846;
  // Newton from the left half only (a right-half start can fall onto the root x = 1
  // of q); the right half follows by symmetry.
  for (int j = 1; j <= N / 2; ++j) {
    double xx = -std::cos((j + 0.25) * pi / N - 3.0 / (8.0 * N * pi * (j + 0.25)));
    for (int it = 0; it < 60; ++it) {
      double q, dq, LN; legendre_q(N, xx, q, dq, LN);
      const double dx = q / dq;
      xx -= dx;
      if (std::fabs(dx) < 1e-16 * std::max(1.0, std::fabs(xx))) break;
    }
    x[j] = xx;
    x[N - j] = -xx;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    double q, dq, LN; legendre_q(N, x[j], q, dq, LN);
    w[j] = 2.0 / (N * (N + 1) * LN * LN);
  }
}

// Differentiation matrix from barycentric weights: D_ij = (b_j/b_i)/(x_i - x_j),
// D_ii = -sum_{j != i} D_ij.
void diff_matrix(const std::vector<double>& x, double D[SC_MAXP][SC_MAXP]) {
  const int p = (int)x.size();
  std::vector<double> b(p, 1.0);
  for (int j = 0; j < p; ++j)
    for (int k = 0; k < p; ++k)
      if (k != j) b[j] /= (x[j] - x[k]);
  for (int i = 0; i < p; ++i) {
    double s = 0.0;
    for (int j = 0; j < p; ++j) {
      if (j == i) continue;
      D[i][j] = (b[j] / b[i]) / (x[i] - x[j]);
      s += D[i][j];
    }
    D[i][i] = -s;
  }
}

void free_all(sc_ctx* c) {
  sc::free_direct_factors(c);
  double** dps[] = {&c->Q, &c->Qh, &c->grad, &c->F, &c->B, &c->NJ, &c->RJ, &c->Aown, &c->X, &c->Ainv,
                    &c->Ytmp, &c->See, &c->V, &c->Wv, &c->Zv, &c->Xb, &c->Gb, &c->Rb, &c->Ui, &c->Tb,
                    &c->Hd, &c->partial, &c->Xfull, &c->Rfull, &c->Cross, &c->Apk, &c->Sls, &c->dQn,
                    &c->OV, &c->OZ, &c->gloc, &c->NJL};
  for (auto p : dps) { if (*p) cudaFree(*p); *p = nullptr; }
  float** fps[] = {&c->Aown32, &c->X32, &c->Ainv32, &c->Y32, &c->See32, &c->Zf, &c->Xbf, &c->Uf, &c->Cross32,
                   &c->Apk32, &c->Sls32, &c->Sdiag, &c->Cpl, &c->Feat, &c->Snorm, &c->Ynet, &c->Hbuf,
                   &c->Ck, &c->Wbias, &c->ExIb, &c->ExBi, &c->ExY, &c->ExW, &c->Zrb, &c->SeeB, &c->SeeL, &c->SlsL,
                   &c->Zinv};
  for (auto p : fps) { if (*p) cudaFree(*p); *p = nullptr; }
  if (c->Dfull) cudaFree(c->Dfull);
  c->Dfull = nullptr;
  if (c->Trb) cudaFree(c->Trb);
  c->Trb = nullptr;
  c->blackL_valid = false;
  if (c->gj_scale) cudaFree(c->gj_scale);
  c->gj_scale = nullptr;
  c->packed = false;
  if (c->Sls16) cudaFree(c->Sls16);
  c->Sls16 = nullptr;
  c->ls16_ok = false;
  if (c->Wbf16) cudaFree(c->Wbf16);
  c->Wbf16 = nullptr;
  c->Sdiag_valid = c->weights_set = c->learned_on = false;
  int** ips[] = {&c->d_nbr, &c->d_perm, &c->d_iperm, &c->d_own_pairs, &c->d_prow, &c->d_pslot, &c->d_pcol, &c->d_pptr,
                 &c->d_pinfo, &c->piv, &c->rowperm, &c->d_status, &c->d_pk_lptr, &c->d_pk_list,
                 &c->d_pk_row_off, &c->d_pk_pos, &c->d_pk_nint, &c->d_lface, &c->d_lmirror, &c->d_ex_nbpos, &c->d_ex_face_idx,
                 &c->d_colour, &c->pivL, &c->rowpermL, &c->d_lnfaces, &c->d_lface3, &c->d_lmirror3,
                 &c->d_lrslot3, &c->d_redidx, &c->d_face_tab};
  for (auto p : ips) { if (*p) cudaFree(*p); *p = nullptr; }
}

template <class T>
cudaError_t dalloc(T** p, size_t n) { return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)); }

void build_pattern(sc_ctx* c) {
  const Geo& G = c->G;
  const int p = G.p, N = G.N, nn = G.nn;
  auto idx = [&](int i, int j, int k) { return i + p * (j + p * k); };
  auto crd = [&](int m, int cc[3]) { cc[0] = m % p; cc[1] = (m / p) % p; cc[2] = m / (p * p); };
  std::set<std::tuple<int, int, int>> S;  // (row node, slot, col node)
  for (int d = 0; d < 3; ++d)
    for (int s = -1; s <= 1; s += 2) {
      const int slot = face_slot(d, s), jend = s > 0 ? N : 0, nend = N - jend;
      for (int m = 0; m < nn; ++m) {
        int cm[3]; crd(m, cm);
        if (cm[d] != jend) continue;
        int cr[3] = {cm[0], cm[1], cm[2]}; cr[d] = nend;
        const int r = idx(cr[0], cr[1], cr[2]);
        // e's rows reaching face node m through their grid lines (own lifting)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < p; ++b) {
            int cj[3] = {cm[0], cm[1], cm[2]}; cj[a] = b;
            S.insert({idx(cj[0], cj[1], cj[2]), slot, r});
          }
        // face row m: neighbour nodes on the grid lines through its partner r
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < p; ++b) {
            int cx[3] = {cr[0], cr[1], cr[2]}; cx[a] = b;
            S.insert({m, slot, idx(cx[0], cx[1], cx[2])});
          }
      }
    }
  for (int pi = 0; pi < 3; ++pi) {
    const int d1 = pi == 2 ? 1 : 0, d2 = pi == 0 ? 1 : 2, d3 = 3 - d1 - d2;
    for (int q = 0; q < 4; ++q) {
      const int s1 = (q & 2) ? 1 : -1, s2 = (q & 1) ? 1 : -1;
      const int slot = 6 + 4 * pi + q;
      for (int b = 0; b < p; ++b) {
        int cj[3]; cj[d1] = s1 > 0 ? N : 0; cj[d2] = s2 > 0 ? N : 0; cj[d3] = b;
        int cr[3] = {cj[0], cj[1], cj[2]}; cr[d1] = N - cj[d1]; cr[d2] = N - cj[d2];
        S.insert({idx(cj[0], cj[1], cj[2]), slot, idx(cr[0], cr[1], cr[2])});
      }
    }
  }
  Pattern& P = c->pat;
  P.row.clear(); P.slot.clear(); P.col.clear();
  for (auto& t : S) { P.row.push_back(std::get<0>(t)); P.slot.push_back(std::get<1>(t)); P.col.push_back(std::get<2>(t)); }
  const int np = (int)P.row.size();
  P.ptr.assign(nn + 1, 0);
  for (int i = 0; i < np; ++i) P.ptr[P.row[i] + 1]++;
  for (int i = 0; i < nn; ++i) P.ptr[i + 1] += P.ptr[i];
  P.ids.assign(np, 0);
  std::vector<int> fill(P.ptr.begin(), P.ptr.end() - 1);
  for (int i = 0; i < np; ++i) P.ids[fill[P.row[i]]++] = i;
  c->G.NP = np;
}

sc_status check(sc_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, SC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(c, SC_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
  return SC_OK;
}

double dnorm2(sc_ctx* c, const double* v, size_t n, double* hd_slot) {
  sc::multidot(c, v, 1, n, v, hd_slot);
  double h = 0.0;
  cudaMemcpyAsync(&h, hd_slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return std::sqrt(h);
}

}  // namespace

namespace sc {
void gl_basis(int N, std::vector<double>& x, std::vector<double>& w, double D[SC_MAXP][SC_MAXP]) {
  gauss_lobatto(N, x, w);
  diff_matrix(x, D);
}
}  // namespace sc

extern "C" {

sc_status sc_default_config(sc_config* cfg) {
  if (!cfg) return SC_ERR_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->gamma = 1.4; cfg->Pr = 0.72; cfg->Re = 1600.0; cfg->Ma = 0.1;
  cfg->Ts = 110.4 / 288.15; cfg->sutherland = 1; cfg->roe_delta = 0.05;
  cfg->visc_flux = SC_VISC_BR1; cfg->ip_penalty = 1.0;
  cfg->precision = SC_PREC_FP64; cfg->precond = SC_PC_BLOCK_JACOBI;
  cfg->gmres_restart = 30; cfg->gmres_max_iters = 4000; cfg->max_refine = 10;
  cfg->rel_tol = 1e-8; cfg->inner_tol = 1e-4; cfg->tensor_cores = 1; cfg->learned_min_reduction = 1.5;
  return SC_OK;
}

sc_status sc_create(const sc_config* cfg, void* cuda_stream, sc_ctx** out) {
  if (!cfg || !out) return SC_ERR_ARG;
  if (cfg->gmres_restart < 1 || cfg->gmres_restart > 400 || cfg->gmres_max_iters < 1 || !(cfg->rel_tol > 0) ||
      !(cfg->Re > 0) || !(cfg->Ma > 0) || !(cfg->gamma > 1) || !(cfg->Pr > 0))
    return SC_ERR_ARG;
  if (cfg->precision != SC_PREC_FP64 && cfg->precision != SC_PREC_MIXED) return SC_ERR_ARG;
  if (cfg->precond < SC_PC_BLOCK_JACOBI || cfg->precond > SC_PC_RB_SCHUR) return SC_ERR_ARG;
  if (cfg->interior_fp64 != 0 && cfg->interior_fp64 != 1) return SC_ERR_ARG;
  if (cfg->adv_flux != SC_FLUX_ROE && cfg->adv_flux != SC_FLUX_LF) return SC_ERR_ARG;
  if (cfg->visc_flux != SC_VISC_BR1 && cfg->visc_flux != SC_VISC_SIPG) return SC_ERR_ARG;
  if (!(cfg->ip_penalty > 0.0) || !std::isfinite(cfg->ip_penalty)) return SC_ERR_ARG;
  if (cfg->outer_krylov < 0 || cfg->outer_krylov > cfg->gmres_restart || cfg->inner_iters < 0) return SC_ERR_ARG;
  sc_ctx* c = new sc_ctx();
  c->cfg = *cfg;
  c->stream = (cudaStream_t)cuda_stream;
  for (auto& e : c->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) { delete c; return SC_ERR_CUDA; }
  }
  *out = c;
  return SC_OK;
}

void sc_destroy(sc_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  for (auto& e : c->ev) if (e) cudaEventDestroy(e);
  delete c;
}

const char* sc_last_error(const sc_ctx* c) { return c ? c->err.c_str() : "null context"; }

sc_status sc_set_mesh(sc_ctx* c, int n, double L, int N) {
  if (!c) return SC_ERR_ARG;
  if (n < 1 || n > 32 || N < 2 || N > 6 || !(L > 0)) return fail(c, SC_ERR_ARG, "mesh: need n in [1,32], N in [2,6], L > 0");
  // the FP64 arm factors S_ee in one CTA's shared memory: n_b x 33 doubles, 200 KB at N = 5
  if (N > 5 && c->cfg.precision != SC_PREC_MIXED)
    return fail(c, SC_ERR_ARG, "mesh: the FP64 arm takes N <= 5 (N = 6 runs on the mixed arm)");
  if (c->cfg.explicit_schur && N > 4)
    return fail(c, SC_ERR_ARG, "explicit Schur blocks: N <= 4 (W_e holds (n_b + 30 (N+1)^2)^2 values per element)");
  if (c->cfg.precond == SC_PC_LEARNED && c->cfg.precision != SC_PREC_MIXED)
    return fail(c, SC_ERR_ARG, "the learned correction runs on the mixed arm's FP32 blocks");
  if (c->cfg.precond == SC_PC_RB_SCHUR && c->cfg.precision != SC_PREC_MIXED)
    return fail(c, SC_ERR_ARG, "the Schur-corrected sweep runs on the mixed arm's FP32 blocks");
  if (c->cfg.explicit_schur && (c->cfg.precision != SC_PREC_MIXED || n < 3))
    return fail(c, SC_ERR_ARG, "explicit Schur blocks: mixed arm on meshes with n >= 3 (distinct neighbours)");
  cudaStreamSynchronize(c->stream);
  free_all(c);
  c->has_mesh = c->has_state = c->assembled = c->condensed = false;
  Geo& G = c->G;
  G = Geo{};
  G.n = n; G.N = N; G.p = N + 1; G.nn = G.p * G.p * G.p; G.K = n * n * n;
  G.nin = (N - 1) * (N - 1) * (N - 1); G.nbn = G.nn - G.nin;
  G.ne = 5 * G.nn; G.ni = 5 * G.nin; G.nb = 5 * G.nbn;
  auto up4 = [](int x) { return (x + 3) & ~3; };
  G.cb0 = up4(G.ni); G.lda = up4(G.cb0 + G.nb); G.ldi = up4(G.ni); G.lds = up4(G.nb);
  c->L = L;
  G.h = L / n; G.Jf = 0.25 * G.h * G.h; G.dx = 2.0 / G.h;
  std::vector<double> w;
  gauss_lobatto(N, c->xi, w);
  for (int i = 0; i <= N; ++i) G.w[i] = w[i];
  diff_matrix(c->xi, G.D);
  G.inv_hw = 1.0 / (G.h * w[N]);
  G.gamma = c->cfg.gamma; G.Pr = c->cfg.Pr; G.Re = c->cfg.Re; G.Ma = c->cfg.Ma; G.Ts = c->cfg.Ts;
  G.roe_delta = c->cfg.roe_delta; G.sutherland = c->cfg.sutherland; G.adv_flux = c->cfg.adv_flux;
  G.visc_flux = c->cfg.visc_flux;
  G.sigma = (G.visc_flux == SC_VISC_SIPG) ? c->cfg.ip_penalty * (N + 1.0) * (N + 1.0) / (G.h * G.Re) : 0.0;
  G.dt = 1.0; G.c0 = 1.0;
  // node permutation: interior nodes first, then boundary nodes, each in natural order
  const int p = G.p;
  c->perm.assign(G.nn, 0); c->iperm.assign(G.nn, 0);
  int ii = 0, bb = G.nin;
  for (int m = 0; m < G.nn; ++m) {
    const int i = m % p, j = (m / p) % p, k = m / (p * p);
    const bool inner = i > 0 && i < N && j > 0 && j < N && k > 0 && k < N;
    c->perm[m] = inner ? ii++ : bb++;
  }
  for (int m = 0; m < G.nn; ++m) c->iperm[c->perm[m]] = m;
  // own node pairs (positions pj, pr) whose nodes share at least one GL index, grouped by the
  // number of differing indices (2, 1, 0) so that a warp of the assembly follows one branch
  c->own_pairs.clear();
  for (int nd = 2; nd >= 0; --nd)
    for (int pj = 0; pj < G.nn; ++pj)
      for (int pr = 0; pr < G.nn; ++pr) {
        const int a = c->iperm[pj], b = c->iperm[pr];
        const int diff = (a % p != b % p) + ((a / p) % p != (b / p) % p) + (a / (p * p) != b / (p * p));
        if (diff == nd) c->own_pairs.push_back((pj << 16) | pr);
      }
  // neighbour table
  c->nbr.assign((size_t)G.K * 18, 0);
  auto E = [&](int x, int y, int z) { x = (x % n + n) % n; y = (y % n + n) % n; z = (z % n + n) % n; return x + n * (y + n * z); };
  for (int e = 0; e < G.K; ++e) {
    const int ex = e % n, ey = (e / n) % n, ez = e / (n * n);
    const int ce[3] = {ex, ey, ez};
    for (int d = 0; d < 3; ++d)
      for (int s = -1; s <= 1; s += 2) {
        int cc[3] = {ce[0], ce[1], ce[2]}; cc[d] += s;
        c->nbr[(size_t)e * 18 + face_slot(d, s)] = E(cc[0], cc[1], cc[2]);
      }
    for (int pi = 0; pi < 3; ++pi) {
      const int d1 = pi == 2 ? 1 : 0, d2 = pi == 0 ? 1 : 2;
      for (int q = 0; q < 4; ++q) {
        int cc[3] = {ce[0], ce[1], ce[2]};
        cc[d1] += (q & 2) ? 1 : -1; cc[d2] += (q & 1) ? 1 : -1;
        c->nbr[(size_t)e * 18 + 6 + 4 * pi + q] = E(cc[0], cc[1], cc[2]);
      }
    }
  }
  build_pattern(c);
  sc::build_packed_pattern(c);
  sc::build_learned_tables(c);
  sc::build_colours(c);
  sc::build_face_tables(c);
  if (c->cfg.explicit_schur) sc::build_explicit_tables(c);
  const size_t nodes = (size_t)G.K * G.nn, dofs = nodes * 5;
  const size_t n1 = (size_t)G.K * G.nb;
  const int m = c->cfg.gmres_restart;
  c->restart_alloc = m;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(dalloc(&c->Q, dofs)); A(dalloc(&c->Qh, dofs)); A(dalloc(&c->B, dofs));
  A(dalloc(&c->Xfull, dofs)); A(dalloc(&c->Rfull, dofs)); A(dalloc(&c->dQn, dofs));
  A(dalloc(&c->grad, nodes * 15)); A(dalloc(&c->F, nodes * 15));
  A(dalloc(&c->NJ, nodes * 375)); A(dalloc(&c->RJ, (size_t)G.K * 6 * 50 * G.p * G.p));
  if (G.visc_flux == SC_VISC_SIPG) { A(dalloc(&c->gloc, nodes * 15)); A(dalloc(&c->NJL, nodes * 375)); }
  A(dalloc(&c->Aown, (size_t)G.K * own_stride(G))); A(dalloc(&c->X, (size_t)G.K * G.NP * 25));
  if (c->cfg.precision == SC_PREC_MIXED) {
    A(dalloc(&c->Aown32, (size_t)G.K * own_stride(G))); A(dalloc(&c->X32, (size_t)G.K * G.NP * 25));
    A(dalloc(&c->Ainv32, (size_t)G.K * G.ni * G.ldi)); A(dalloc(&c->Y32, (size_t)G.K * G.nb * G.ldi));  // Y^T (nb x ldi) on the tensor-core path
    if (c->cfg.interior_fp64 && G.ni > sc::kGjRegRows) A(dalloc(&c->Ainv, (size_t)G.K * G.ni * G.ldi));  // FP64 A_ii^-1
    A(dalloc(&c->See32, (size_t)G.K * G.nb * G.lds)); A(dalloc(&c->Dfull, dofs));
    A(dalloc(&c->Zf, n1)); A(dalloc(&c->Xbf, n1)); A(dalloc(&c->Uf, (size_t)G.K * G.ni));
    A(dalloc(&c->Cross32, n1 + (size_t)G.K * G.ni));
    if (c->cfg.outer_krylov > 0) {
      A(dalloc(&c->OV, dofs * (size_t)(c->cfg.outer_krylov + 1))); A(dalloc(&c->OZ, dofs * (size_t)c->cfg.outer_krylov));
    }
  } else {
    A(dalloc(&c->Ainv, (size_t)G.K * G.ni * G.ldi)); A(dalloc(&c->Ytmp, (size_t)G.K * G.ni * G.nb));
    A(dalloc(&c->See, (size_t)G.K * G.nb * G.lds));
  }
  A(dalloc(&c->piv, (size_t)G.K * G.nb)); A(dalloc(&c->rowperm, (size_t)G.K * G.nb));
  A(dalloc(&c->Cross, n1 + (size_t)G.K * G.ni));
  A(dalloc(&c->V, n1 * (m + 1))); A(dalloc(&c->Wv, n1)); A(dalloc(&c->Zv, n1)); A(dalloc(&c->Xb, n1));
  A(dalloc(&c->Gb, n1)); A(dalloc(&c->Rb, n1)); A(dalloc(&c->Tb, n1));
  A(dalloc(&c->Ui, (size_t)G.K * G.ni)); A(dalloc(&c->Hd, 3 * (size_t)(m + 2) + 16));
  A(dalloc(&c->partial, 152 * (size_t)(m + 2)));
  A(dalloc(&c->d_status, 3));  // [0] first bad element / error code, [1] FP16 range overflow,
                                // [2] first singular corrected black block
  A(dalloc(&c->d_nbr, c->nbr.size())); A(dalloc(&c->d_perm, G.nn)); A(dalloc(&c->d_iperm, G.nn));
  A(dalloc(&c->d_own_pairs, c->own_pairs.size()));
  A(dalloc(&c->gj_scale, (size_t)G.K * G.ni));
  const int np = G.NP;
  A(dalloc(&c->d_prow, np)); A(dalloc(&c->d_pslot, np)); A(dalloc(&c->d_pcol, np));
  A(dalloc(&c->d_pptr, G.nn + 1)); A(dalloc(&c->d_pinfo, np));
  A(dalloc(&c->d_pk_lptr, c->pk_lptr.size())); A(dalloc(&c->d_pk_list, c->pk_list.size()));
  A(dalloc(&c->d_pk_row_off, c->pk_row_off.size())); A(dalloc(&c->d_pk_pos, c->pk_pos.size()));
  A(dalloc(&c->d_pk_nint, c->pk_nint.size()));
  A(dalloc(&c->d_lface, G.nbn)); A(dalloc(&c->d_lmirror, G.nbn)); A(dalloc(&c->d_lnfaces, G.nbn));
  A(dalloc(&c->d_lface3, 3 * (size_t)G.nbn)); A(dalloc(&c->d_lmirror3, 3 * (size_t)G.nbn));
  A(dalloc(&c->d_lrslot3, 3 * (size_t)G.nbn));
  if (c->cfg.precision == SC_PREC_MIXED) {
    const size_t nsmp = (size_t)G.K * G.nbn;
    A(dalloc(&c->Sdiag, nsmp * 25)); A(dalloc(&c->Cpl, nsmp * 75));  // 3 face slots per node
    if (c->cfg.precond == SC_PC_LEARNED) {
      A(dalloc(&c->Feat, nsmp * sc::kMlpInputs)); A(dalloc(&c->Snorm, nsmp)); A(dalloc(&c->Ynet, nsmp * 25));
      A(dalloc(&c->Hbuf, nsmp * 512)); A(dalloc(&c->Ck, nsmp * 25)); A(dalloc(&c->Wbias, (size_t)sc::kMlpBiases));
      A(dalloc(&c->Wbf16, (size_t)sc::kMlpWeights));
    }
    A(dalloc(&c->Apk32, (size_t)G.K * c->pk_stride)); A(dalloc(&c->Sls32, sc::solve_layout_elems(G)));
    if (c->cfg.factor_fp16) A(dalloc(&c->Sls16, sc::solve_layout_elems(G)));
    if (c->cfg.explicit_schur) {
      A(dalloc(&c->d_ex_nbpos, c->ex_nbpos.size())); A(dalloc(&c->d_ex_face_idx, c->ex_face_idx.size()));
      A(dalloc(&c->ExIb, (size_t)G.K * G.ni * c->ex_ldm)); A(dalloc(&c->ExBi, (size_t)G.K * c->ex_m * G.ldi));
      A(dalloc(&c->ExY, (size_t)G.K * G.ni * c->ex_ldm)); A(dalloc(&c->ExW, sc::explicit_elems_W(G, c)));
    }
  } else {
    A(dalloc(&c->Apk, (size_t)G.K * c->pk_stride)); A(dalloc(&c->Sls, sc::solve_layout_elems(G)));
  }
  const bool sweep = c->cfg.precond == SC_PC_RED_BLACK || c->cfg.precond == SC_PC_LEARNED ||
                     c->cfg.precond == SC_PC_RB_SCHUR;
  if (sweep) {
    A(dalloc(&c->d_colour, (size_t)G.K)); A(dalloc(&c->Trb, n1));
    if (c->cfg.precision == SC_PREC_MIXED) A(dalloc(&c->Zrb, n1));
  }
  if (c->cfg.precond == SC_PC_RB_SCHUR) {
    A(dalloc(&c->Zinv, (size_t)c->n_red * G.nb * G.nb));
    A(dalloc(&c->d_redidx, (size_t)G.K)); A(dalloc(&c->d_face_tab, c->face_tab.size()));
  }
  if (c->cfg.precond == SC_PC_LEARNED || c->cfg.precond == SC_PC_RB_SCHUR) {
    const size_t nbk = (size_t)c->n_black;
    // SeeL also stages the red blocks for their factorisation (SC_PC_RB_SCHUR; n_red = n_black + 1 for odd K)
    A(dalloc(&c->SeeB, nbk * G.nb * G.lds));
    A(dalloc(&c->SeeL, (size_t)std::max(c->n_red, c->n_black) * G.nb * G.lds));
    A(dalloc(&c->SlsL, nbk * (size_t)sc::solve_layout_stride(G)));
    A(dalloc(&c->pivL, nbk * G.nb)); A(dalloc(&c->rowpermL, nbk * G.nb));
  }
  if (e != cudaSuccess) { free_all(c); cudaGetLastError(); return fail(c, SC_ERR_OOM, std::string("allocation: ") + cudaGetErrorString(e)); }
  SC_CUDA(cudaMemcpy(c->d_nbr, c->nbr.data(), c->nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_perm, c->perm.data(), G.nn * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_iperm, c->iperm.data(), G.nn * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_own_pairs, c->own_pairs.data(), c->own_pairs.size() * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_prow, c->pat.row.data(), np * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_pslot, c->pat.slot.data(), np * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_pcol, c->pat.col.data(), np * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_pptr, c->pat.ptr.data(), (G.nn + 1) * sizeof(int), cudaMemcpyHostToDevice));
  // pairs are stored row by row, so the row lists are contiguous ranges of pair ids
  for (int i = 0; i < np; ++i)
    if (c->pat.ids[i] != i) return fail(c, SC_ERR_ARG, "internal: coupling pattern not row ordered");
  std::vector<int> pinfo(np);
  for (int i = 0; i < np; ++i) {
    const int pos = c->perm[c->pat.col[i]];
    const int interior = pos < G.nin ? 1 : 0;
    const int off = interior ? 5 * pos : 5 * (pos - G.nin);
    pinfo[i] = (c->pat.slot[i] << 26) | (interior << 25) | off;
  }
  SC_CUDA(cudaMemcpy(c->d_pinfo, pinfo.data(), np * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(sc::upload_packed_pattern(c));
  if (c->cfg.explicit_schur) SC_CUDA(sc::upload_explicit_tables(c));
  SC_CUDA(cudaMemcpy(c->d_lface, c->l_face.data(), G.nbn * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_lmirror, c->l_mirror.data(), G.nbn * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_lnfaces, c->l_nfaces.data(), G.nbn * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_lface3, c->l_face3.data(), 3 * G.nbn * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_lmirror3, c->l_mirror3.data(), 3 * G.nbn * sizeof(int), cudaMemcpyHostToDevice));
  SC_CUDA(cudaMemcpy(c->d_lrslot3, c->l_rslot3.data(), 3 * G.nbn * sizeof(int), cudaMemcpyHostToDevice));
  if (c->d_colour)
    SC_CUDA(cudaMemcpy(c->d_colour, c->colour_list.data(), (size_t)G.K * sizeof(int), cudaMemcpyHostToDevice));
  if (c->d_redidx) {
    SC_CUDA(cudaMemcpy(c->d_redidx, c->red_index.data(), (size_t)G.K * sizeof(int), cudaMemcpyHostToDevice));
    SC_CUDA(cudaMemcpy(c->d_face_tab, c->face_tab.data(), c->face_tab.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  // the alignment padding of the element blocks (dense and packed) must read as zero
  if (c->Apk) SC_CUDA(cudaMemset(c->Apk, 0, (size_t)G.K * c->pk_stride * sizeof(double)));
  if (c->Apk32) SC_CUDA(cudaMemset(c->Apk32, 0, (size_t)G.K * c->pk_stride * sizeof(float)));
  SC_CUDA(cudaMemset(c->Aown, 0, (size_t)G.K * own_stride(G) * sizeof(double)));
  if (c->Ainv) SC_CUDA(cudaMemset(c->Ainv, 0, (size_t)G.K * G.ni * G.ldi * sizeof(double)));
  if (c->Ainv32) SC_CUDA(cudaMemset(c->Ainv32, 0, (size_t)G.K * G.ni * G.ldi * sizeof(float)));
  c->has_mesh = true;
  return SC_OK;
}

sc_status sc_sizes(const sc_ctx* c, int* K, int* ne, int* ni, int* nb) {
  if (!c || !c->has_mesh) return SC_ERR_STATE;
  if (K) *K = c->G.K;
  if (ne) *ne = c->G.ne;
  if (ni) *ni = c->G.ni;
  if (nb) *nb = c->G.nb;
  return SC_OK;
}

sc_status sc_node_coords(sc_ctx* c, double* xyz) {
  if (!c || !xyz) return SC_ERR_ARG;
  if (!c->has_mesh) return fail(c, SC_ERR_STATE, "node_coords before set_mesh");
  const Geo& G = c->G;
  for (int e = 0; e < G.K; ++e) {
    const int ce[3] = {e % G.n, (e / G.n) % G.n, e / (G.n * G.n)};
    for (int m = 0; m < G.nn; ++m) {
      const int cm[3] = {m % G.p, (m / G.p) % G.p, m / (G.p * G.p)};
      for (int a = 0; a < 3; ++a)
        xyz[((size_t)e * G.nn + m) * 3 + a] = G.h * ce[a] + 0.5 * G.h * (1.0 + c->xi[cm[a]]);
    }
  }
  return SC_OK;
}

sc_status sc_set_timestep(sc_ctx* c, double dt, int bdf) {
  if (!c) return SC_ERR_ARG;
  if (!(dt > 0) || (bdf != 1 && bdf != 2)) return fail(c, SC_ERR_ARG, "timestep: dt > 0, bdf in {1,2}");
  c->G.dt = dt; c->bdf = bdf; c->G.c0 = bdf == 2 ? 1.5 : 1.0;
  c->has_dt = true; c->assembled = c->condensed = false;
  return SC_OK;
}

sc_status sc_set_state(sc_ctx* c, const double* Q, const double* Qs, const double* Qsm1, int on_device) {
  if (!c || !Q || !Qs) return fail(c, SC_ERR_ARG, "set_state: Q and Qs required");
  if (!c->has_mesh) return fail(c, SC_ERR_STATE, "set_state before set_mesh");
  if (c->bdf == 2 && !Qsm1) return fail(c, SC_ERR_ARG, "set_state: BDF2 needs Qsm1");
  const size_t n = (size_t)c->G.K * c->G.nn * 5, bytes = n * sizeof(double);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  SC_CUDA(cudaMemcpyAsync(c->Q, Q, bytes, kind, c->stream));
  // the history combination is formed in Rfull/Xfull as scratch
  SC_CUDA(cudaMemcpyAsync(c->Rfull, Qs, bytes, kind, c->stream));
  if (Qsm1) SC_CUDA(cudaMemcpyAsync(c->Xfull, Qsm1, bytes, kind, c->stream));
  SC_CUDA(sc::launch_history(c, c->Rfull, Qsm1 ? c->Xfull : c->Rfull));
  sc_status s = check(c);
  if (s != SC_OK) return s;
  c->has_state = true; c->assembled = c->condensed = false;
  return SC_OK;
}

sc_status sc_assemble(sc_ctx* c) {
  if (!c) return SC_ERR_ARG;
  if (!c->has_mesh || !c->has_state || !c->has_dt) return fail(c, SC_ERR_STATE, "assemble needs mesh, state and timestep");
  SC_CUDA(sc::launch_residual(c));
  SC_CUDA(sc::launch_assembly(c));
  sc_status s = check(c);
  if (s != SC_OK) return s;
  c->assembled = true; c->condensed = false; c->packed = false;
  return SC_OK;
}

sc_status sc_condense(sc_ctx* c) {
  if (!c) return SC_ERR_ARG;
  if (!c->assembled) return fail(c, SC_ERR_STATE, "condense before assemble");
  const int minus1 = -1;
  SC_CUDA(cudaMemcpyAsync(c->d_status, &minus1, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  if (c->cfg.precond == SC_PC_LEARNED && !c->weights_set)
    return fail(c, SC_ERR_STATE, "learned preconditioner without weights (sc_set_learned_weights)");
  c->Sdiag_valid = false;
  const int zero = 0;
  SC_CUDA(cudaMemcpyAsync(c->d_status + 1, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  SC_CUDA(sc::launch_condense(c));
  SC_CUDA(cudaMemsetAsync(c->d_status + 2, 0xff, sizeof(int), c->stream));  // -1: no singular black block
  if (c->cfg.precond == SC_PC_LEARNED) {  // network -> C_k -> factors of the corrected black blocks
    SC_CUDA(sc::learned_correction(c));
    SC_CUDA(sc::learned_black_factor(c, c->Ck, 1.0f));
  }
  if (c->cfg.precond == SC_PC_RB_SCHUR) SC_CUDA(sc::schur_black_factor(c));
  if (c->cfg.explicit_schur) SC_CUDA(sc::explicit_build(c));
  int bad = -1, ovf = 0, bad_black = -1;
  SC_CUDA(cudaMemcpyAsync(&bad, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SC_CUDA(cudaMemcpyAsync(&ovf, c->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SC_CUDA(cudaMemcpyAsync(&bad_black, c->d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  sc_status s = check(c);
  if (s != SC_OK) return s;
  if (bad == SC_TC_TIMEOUT) return fail(c, SC_ERR_CUDA, "tensor-core wait timed out in the condensation");
  if (bad == SC_EXPLICIT_PATTERN)
    return fail(c, SC_ERR_STATE, "an interior row couples outside the extended boundary set");
  if (bad == SC_PACK_VIOLATION)
    return fail(c, SC_ERR_STATE, "own-block entry outside the packed node pattern is nonzero");
  if (bad >= 0) {  // with compact red factors the index is the red list's
    const int el = c->red_compact && bad < (int)c->colour_list.size() ? c->colour_list[bad] : bad;
    return fail(c, SC_ERR_SINGULAR_BLOCK, "singular element block in element " + std::to_string(el));
  }
  if (bad_black >= 0) {  // a corrected black block is singular: the plain sweep
    c->blackL_valid = false;
    if (c->red_compact) {  // its black factors too come from SlsL (the red ones are compact)
      SC_CUDA(cudaMemsetAsync(c->d_status + 2, 0xff, sizeof(int), c->stream));
      SC_CUDA(sc::plain_black_factor(c));
      SC_CUDA(cudaMemcpyAsync(&bad_black, c->d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      s = check(c);
      if (s != SC_OK) return s;
      if (bad_black >= 0) return fail(c, SC_ERR_SINGULAR_BLOCK, "singular black element block");
      c->blackL_valid = true;
    }
  }
  // FP16 factors for the block-Jacobi solve only when every entry fits the FP16 range
  c->ls16_ok = c->Sls16 != nullptr && ovf == 0 && c->cfg.precond != SC_PC_NONE && !c->red_compact;
  c->condensed = true;
  return SC_OK;
}

sc_status sc_get_state(sc_ctx* c, double* Qout, int on_device) {
  if (!c || !Qout) return SC_ERR_ARG;
  if (!c->has_state) return fail(c, SC_ERR_STATE, "get_state before set_state");
  const size_t bytes = (size_t)c->G.K * c->G.ne * sizeof(double);
  SC_CUDA(cudaMemcpyAsync(Qout, c->Q, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return check(c);
}

sc_status sc_condensed_rhs(sc_ctx* c, double* g, int on_device) {
  if (!c || !g) return SC_ERR_ARG;
  if (!c->condensed) return fail(c, SC_ERR_STATE, "condensed_rhs before condense");
  const size_t n1 = (size_t)c->G.K * c->G.nb;
  double* out = on_device ? g : c->Gb;
  if (c->cfg.precision == SC_PREC_MIXED) {
    SC_CUDA(sc::cond_interior32(c, nullptr, 0.0, c->B, 1.0, c->Uf));
    SC_CUDA(sc::cond_boundary32(c, nullptr, 0.0, c->B, 1.0, c->Uf, out));
  } else {
    SC_CUDA(sc::cond_interior(c, nullptr, 0.0, c->B, 1.0, c->Ui));
    SC_CUDA(sc::cond_boundary(c, nullptr, 0.0, c->B, 1.0, c->Ui, out));
  }
  if (!on_device) SC_CUDA(cudaMemcpyAsync(g, c->Gb, n1 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check(c);
}

sc_status sc_backsubstitute(sc_ctx* c, const double* xb, double* dQ, int on_device) {
  if (!c || !xb || !dQ) return SC_ERR_ARG;
  if (!c->condensed) return fail(c, SC_ERR_STATE, "backsubstitute before condense");
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb, dofs = (size_t)G.K * G.ne;
  const double* xd = xb;
  if (!on_device) {
    SC_CUDA(cudaMemcpyAsync(c->Xb, xb, n1 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    xd = c->Xb;
  }
  double* out = on_device ? dQ : c->Xfull;
  if (c->cfg.precision == SC_PREC_MIXED) {
    SC_CUDA(sc::vec_to_float(c, c->Xbf, xd, n1));
    SC_CUDA(sc::cond_interior32(c, c->Xbf, -1.0, c->B, 1.0, c->Uf));
    SC_CUDA(sc::scatter_solution32(c, xd, c->Uf, out));
  } else {
    SC_CUDA(sc::cond_interior(c, xd, -1.0, c->B, 1.0, c->Ui));
    SC_CUDA(sc::scatter_solution(c, xd, c->Ui, out));
  }
  if (!on_device) SC_CUDA(cudaMemcpyAsync(dQ, c->Xfull, dofs * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check(c);
}

sc_status sc_newton_step(sc_ctx* c, int max_newton, double newton_tol, sc_solve_stats* last, int* newton_iters,
                         double* newton_rel) {
  if (!c || max_newton < 1 || !(newton_tol > 0)) return SC_ERR_ARG;
  if (!c->has_mesh || !c->has_state || !c->has_dt) return fail(c, SC_ERR_STATE, "newton_step needs mesh, state, timestep");
  const size_t dofs = (size_t)c->G.K * c->G.ne;
  double* hs = c->Hd + 2 * (c->restart_alloc + 1) + 2;
  double r0 = -1.0, rn = 0.0;
  int it = 0;
  sc_solve_stats st{};
  for (;;) {
    sc_status s = sc_assemble(c);
    if (s != SC_OK) return s;
    rn = dnorm2(c, c->B, dofs, hs);
    if (r0 < 0.0) r0 = rn;
    if (!std::isfinite(rn)) return fail(c, SC_ERR_NONFINITE, "non-finite Newton residual");
    if (rn <= newton_tol * r0 || it >= max_newton) break;
    s = sc_condense(c);
    if (s == SC_OK) s = sc_solve(c, c->dQn, 1, &st);
    if (s != SC_OK) return s;
    // Q <- Q + dQ (the Newton update of eq. NeqtonEq)
    SC_CUDA(sc::vec_axpby(c, c->Q, 1.0, c->dQn, 1.0, dofs));
    ++it;
  }
  if (last) *last = st;
  if (newton_iters) *newton_iters = it;
  if (newton_rel) *newton_rel = r0 > 0.0 ? rn / r0 : 0.0;
  if (rn > newton_tol * r0) return fail(c, SC_ERR_NOT_CONVERGED, "Newton did not reach the tolerance");
  return SC_OK;
}

sc_status sc_get_rhs(sc_ctx* c, double* Bout, int on_device) {
  if (!c || !Bout) return SC_ERR_ARG;
  if (!c->assembled) return fail(c, SC_ERR_STATE, "get_rhs before assemble");
  const size_t bytes = (size_t)c->G.K * c->G.ne * sizeof(double);
  SC_CUDA(cudaMemcpyAsync(Bout, c->B, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  return check(c);
}

sc_status sc_apply_jacobian(sc_ctx* c, const double* x, double* y, int on_device) {
  if (!c || !x || !y) return SC_ERR_ARG;
  if (!c->assembled) return fail(c, SC_ERR_STATE, "apply_jacobian before assemble");
  const size_t bytes = (size_t)c->G.K * c->G.ne * sizeof(double);
  const double* xd = x;
  if (!on_device) { SC_CUDA(cudaMemcpyAsync(c->Xfull, x, bytes, cudaMemcpyHostToDevice, c->stream)); xd = c->Xfull; }
  double* yd = on_device ? y : c->Rfull;
  SC_CUDA(sc::global_apply(c, xd, yd));
  if (!on_device) SC_CUDA(cudaMemcpyAsync(y, yd, bytes, cudaMemcpyDeviceToHost, c->stream));
  return check(c);
}

sc_status sc_get_jacobian_block(sc_ctx* c, int e, int col, double* block) {
  if (!c || !block) return SC_ERR_ARG;
  if (!c->assembled) return fail(c, SC_ERR_STATE, "get_jacobian_block before assemble");
  const Geo& G = c->G;
  if (e < 0 || e >= G.K || col < 0 || col >= G.K) return fail(c, SC_ERR_ARG, "element index out of range");
  const int ne = G.ne;
  std::vector<double> own(own_stride(G)), X((size_t)G.NP * 25);
  SC_CUDA(cudaMemcpyAsync(own.data(), c->Aown + (size_t)e * own_stride(G), own.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SC_CUDA(cudaMemcpyAsync(X.data(), c->X + (size_t)e * G.NP * 25, X.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  sc_status s = check(c);
  if (s != SC_OK) return s;
  std::fill(block, block + (size_t)ne * ne, 0.0);
  if (col == e)
    for (int j = 0; j < G.nn; ++j)
      for (int r = 0; r < G.nn; ++r)
        for (int k = 0; k < 5; ++k)
          for (int l = 0; l < 5; ++l)
            block[(size_t)(5 * j + k) * ne + 5 * r + l] = own[(size_t)(5 * c->perm[j] + k) * G.lda + own_col(G, c->perm[r], l)];
  bool any = col == e;
  for (int pr = 0; pr < G.NP; ++pr) {
    if (c->nbr[(size_t)e * 18 + c->pat.slot[pr]] != col) continue;
    any = true;
    const int j = c->pat.row[pr], r = c->pat.col[pr];
    for (int k = 0; k < 5; ++k)
      for (int l = 0; l < 5; ++l) block[(size_t)(5 * j + k) * ne + 5 * r + l] += X[((size_t)k * G.NP + pr) * 5 + l];
  }
  if (!any) return fail(c, SC_ERR_ARG, "element c is not in the stencil of e");
  return SC_OK;
}

sc_status sc_condensed_matvec(sc_ctx* c, const double* xb, double* yb) {
  if (!c || !xb || !yb) return SC_ERR_ARG;
  if (!c->condensed) return fail(c, SC_ERR_STATE, "condensed_matvec before condense");
  if (c->cfg.precision == SC_PREC_MIXED) {
    const size_t n1 = (size_t)c->G.K * c->G.nb;
    SC_CUDA(sc::vec_to_float(c, c->Xbf, xb, n1));
    if (c->cfg.explicit_schur) {
      SC_CUDA(sc::explicit_matvec32(c, c->Xbf, yb));
    } else {
      SC_CUDA(sc::cond_interior32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf));
      SC_CUDA(sc::cond_boundary32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf, yb));
    }
  } else {
    SC_CUDA(sc::cond_interior(c, xb, 1.0, nullptr, 0.0, c->Ui));
    SC_CUDA(sc::cond_boundary(c, xb, 1.0, nullptr, 0.0, c->Ui, yb));
  }
  return check(c);
}

sc_status sc_precond_apply(sc_ctx* c, const double* v, double* z) {
  if (!c || !v || !z || v == z) return SC_ERR_ARG;
  if (!c->condensed) return fail(c, SC_ERR_STATE, "precond_apply before condense");
  c->learned_on = c->cfg.precond == SC_PC_LEARNED && c->weights_set && c->blackL_valid;
  if (c->cfg.precision == SC_PREC_MIXED) {
    SC_CUDA(sc::precond_apply32(c, v, z, nullptr));
  } else {
    SC_CUDA(sc::precond_apply(c, v, z));
  }
  c->learned_on = false;
  return check(c);
}

}  // extern "C"

namespace {

// Right-preconditioned restarted GMRES (classical Gram-Schmidt applied twice, Givens
// rotations) on the condensed operator, right-hand side c->Gb, x0 = 0, solution in
// c->Xb.  Stops when the true condensed residual ||g - S x|| <= abs_tol or after
// max_iters iterations.  The operator and preconditioner precision follow c->op32.
sc_status gmres_condensed(sc_ctx* c, double abs_tol, int max_iters, int* iters_out, double* resid_out) {
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb;
  const int m = c->restart_alloc;
  double* const hs = c->Hd + 2 * (m + 1) + 2;  // scratch slot
  double* const h1 = c->Hd;
  double* const h2 = c->Hd + (m + 1);
  double* const hn2 = c->Hd + 2 * (m + 1);
  SC_CUDA(cudaMemsetAsync(c->Xb, 0, n1 * sizeof(double), c->stream));
  SC_CUDA(cudaMemcpyAsync(c->Rb, c->Gb, n1 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  double beta = dnorm2(c, c->Rb, n1, hs);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hbuf(2 * (m + 1) + 1), y(m);
  int iters = 0;
  double resid = beta;
  bool ok = beta <= abs_tol;
  while (!ok && iters < max_iters) {
    const double beta_cycle = beta;
    SC_CUDA(sc::vec_axpby(c, c->V, 1.0 / beta, c->Rb, 0.0, n1));
    std::fill(gv.begin(), gv.end(), 0.0); gv[0] = beta;
    int k = 0;
    for (int j = 0; j < m && iters < max_iters; ++j) {
      double* Vj = c->V + (size_t)j * n1;
      if (c->op32) {
        SC_CUDA(sc::precond_apply32(c, Vj, nullptr, c->Zf));
        if (c->cfg.explicit_schur) {
          SC_CUDA(sc::explicit_matvec32(c, c->Zf, c->Wv));
        } else {
          SC_CUDA(sc::cond_interior32(c, c->Zf, 1.0, nullptr, 0.0, c->Uf));
          SC_CUDA(sc::cond_boundary32(c, c->Zf, 1.0, nullptr, 0.0, c->Uf, c->Wv));
        }
      } else {
        SC_CUDA(sc::precond_apply(c, Vj, c->Zv));
        SC_CUDA(sc::cond_interior(c, c->Zv, 1.0, nullptr, 0.0, c->Ui));
        SC_CUDA(sc::cond_boundary(c, c->Zv, 1.0, nullptr, 0.0, c->Ui, c->Wv));
      }
      SC_CUDA(sc::multidot(c, c->V, j + 1, n1, c->Wv, h1));
      SC_CUDA(sc::vec_update(c, c->Wv, c->V, j + 1, n1, h1, -1.0));
      SC_CUDA(sc::multidot(c, c->V, j + 1, n1, c->Wv, h2));
      SC_CUDA(sc::vec_update(c, c->Wv, c->V, j + 1, n1, h2, -1.0));
      SC_CUDA(sc::multidot(c, c->Wv, 1, n1, c->Wv, hn2));
      SC_CUDA(cudaMemcpyAsync(hbuf.data(), c->Hd, (2 * (m + 1) + 1) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      SC_CUDA(cudaStreamSynchronize(c->stream));
      double* Hc = &H[(size_t)j];  // column j, row stride m
      for (int i = 0; i <= j; ++i) Hc[(size_t)i * m] = hbuf[i] + hbuf[(m + 1) + i];
      const double hn = std::sqrt(std::max(hbuf[2 * (m + 1)], 0.0));
      Hc[(size_t)(j + 1) * m] = hn;
      if (!std::isfinite(hn)) return fail(c, SC_ERR_NONFINITE, "non-finite value in GMRES");
      if (hn > 0) SC_CUDA(sc::vec_axpby(c, c->V + (size_t)(j + 1) * n1, 1.0 / hn, c->Wv, 0.0, n1));
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hc[(size_t)i * m] + sn[i] * Hc[(size_t)(i + 1) * m];
        Hc[(size_t)(i + 1) * m] = -sn[i] * Hc[(size_t)i * m] + cs[i] * Hc[(size_t)(i + 1) * m];
        Hc[(size_t)i * m] = t;
      }
      const double den = std::hypot(Hc[(size_t)j * m], Hc[(size_t)(j + 1) * m]);
      cs[j] = Hc[(size_t)j * m] / den; sn[j] = Hc[(size_t)(j + 1) * m] / den;
      Hc[(size_t)j * m] = den; Hc[(size_t)(j + 1) * m] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++iters; k = j + 1;
      resid = std::fabs(gv[j + 1]);
      if (resid <= abs_tol || hn == 0.0) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double sum = gv[i];
      for (int l = i + 1; l < k; ++l) sum -= H[(size_t)i * m + l] * y[l];
      y[i] = sum / H[(size_t)i * m + i];
    }
    SC_CUDA(cudaMemcpyAsync(c->Hd, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    SC_CUDA(cudaMemsetAsync(c->Tb, 0, n1 * sizeof(double), c->stream));
    SC_CUDA(sc::vec_update(c, c->Tb, c->V, k, n1, c->Hd, 1.0));
    // true condensed residual r = g - S x
    if (c->op32) {
      SC_CUDA(sc::precond_apply32(c, c->Tb, c->Zv, nullptr));
      SC_CUDA(sc::vec_axpby(c, c->Xb, 1.0, c->Zv, 1.0, n1));
      SC_CUDA(sc::vec_to_float(c, c->Xbf, c->Xb, n1));
      if (c->cfg.explicit_schur) {
        SC_CUDA(sc::explicit_matvec32(c, c->Xbf, c->Wv));
      } else {
        SC_CUDA(sc::cond_interior32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf));
        SC_CUDA(sc::cond_boundary32(c, c->Xbf, 1.0, nullptr, 0.0, c->Uf, c->Wv));
      }
    } else {
      SC_CUDA(sc::precond_apply(c, c->Tb, c->Zv));
      SC_CUDA(sc::vec_axpby(c, c->Xb, 1.0, c->Zv, 1.0, n1));
      SC_CUDA(sc::cond_interior(c, c->Xb, 1.0, nullptr, 0.0, c->Ui));
      SC_CUDA(sc::cond_boundary(c, c->Xb, 1.0, nullptr, 0.0, c->Ui, c->Wv));
    }
    SC_CUDA(cudaMemcpyAsync(c->Rb, c->Gb, n1 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    SC_CUDA(sc::vec_axpby(c, c->Rb, -1.0, c->Wv, 1.0, n1));
    beta = dnorm2(c, c->Rb, n1, hs);
    resid = beta;
    if (!std::isfinite(beta)) return fail(c, SC_ERR_NONFINITE, "non-finite condensed residual");
    if (beta <= abs_tol) ok = true;
    // learned correction: a full restart cycle that reduces the residual by less than the
    // configured factor hands the rest of the solve to plain block Jacobi (a cycle cut short
    // by the Givens estimate reaching the tolerance is no measure of the preconditioner)
    if (!ok && c->learned_on && k == m && beta_cycle < c->cfg.learned_min_reduction * beta) {
      c->learned_on = false;
      c->learned_fallbacks++;
    }
  }
  *iters_out = iters;
  *resid_out = resid;
  return SC_OK;
}

// One condensed solve of A d = r (r a full vector): condensed right-hand side
// (eq. SC_step1), GMRES, back-substitution (eq. SC_step2) into d.
sc_status condensed_solve(sc_ctx* c, const double* r, double* d, double rel_tol_g, double abs_floor, int max_iters,
                          int* iters, double* resid, double* gnorm) {
  const Geo& G = c->G;
  const size_t n1 = (size_t)G.K * G.nb;
  if (c->op32) {
    SC_CUDA(sc::cond_interior32(c, nullptr, 0.0, r, 1.0, c->Uf));
    SC_CUDA(sc::cond_boundary32(c, nullptr, 0.0, r, 1.0, c->Uf, c->Gb));
  } else {
    SC_CUDA(sc::cond_interior(c, nullptr, 0.0, r, 1.0, c->Ui));
    SC_CUDA(sc::cond_boundary(c, nullptr, 0.0, r, 1.0, c->Ui, c->Gb));
  }
  *gnorm = dnorm2(c, c->Gb, n1, c->Hd + 2 * (c->restart_alloc + 1) + 2);
  sc_status s = gmres_condensed(c, std::max(rel_tol_g * *gnorm, abs_floor), max_iters, iters, resid);
  if (s != SC_OK) return s;
  if (c->op32) {
    SC_CUDA(sc::vec_to_float(c, c->Xbf, c->Xb, n1));
    SC_CUDA(sc::cond_interior32(c, c->Xbf, -1.0, r, 1.0, c->Uf));
    SC_CUDA(sc::scatter_solution32(c, c->Xb, c->Uf, d));
  } else {
    SC_CUDA(sc::cond_interior(c, c->Xb, -1.0, r, 1.0, c->Ui));
    SC_CUDA(sc::scatter_solution(c, c->Xb, c->Ui, d));
  }
  return SC_OK;
}

// FGMRES(m) on the global FP64 system A x = B with the FP32 condensed solve (condensed
// right-hand side, inner GMRES, back-substitution) as a flexible preconditioner: the
// FP64 products with A keep the outer iteration exact, so it converges even where the
// inner solves are too inexact for refinement sweeps to contract.  x starts at 0.
sc_status fgmres_global(sc_ctx* c, double* x, double target, int* iters_io, int* outer_io, double* rn_io) {
  const Geo& G = c->G;
  const size_t dofs = (size_t)G.K * G.ne;
  const int m = c->cfg.outer_krylov, ma = c->restart_alloc;
  double* const hs = c->Hd + 2 * (ma + 1) + 2;
  double* const h1 = c->Hd;
  double* const h2 = c->Hd + (ma + 1);
  double* const hn2 = c->Hd + 2 * (ma + 1);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hbuf(2 * (ma + 1) + 1), y(m);
  const int cap = c->cfg.inner_iters > 0 ? c->cfg.inner_iters : c->cfg.gmres_max_iters;
  int iters = *iters_io, outer = *outer_io;
  double rn = *rn_io;
  const int max_outer = std::max(1, c->cfg.max_refine) * m;
  while (rn > target && iters < c->cfg.gmres_max_iters && outer < max_outer) {
    SC_CUDA(sc::vec_axpby(c, c->OV, 1.0 / rn, c->Rfull, 0.0, dofs));
    std::fill(gv.begin(), gv.end(), 0.0); gv[0] = rn;
    int k = 0;
    for (int j = 0; j < m && iters < c->cfg.gmres_max_iters && outer < max_outer; ++j) {
      double* Vj = c->OV + (size_t)j * dofs;
      double* Zj = c->OZ + (size_t)j * dofs;
      int it = 0;
      double resid = 0.0, gnorm = 0.0;
      sc_status s = condensed_solve(c, Vj, Zj, c->cfg.inner_tol, 0.0, std::min(cap, c->cfg.gmres_max_iters - iters),
                                    &it, &resid, &gnorm);
      if (s != SC_OK) return s;
      iters += it;
      ++outer;
      SC_CUDA(sc::global_apply(c, Zj, c->Rfull));  // w = A z_j
      SC_CUDA(sc::multidot(c, c->OV, j + 1, dofs, c->Rfull, h1));
      SC_CUDA(sc::vec_update(c, c->Rfull, c->OV, j + 1, dofs, h1, -1.0));
      SC_CUDA(sc::multidot(c, c->OV, j + 1, dofs, c->Rfull, h2));
      SC_CUDA(sc::vec_update(c, c->Rfull, c->OV, j + 1, dofs, h2, -1.0));
      SC_CUDA(sc::multidot(c, c->Rfull, 1, dofs, c->Rfull, hn2));
      SC_CUDA(cudaMemcpyAsync(hbuf.data(), c->Hd, (2 * (ma + 1) + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
      SC_CUDA(cudaStreamSynchronize(c->stream));
      double* Hc = &H[(size_t)j];  // column j, row stride m
      for (int i = 0; i <= j; ++i) Hc[(size_t)i * m] = hbuf[i] + hbuf[(ma + 1) + i];
      const double hn = std::sqrt(std::max(hbuf[2 * (ma + 1)], 0.0));
      Hc[(size_t)(j + 1) * m] = hn;
      if (!std::isfinite(hn)) return fail(c, SC_ERR_NONFINITE, "non-finite value in the outer FGMRES");
      if (hn > 0) SC_CUDA(sc::vec_axpby(c, c->OV + (size_t)(j + 1) * dofs, 1.0 / hn, c->Rfull, 0.0, dofs));
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hc[(size_t)i * m] + sn[i] * Hc[(size_t)(i + 1) * m];
        Hc[(size_t)(i + 1) * m] = -sn[i] * Hc[(size_t)i * m] + cs[i] * Hc[(size_t)(i + 1) * m];
        Hc[(size_t)i * m] = t;
      }
      const double den = std::hypot(Hc[(size_t)j * m], Hc[(size_t)(j + 1) * m]);
      cs[j] = Hc[(size_t)j * m] / den; sn[j] = Hc[(size_t)(j + 1) * m] / den;
      Hc[(size_t)j * m] = den; Hc[(size_t)(j + 1) * m] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      k = j + 1;
      if (std::fabs(gv[j + 1]) <= 0.9 * target || hn == 0.0) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double sum = gv[i];
      for (int l = i + 1; l < k; ++l) sum -= H[(size_t)i * m + l] * y[l];
      y[i] = sum / H[(size_t)i * m + i];
    }
    SC_CUDA(cudaMemcpyAsync(c->Hd, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    SC_CUDA(sc::vec_update(c, x, c->OZ, k, dofs, c->Hd, 1.0));
    // true FP64 residual
    SC_CUDA(sc::global_apply(c, x, c->Rfull));
    SC_CUDA(sc::vec_axpby(c, c->Rfull, 1.0, c->B, -1.0, dofs));
    rn = dnorm2(c, c->Rfull, dofs, hs);
    if (!std::isfinite(rn)) return fail(c, SC_ERR_NONFINITE, "non-finite outer FGMRES residual");
  }
  *iters_io = iters;
  *outer_io = outer;
  *rn_io = rn;
  return SC_OK;
}

}  // namespace

extern "C" {

sc_status sc_solve(sc_ctx* c, double* dQ, int on_device, sc_solve_stats* st) {
  if (!c || !dQ) return SC_ERR_ARG;
  if (!c->condensed) return fail(c, SC_ERR_STATE, "solve before condense");
  const Geo& G = c->G;
  const size_t dofs = (size_t)G.K * G.ne;
  sc_solve_stats S{};
  S.first_bad_element = -1;
  cudaEvent_t* ev = c->ev;
  double* const hs = c->Hd + 2 * (c->restart_alloc + 1) + 2;
  double* xout = on_device ? dQ : c->Xfull;
  c->learned_on = c->cfg.precond == SC_PC_LEARNED && c->weights_set && c->blackL_valid;
  c->learned_fallbacks = 0;
  SC_CUDA(cudaEventRecord(ev[0], c->stream));
  const double bnorm = dnorm2(c, c->B, dofs, hs);
  const double target = c->cfg.rel_tol * bnorm;
  double rn = 0.0;
  int iters = 0;
  double resid = 0.0, gnorm = 0.0;
  if (c->cfg.precision == SC_PREC_FP64) {
    // one condensed FP64 solve to the target
    sc_status s = condensed_solve(c, c->B, xout, 0.0, target, c->cfg.gmres_max_iters, &iters, &resid, &gnorm);
    if (s != SC_OK) return s;
    SC_CUDA(cudaEventRecord(ev[2], c->stream));
    SC_CUDA(sc::global_apply(c, xout, c->Rfull));
    SC_CUDA(sc::vec_axpby(c, c->Rfull, 1.0, c->B, -1.0, dofs));
    rn = dnorm2(c, c->Rfull, dofs, hs);
  } else {
    // FP64 iterative refinement around FP32 condensed solves
    c->op32 = true;
    SC_CUDA(cudaMemsetAsync(xout, 0, dofs * sizeof(double), c->stream));
    SC_CUDA(cudaMemcpyAsync(c->Rfull, c->B, dofs * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    rn = bnorm;
    int sweeps = 0;
    if (c->cfg.outer_krylov > 0) {
      sc_status s = fgmres_global(c, xout, target, &iters, &sweeps, &rn);
      if (s != SC_OK) { c->op32 = false; return s; }
    }
    while (rn > target && sweeps < c->cfg.max_refine && iters < c->cfg.gmres_max_iters &&
           c->cfg.outer_krylov == 0) {
      int it = 0;
      sc_status s = condensed_solve(c, c->Rfull, c->Dfull, c->cfg.inner_tol, 0.5 * target,
                                    c->cfg.gmres_max_iters - iters, &it, &resid, &gnorm);
      if (s != SC_OK) { c->op32 = false; return s; }
      iters += it;
      SC_CUDA(sc::vec_axpby(c, xout, 1.0, c->Dfull, 1.0, dofs));
      SC_CUDA(sc::global_apply(c, xout, c->Rfull));
      SC_CUDA(sc::vec_axpby(c, c->Rfull, 1.0, c->B, -1.0, dofs));
      rn = dnorm2(c, c->Rfull, dofs, hs);
      ++sweeps;
      if (!std::isfinite(rn)) { c->op32 = false; return fail(c, SC_ERR_NONFINITE, "non-finite refinement residual"); }
    }
    c->op32 = false;
    S.refinements = sweeps;
    SC_CUDA(cudaEventRecord(ev[2], c->stream));
  }
  SC_CUDA(cudaEventRecord(ev[3], c->stream));
  if (!on_device) SC_CUDA(cudaMemcpyAsync(dQ, xout, dofs * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  sc_status s = check(c);
  if (s != SC_OK) return s;
  float t02 = 0;
  cudaEventElapsedTime(&t02, ev[0], ev[2]);
  S.ms_gmres = t02;
  S.gmres_iters = iters;
  S.learned_fallbacks = c->learned_fallbacks;
  S.cond_rel_residual = bnorm > 0 ? resid / bnorm : 0.0;
  S.rel_residual = bnorm > 0 ? rn / bnorm : 0.0;
  if (st) *st = S;
  if (!std::isfinite(S.rel_residual)) return fail(c, SC_ERR_NONFINITE, "non-finite solution");
  if (S.rel_residual > c->cfg.rel_tol * 1.0000001 && !(bnorm == 0.0))
    return fail(c, SC_ERR_NOT_CONVERGED, "relative residual " + std::to_string(S.rel_residual) + " above tolerance");
  return SC_OK;
}

sc_status sc_launch_count(const sc_ctx* c, long long* count) {
  if (!c || !count) return SC_ERR_ARG;
  *count = c->launches;
  return SC_OK;
}

sc_status sc_profile_kernel(sc_ctx* c, int kernel_id) {
  if (!c) return SC_ERR_ARG;
  if (kernel_id < -1 || kernel_id >= SCK_COUNT) return fail(c, SC_ERR_ARG, "unknown kernel id");
  cudaStreamSynchronize(c->stream);
  c->prof_kernel = kernel_id;
  c->prof_used = 0; c->prof_ms = 0.0; c->prof_count = 0; c->prof_elems = 0;
  return SC_OK;
}

sc_status sc_profile_elements(const sc_ctx* c, long long* elements) {
  if (!c || !elements) return SC_ERR_ARG;
  *elements = c->prof_elems;
  return SC_OK;
}

sc_status sc_profile_read(sc_ctx* c, long long* launches, double* total_ms) {
  if (!c || !launches || !total_ms) return SC_ERR_ARG;
  SC_CUDA(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->prof_used; ++i) {
    float ms = 0.f;
    SC_CUDA(cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
    c->prof_ms += ms; c->prof_count++;
  }
  c->prof_used = 0;
  *launches = c->prof_count; *total_ms = c->prof_ms;
  return SC_OK;
}

sc_status sc_kernel_work(const sc_ctx* c, int kernel_id, double* flops, double* bytes) {
  if (!c || !flops || !bytes) return SC_ERR_ARG;
  if (!c->has_mesh) return SC_ERR_STATE;
  const Geo& G = c->G;
  // matrices of the condensed solve are stored in FP32 by the mixed arm
  const double w = c->cfg.precision == SC_PREC_MIXED ? 4.0 : 8.0;
  double pairs = (double)c->pat.row.size();
  // neighbour node pairs on interior / boundary rows (the pattern is the same for every element)
  double pairs_i = 0.0;
  for (int r : c->pat.row) pairs_i += c->perm[r] < G.nin ? 1.0 : 0.0;
  const double pairs_b = pairs - pairs_i;
  const double K = G.K, ni = G.ni, nb = G.nb, ne = G.ne, lda = G.lda, ldi = G.ldi, lds = G.lds, cb0 = G.cb0;
  double f = 0.0, b = 0.0;
  switch (kernel_id) {
    case SCK_COND_INTERIOR:  // A_ib,ee x_b and the couplings of interior rows (structural nonzeros), then A_ii^-1 t
      f = K * (2.0 * (double)c->pk_nnz_int + 50.0 * pairs_i + 2.0 * ni * ni);
      b = K * (w * ((double)c->pk_nnz_int + 25.0 * pairs_i + ni * ldi) + w * nb + 8.0 * ni);
      break;
    case SCK_COND_BOUNDARY:  // [A_bi A_bb] [-u; x_b] and the couplings of boundary rows (structural nonzeros)
      f = K * (2.0 * (double)c->pk_nnz_bnd + 50.0 * pairs_b);
      b = K * (w * ((double)c->pk_nnz_bnd + 25.0 * pairs_b) + w * (ni + nb) + 8.0 * nb);
      break;
    case SCK_LU_SOLVE: {  // forward + backward substitution with the S_ee factors (FP16 when stored so)
      const double wf = c->ls16_ok ? 2.0 : w;
      f = K * 2.0 * nb * nb;
      b = K * (wf * nb * lds + 4.0 * nb + 8.0 * 2.0 * nb);
    }
      break;
    case SCK_LU:
      f = K * (2.0 / 3.0) * nb * nb * nb;
      b = K * w * 2.0 * nb * lds;
      break;
    case SCK_GEMM:  // S_ee -= A_bi,ee Y
      f = K * 2.0 * nb * nb * ni;
      b = K * w * (nb * ni + ni * nb + 2.0 * nb * lds);
      break;
    case SCK_GJ_INV:
      f = K * 2.0 * ni * ni * ni;
      b = K * w * (ni * lda + ni * ldi);
      break;
    case SCK_ASM_OWN:  // the 5x5 blocks of the node pairs sharing a GL index
      f = 0.0;
      b = K * 8.0 * 25.0 * (double)c->own_pairs.size();
      break;
    case SCK_EXPLICIT_GEMM:  // Y_e = A_ii^-1 A_ib[., E_e], W_e = A_bi[E_e, .] Y_e
      f = K * (2.0 * ni * ni * c->ex_m + 2.0 * (double)c->ex_m * c->ex_m * ni);
      b = K * 4.0 * (ni * ldi + 2.0 * ni * c->ex_m + c->ex_m * ldi + 2.0 * ni * c->ex_m + (double)c->ex_m * c->ex_m);
      break;
    case SCK_EXPLICIT_APPLY:  // W_e (P_e x), subtracted at the extended dofs
      f = K * 2.0 * (double)c->ex_m * c->ex_m;
      b = K * (4.0 * (double)c->ex_m * c->ex_ldm + 4.0 * c->ex_m + 8.0 * c->ex_m);
      break;
    case SCK_GLOBAL_APPLY:  // always FP64
      f = K * (2.0 * ne * ne + 2.0 * 25.0 * pairs);
      b = K * 8.0 * (ne * lda + 25.0 * pairs + 2.0 * ne);
      break;
    default:
      return SC_ERR_ARG;
  }
  *flops = f; *bytes = b;
  return SC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Spectrum estimate of the global and the condensed matrices (Sec. 4, Fig.
// ConditionNumber): the L2 condition number approximated by the ratio of the largest and
// the smallest eigenvalue moduli, the largest from Arnoldi on the matrix, the smallest
// from Arnoldi on its inverse (shift-and-invert with shift 0), each inverse applied by a
// condensed GMRES solve.
// ---------------------------------------------------------------------------------
namespace {
using cplx = std::complex<double>;

// Eigenvalues of an upper Hessenberg matrix (row-major m x m) by the shifted QR algorithm
// in complex arithmetic: Wilkinson shift from the trailing 2 x 2 block of the active
// window (an exceptional shift every tenth sweep), one Givens rotation per subdiagonal
// entry, deflation when a subdiagonal entry falls below eps times its diagonal
// neighbours.  Returns false if one eigenvalue needs more than 200 sweeps.
bool hessenberg_eigvals(int m, const double* Hin, std::vector<cplx>& ev) {
  std::vector<cplx> H((size_t)m * m);
  double hnorm = 0.0;
  for (size_t i = 0; i < (size_t)m * m; ++i) { H[i] = Hin[i]; hnorm = std::max(hnorm, std::fabs(Hin[i])); }
  ev.assign(m, cplx(0.0));
  const double eps = 2.220446049250313e-16;
  auto at = [&](int i, int j) -> cplx& { return H[(size_t)i * m + j]; };
  int hi = m - 1, iter = 0;
  std::vector<double> cs(m);
  std::vector<cplx> sn(m);
  while (hi >= 0) {
    if (hi == 0) { ev[0] = at(0, 0); break; }
    int l = hi;
    while (l > 0) {
      double s = std::abs(at(l - 1, l - 1)) + std::abs(at(l, l));
      if (s == 0.0) s = hnorm;
      if (std::abs(at(l, l - 1)) <= eps * s) { at(l, l - 1) = 0.0; break; }
      --l;
    }
    if (l == hi) { ev[hi] = at(hi, hi); --hi; iter = 0; continue; }
    if (++iter > 200) return false;
    const cplx a = at(hi - 1, hi - 1), b = at(hi - 1, hi), cc = at(hi, hi - 1), d = at(hi, hi);
    const cplx tr = a + d, det = a * d - b * cc;
    const cplx disc = std::sqrt(tr * tr * 0.25 - det);
    const cplx mu1 = tr * 0.5 + disc, mu2 = tr * 0.5 - disc;
    cplx mu = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
    if (iter % 10 == 0) mu = d + cplx(std::abs(cc), 0.0);
    for (int k = l; k <= hi; ++k) at(k, k) -= mu;
    // H - mu I = Q R by Givens rotations G_k acting on rows k, k+1 ...
    for (int k = l; k < hi; ++k) {
      const cplx x = at(k, k), y = at(k + 1, k);
      const double ax = std::abs(x), r = std::hypot(ax, std::abs(y));
      double c = 1.0;
      cplx sv = 0.0;
      if (r > 0.0) {
        if (ax == 0.0) { c = 0.0; sv = 1.0; }
        else { c = ax / r; sv = (x / ax) * std::conj(y) / r; }
      }
      for (int j = k; j <= hi; ++j) {
        const cplx t1 = at(k, j), t2 = at(k + 1, j);
        at(k, j) = c * t1 + sv * t2;
        at(k + 1, j) = -std::conj(sv) * t1 + c * t2;
      }
      cs[k] = c; sn[k] = sv;
    }
    // ... then R Q + mu I: the adjoint rotations from the right on columns k, k+1
    for (int k = l; k < hi; ++k) {
      const double c = cs[k];
      const cplx sv = sn[k];
      const int iend = std::min(k + 2, hi);
      for (int i = l; i <= iend; ++i) {
        const cplx t1 = at(i, k), t2 = at(i, k + 1);
        at(i, k) = c * t1 + std::conj(sv) * t2;
        at(i, k + 1) = -sv * t1 + c * t2;
      }
    }
    for (int k = l; k <= hi; ++k) at(k, k) += mu;
  }
  return true;
}

// m steps of Arnoldi (classical Gram-Schmidt applied twice) on the operator op over
// vectors of length n, from a fixed pseudo-random start vector; the Ritz values (the
// eigenvalues of the m x m Hessenberg matrix) in ritz.  V holds (m + 1) n doubles, w n.
template <class Op>
sc_status arnoldi_ritz(sc_ctx* c, size_t n, int m, Op op, double* V, double* w, std::vector<cplx>& ritz,
                       int* steps) {
  const int ma = c->restart_alloc;
  double* const h1 = c->Hd;
  double* const h2 = c->Hd + (ma + 1);
  double* const hn2 = c->Hd + 2 * (ma + 1);
  double* const hs = c->Hd + 2 * (ma + 1) + 2;
  {
    std::vector<double> v0(n);
    uint64_t z = 0x2545F4914F6CDD1DULL;
    for (size_t i = 0; i < n; ++i) {  // xorshift64*: a fixed, well-spread start vector
      z ^= z >> 12; z ^= z << 25; z ^= z >> 27;
      v0[i] = (double)((z * 0x2545F4914F6CDD1DULL) >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    SC_CUDA(cudaMemcpyAsync(V, v0.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const double nv = dnorm2(c, V, n, hs);
    SC_CUDA(sc::vec_axpby(c, V, 1.0 / nv, V, 0.0, n));
  }
  std::vector<double> H((size_t)m * m, 0.0), hbuf(2 * (ma + 1) + 1);
  int k = 0;
  for (int j = 0; j < m; ++j) {
    sc_status s = op(V + (size_t)j * n, w);
    if (s != SC_OK) return s;
    SC_CUDA(sc::multidot(c, V, j + 1, n, w, h1));
    SC_CUDA(sc::vec_update(c, w, V, j + 1, n, h1, -1.0));
    SC_CUDA(sc::multidot(c, V, j + 1, n, w, h2));
    SC_CUDA(sc::vec_update(c, w, V, j + 1, n, h2, -1.0));
    SC_CUDA(sc::multidot(c, w, 1, n, w, hn2));
    SC_CUDA(cudaMemcpyAsync(hbuf.data(), c->Hd, (2 * (ma + 1) + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    SC_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hbuf[i] + hbuf[(ma + 1) + i];
    const double hn = std::sqrt(std::max(hbuf[2 * (ma + 1)], 0.0));
    if (!std::isfinite(hn)) return fail(c, SC_ERR_NONFINITE, "non-finite value in the Arnoldi process");
    k = j + 1;
    if (j + 1 < m) H[(size_t)(j + 1) * m + j] = hn;
    if (hn == 0.0) break;  // invariant subspace: its Ritz values are exact
    SC_CUDA(sc::vec_axpby(c, V + (size_t)(j + 1) * n, 1.0 / hn, w, 0.0, n));
  }
  std::vector<double> Hk((size_t)k * k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Hk[(size_t)i * k + j] = H[(size_t)i * m + j];
  if (!hessenberg_eigvals(k, Hk.data(), ritz)) return fail(c, SC_ERR_NOT_CONVERGED, "Hessenberg QR did not converge");
  *steps = k;
  return SC_OK;
}

cplx largest_modulus(const std::vector<cplx>& v) {
  cplx best = 0.0;
  for (const cplx& z : v) if (std::abs(z) > std::abs(best)) best = z;
  return best;
}
}  // namespace

extern "C" {

sc_status sc_hessenberg_eigvals(int m, const double* H, double* re, double* im) {
  if (m < 1 || !H || !re || !im) return SC_ERR_ARG;
  std::vector<cplx> ev;
  if (!hessenberg_eigvals(m, H, ev)) return SC_ERR_NOT_CONVERGED;
  for (int i = 0; i < m; ++i) { re[i] = ev[i].real(); im[i] = ev[i].imag(); }
  return SC_OK;
}

sc_status sc_spectrum_estimate(sc_ctx* c, int which, int m_max, int m_min, double inv_tol, double* out) {
  if (!c || !out || (which != 0 && which != 1)) return SC_ERR_ARG;
  if (m_max < 1 || m_min < 1 || m_max > c->restart_alloc || m_min > c->restart_alloc || !(inv_tol > 0.0))
    return fail(c, SC_ERR_ARG, "spectrum: need 1 <= m_max, m_min <= gmres_restart and inv_tol > 0");
  if (!c->condensed) return fail(c, SC_ERR_STATE, "spectrum estimate before condense");
  if (c->cfg.precision != SC_PREC_FP64)
    return fail(c, SC_ERR_STATE, "spectrum estimate: needs the FP64 arm (its operators and solves are exact to FP64)");
  const Geo& G = c->G;
  const size_t n = which == 0 ? (size_t)G.K * G.ne : (size_t)G.K * G.nb;
  double *V = nullptr, *w = nullptr;
  cudaError_t e = cudaMalloc((void**)&V, (size_t)(std::max(m_max, m_min) + 1) * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&w, n * sizeof(double));
  if (e != cudaSuccess) {
    if (V) cudaFree(V);
    cudaGetLastError();
    return fail(c, SC_ERR_OOM, "spectrum estimate: Arnoldi basis does not fit");
  }
  struct Free { double *a, *b; ~Free() { cudaFree(a); cudaFree(b); } } guard{V, w};
  const size_t n1 = (size_t)G.K * G.nb;
  double* const hs = c->Hd + 2 * (c->restart_alloc + 1) + 2;
  long long inner = 0;
  auto fwd = [&](const double* x, double* y) -> sc_status {
    if (which == 0) {
      SC_CUDA(sc::global_apply(c, x, y));
    } else {
      SC_CUDA(sc::cond_interior(c, x, 1.0, nullptr, 0.0, c->Ui));
      SC_CUDA(sc::cond_boundary(c, x, 1.0, nullptr, 0.0, c->Ui, y));
    }
    return SC_OK;
  };
  auto inv = [&](const double* x, double* y) -> sc_status {
    int it = 0;
    double resid = 0.0, gnorm = 0.0;
    sc_status s;
    if (which == 0) {  // y = A^-1 x by condensation: condensed rhs, GMRES on S, back-substitution
      s = condensed_solve(c, x, y, inv_tol, 0.0, c->cfg.gmres_max_iters, &it, &resid, &gnorm);
    } else {           // y = S^-1 x by GMRES on S
      SC_CUDA(cudaMemcpyAsync(c->Gb, x, n1 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      const double xn = dnorm2(c, c->Gb, n1, hs);
      s = gmres_condensed(c, inv_tol * xn, c->cfg.gmres_max_iters, &it, &resid);
      if (s == SC_OK) SC_CUDA(cudaMemcpyAsync(y, c->Xb, n1 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    inner += it;
    return s;
  };
  std::vector<cplx> ritz;
  int steps = 0;
  sc_status s = arnoldi_ritz(c, n, m_max, fwd, V, w, ritz, &steps);
  if (s != SC_OK) return s;
  const cplx lmax = largest_modulus(ritz);
  s = arnoldi_ritz(c, n, m_min, inv, V, w, ritz, &steps);
  if (s != SC_OK) return s;
  const cplx th = largest_modulus(ritz);
  if (std::abs(th) == 0.0) return fail(c, SC_ERR_NONFINITE, "spectrum estimate: zero Ritz value of the inverse");
  const cplx lmin = 1.0 / th;
  out[0] = lmax.real(); out[1] = lmax.imag();
  out[2] = lmin.real(); out[3] = lmin.imag();
  out[4] = std::abs(lmax) / std::abs(lmin);
  out[5] = (double)inner;
  return check(c);
}

}  // extern "C"
