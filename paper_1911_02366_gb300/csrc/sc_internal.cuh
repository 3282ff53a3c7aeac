// Internal declarations of the GB300 condensed GL-DGSEM library.
//
// Shared by the CUDA translation units of paper_1911_02366_gb300/csrc only.  The
// public ABI is include/sc.h.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sc.h"

#define SC_MAXP 8  // N + 1 <= 8
#define SC_HD __host__ __device__

// Geometry, basis and physics, passed by value to every kernel.
struct Geo {
  int n, N, p, nn, K;     // elements per direction, order, N+1, nodes/element, elements
  int ne, nin, nbn, ni, nb;  // dofs/element, interior nodes, boundary nodes, interior dofs, boundary dofs
  int NP;                 // neighbour-coupling pairs per element
  int lda, cb0;           // own block: row stride, column of the first boundary dof (both % 4 == 0)
  int ldi, lds;           // row strides of A_ii^-1 and of the S_ee factors (% 4 == 0)
  double h, Jf, dx, inv_hw;  // element size, (h/2)^2, 2/h, 1/(h w_N)
  double dt, c0;          // time step, BDF leading coefficient (1 or 3/2)
  double gamma, Pr, Re, Ma, Ts, roe_delta;
  int adv_flux;  // 0 Roe, 1 local Lax-Friedrichs
  int visc_flux;  // 0 BR1 (lifted gradients at the faces), 1 symmetric interior penalty
  double sigma;   // interior-penalty coefficient C_IP (N+1)^2 / (h Re) (0 with BR1)
  int sutherland;
  double D[SC_MAXP][SC_MAXP];  // D[a][b] = l_b'(xi_a)
  double w[SC_MAXP];           // Gauss-Lobatto weights
};

// Slot numbering of an element's neighbours: faces 0..5 = (d, s) -> 2d + (s > 0);
// edges 6..17 = 6 + 4*pairIndex(d1 < d2) + 2*(s1 > 0) + (s2 > 0).
SC_HD inline int face_slot(int d, int s) { return 2 * d + (s > 0); }
SC_HD inline int edge_pair_index(int d1, int d2) {  // d1 < d2
  return d1 == 0 ? (d2 == 1 ? 0 : 1) : 2;
}

// Column of dof (permuted node position pos, variable l) in an own element block:
// interior dofs first, then the boundary dofs starting at the aligned column cb0.
SC_HD inline int own_col(const Geo& G, int pos, int l) {
  return pos < G.nin ? 5 * pos + l : G.cb0 + 5 * (pos - G.nin) + l;
}
SC_HD inline size_t own_stride(const Geo& G) { return (size_t)G.ne * G.lda; }

// Packed description of one neighbour coupling column: neighbour slot (bits 26..30),
// interior flag (bit 25), offset of the column inside that neighbour's boundary (or
// interior) part of a condensed vector (bits 0..24).
SC_HD inline int pinfo_slot(int v) { return (v >> 26) & 31; }
SC_HD inline int pinfo_interior(int v) { return (v >> 25) & 1; }
SC_HD inline int pinfo_offset(int v) { return v & ((1 << 25) - 1); }

// ------------------------------------------------------------------ dual numbers
// Five-direction forward-mode dual used to differentiate the point fluxes.
struct D5 {
  double v, d[5];
  __host__ __device__ D5() : v(0.0) { for (int i = 0; i < 5; ++i) d[i] = 0.0; }
  __host__ __device__ D5(double x) : v(x) { for (int i = 0; i < 5; ++i) d[i] = 0.0; }
};
SC_HD inline D5 operator+(const D5& a, const D5& b) { D5 r; r.v = a.v + b.v;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
SC_HD inline D5 operator-(const D5& a, const D5& b) { D5 r; r.v = a.v - b.v;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
SC_HD inline D5 operator-(const D5& a) { D5 r; r.v = -a.v;
  for (int i = 0; i < 5; ++i) r.d[i] = -a.d[i]; return r; }
SC_HD inline D5 operator*(const D5& a, const D5& b) { D5 r; r.v = a.v * b.v;
  for (int i = 0; i < 5; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]); return r; }
SC_HD inline D5 operator*(const D5& a, double b) { D5 r; r.v = a.v * b;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] * b; return r; }
SC_HD inline D5 operator*(double b, const D5& a) { return a * b; }
SC_HD inline D5 operator+(const D5& a, double b) { D5 r = a; r.v += b; return r; }
SC_HD inline D5 operator+(double b, const D5& a) { D5 r = a; r.v += b; return r; }
SC_HD inline D5 operator-(const D5& a, double b) { D5 r = a; r.v -= b; return r; }
SC_HD inline D5 operator-(double b, const D5& a) { D5 r = -a; r.v += b; return r; }
SC_HD inline D5 recip(const D5& a) { D5 r; r.v = 1.0 / a.v; const double s = -r.v * r.v;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] * s; return r; }
SC_HD inline D5 operator/(const D5& a, const D5& b) { return a * recip(b); }
SC_HD inline D5 operator/(const D5& a, double b) { return a * (1.0 / b); }
SC_HD inline D5 operator/(double a, const D5& b) { return recip(b) * a; }
SC_HD inline D5 dsqrt(const D5& a) { D5 r; r.v = sqrt(a.v); const double s = 0.5 / r.v;
  for (int i = 0; i < 5; ++i) r.d[i] = a.d[i] * s; return r; }
SC_HD inline double dsqrt(double a) { return sqrt(a); }
SC_HD inline double vval(double a) { return a; }
SC_HD inline double vval(const D5& a) { return a.v; }
SC_HD inline double recip(double a) { return 1.0 / a; }

// ------------------------------------------------------------------ point physics
// Inviscid flux of the compressible Euler equations along x_d (App. B).
template <class T>
SC_HD inline void flux_inviscid(const Geo& G, const T q[5], int d, T f[5]) {
  const T ir = recip(q[0]);
  const T ux = q[1] * ir, uy = q[2] * ir, uz = q[3] * ir;
  const T ud = d == 0 ? ux : (d == 1 ? uy : uz);
  const T kin = 0.5 * (q[1] * ux + q[2] * uy + q[3] * uz);
  const T pr = (G.gamma - 1.0) * (q[4] - kin);
  f[0] = q[1 + d];
  f[1] = q[1] * ud;
  f[2] = q[2] * ud;
  f[3] = q[3] * ud;
  f[1 + d] = f[1 + d] + pr;
  f[4] = (q[4] + pr) * ud;
}

// Viscous flux along x_d from the state and the gradients of the conserved
// variables g[a][k] = d q_k / d x_a (App. B).  The heat flux is written through the
// specific internal energy: kappa dT/dx = (mu gamma / Pr) de/dx.
template <class T, class TG>
SC_HD inline void flux_viscous(const Geo& G, const T q[5], const TG g[3][5], int d, T f[5]) {
  const T ir = recip(q[0]);
  const T u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const T Et = q[4] * ir;
  T grad_u[3][3];  // grad_u[a][i] = d u_i / d x_a
  T grad_e[3];
  for (int a = 0; a < 3; ++a) {
    T su = 0.0;
    for (int i = 0; i < 3; ++i) {
      grad_u[a][i] = (g[a][1 + i] - u[i] * g[a][0]) * ir;
      su = su + u[i] * grad_u[a][i];
    }
    grad_e[a] = (g[a][4] - Et * g[a][0]) * ir - su;
  }
  const T eint = Et - 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  T mu;
  if (G.sutherland) {
    const T Tt = (G.gamma * (G.gamma - 1.0) * G.Ma * G.Ma) * eint;
    mu = (1.0 + G.Ts) * Tt * dsqrt(Tt) * recip(Tt + G.Ts);
  } else {
    mu = T(1.0);
  }
  const T divu = grad_u[0][0] + grad_u[1][1] + grad_u[2][2];
  const double iRe = 1.0 / G.Re;
  T tau[3];
  for (int i = 0; i < 3; ++i) tau[i] = mu * (grad_u[d][i] + grad_u[i][d]);
  tau[d] = tau[d] - (2.0 / 3.0) * mu * divu;
  f[0] = T(0.0);
  for (int i = 0; i < 3; ++i) f[1 + i] = iRe * tau[i];
  f[4] = iRe * (u[0] * tau[0] + u[1] * tau[1] + u[2] * tau[2] + (G.gamma / G.Pr) * mu * grad_e[d]);
}

// Viscous fluxes along all three directions at once, f[d][k], with every array
// index a compile-time constant after unrolling (used for the dual-number Jacobians).
template <class T>
SC_HD inline void flux_viscous_all(const Geo& G, const T q[5], const T g[3][5], T f[3][5]) {
  const T ir = recip(q[0]);
  const T u0 = q[1] * ir, u1 = q[2] * ir, u2 = q[3] * ir;
  const T Et = q[4] * ir;
  // velocity gradients du_i/dx_a
  const T a00 = (g[0][1] - u0 * g[0][0]) * ir, a01 = (g[0][2] - u1 * g[0][0]) * ir, a02 = (g[0][3] - u2 * g[0][0]) * ir;
  const T a10 = (g[1][1] - u0 * g[1][0]) * ir, a11 = (g[1][2] - u1 * g[1][0]) * ir, a12 = (g[1][3] - u2 * g[1][0]) * ir;
  const T a20 = (g[2][1] - u0 * g[2][0]) * ir, a21 = (g[2][2] - u1 * g[2][0]) * ir, a22 = (g[2][3] - u2 * g[2][0]) * ir;
  const T e0 = (g[0][4] - Et * g[0][0]) * ir - (u0 * a00 + u1 * a01 + u2 * a02);
  const T e1 = (g[1][4] - Et * g[1][0]) * ir - (u0 * a10 + u1 * a11 + u2 * a12);
  const T e2 = (g[2][4] - Et * g[2][0]) * ir - (u0 * a20 + u1 * a21 + u2 * a22);
  const T eint = Et - 0.5 * (u0 * u0 + u1 * u1 + u2 * u2);
  T mu;
  if (G.sutherland) {
    const T Tt = (G.gamma * (G.gamma - 1.0) * G.Ma * G.Ma) * eint;
    mu = (1.0 + G.Ts) * Tt * dsqrt(Tt) * recip(Tt + G.Ts);
  } else {
    mu = T(1.0);
  }
  const double iRe = 1.0 / G.Re;
  const T mR = iRe * mu;
  const T lam = (2.0 / 3.0) * (a00 + a11 + a22);
  const T t00 = mR * (2.0 * a00 - lam), t11 = mR * (2.0 * a11 - lam), t22 = mR * (2.0 * a22 - lam);
  const T t01 = mR * (a01 + a10), t02 = mR * (a02 + a20), t12 = mR * (a12 + a21);
  const T kq = (iRe * G.gamma / G.Pr) * mu;
  f[0][0] = T(0.0); f[0][1] = t00; f[0][2] = t01; f[0][3] = t02;
  f[0][4] = u0 * t00 + u1 * t01 + u2 * t02 + kq * e0;
  f[1][0] = T(0.0); f[1][1] = t01; f[1][2] = t11; f[1][3] = t12;
  f[1][4] = u0 * t01 + u1 * t11 + u2 * t12 + kq * e1;
  f[2][0] = T(0.0); f[2][1] = t02; f[2][2] = t12; f[2][3] = t22;
  f[2][4] = u0 * t02 + u1 * t12 + u2 * t22 + kq * e2;
}

template <class T>
SC_HD inline T abs_harten(const T& lam, const T& del) {
  const double l = vval(lam);
  if (fabs(l) >= vval(del)) return l < 0.0 ? -lam : lam;
  return (lam * lam + del * del) * recip(2.0 * del);
}

// Roe numerical flux fhat(qa, qb, n) . n, n = s e_d outward from qa's element,
// with Roe-averaged wave decomposition and Harten's entropy fix on every wave.
template <class T>
SC_HD inline void flux_roe(const Geo& G, const T qa[5], const T qb[5], int d, int s, T fh[5]) {
  const double gm1 = G.gamma - 1.0;
  T fa[5], fb[5];
  flux_inviscid(G, qa, d, fa);
  flux_inviscid(G, qb, d, fb);
  const T ira = recip(qa[0]), irb = recip(qb[0]);
  T ua[3], ub[3];
  for (int i = 0; i < 3; ++i) { ua[i] = qa[1 + i] * ira; ub[i] = qb[1 + i] * irb; }
  const T pa = gm1 * (qa[4] - 0.5 * (qa[1] * ua[0] + qa[2] * ua[1] + qa[3] * ua[2]));
  const T pb = gm1 * (qb[4] - 0.5 * (qb[1] * ub[0] + qb[2] * ub[1] + qb[3] * ub[2]));
  const T ra = dsqrt(qa[0]), rb = dsqrt(qb[0]);
  const T iw = recip(ra + rb);
  T um[3];
  for (int i = 0; i < 3; ++i) um[i] = (ra * ua[i] + rb * ub[i]) * iw;
  const T Hm = (ra * (qa[4] + pa) * ira + rb * (qb[4] + pb) * irb) * iw;
  const T vsq = um[0] * um[0] + um[1] * um[1] + um[2] * um[2];
  const T cm = dsqrt(gm1 * (Hm - 0.5 * vsq));
  const T rhom = ra * rb;
  const double sd = (double)s;
  const T un = um[d] * sd;
  const T jr = qb[0] - qa[0];
  const T jp = pb - pa;
  T ju[3];
  for (int i = 0; i < 3; ++i) ju[i] = ub[i] - ua[i];
  const T jun = ju[d] * sd;
  const T ic2 = recip(cm * cm);
  const T wm = 0.5 * (jp - rhom * cm * jun) * ic2;  // strength of the u - c wave
  const T wp = 0.5 * (jp + rhom * cm * jun) * ic2;  // strength of the u + c wave
  const T we = jr - jp * ic2;                        // entropy wave
  const T del = G.roe_delta * cm;
  const T am = abs_harten(un - cm, del) * wm;
  const T ap = abs_harten(un + cm, del) * wp;
  const T a0 = abs_harten(un, del);
  // shear: tangential velocity jump
  T jt[3];
  for (int i = 0; i < 3; ++i) jt[i] = ju[i];
  jt[d] = T(0.0);
  const T umjt = um[0] * jt[0] + um[1] * jt[1] + um[2] * jt[2];
  T diss[5];
  diss[0] = am + ap + a0 * we;
  for (int i = 0; i < 3; ++i) diss[1 + i] = (am + ap) * um[i] + a0 * (we * um[i] + rhom * jt[i]);
  diss[1 + d] = diss[1 + d] + (ap - am) * cm * sd;
  diss[4] = (am + ap) * Hm + (ap - am) * cm * un + a0 * (0.5 * we * vsq + rhom * umjt);
  for (int k = 0; k < 5; ++k) fh[k] = 0.5 * sd * (fa[k] + fb[k]) - 0.5 * diss[k];
}

// Local Lax-Friedrichs flux (the paper's experiment, Sec. 4): the central flux minus half the
// larger of the two states' fastest wave speeds |u . e_d| + c times the jump, n = s e_d.
template <class T>
SC_HD inline void flux_lf(const Geo& G, const T qa[5], const T qb[5], int d, int s, T fh[5]) {
  const double gm1 = G.gamma - 1.0;
  T fa[5], fb[5];
  flux_inviscid(G, qa, d, fa);
  flux_inviscid(G, qb, d, fb);
  const T ira = recip(qa[0]), irb = recip(qb[0]);
  const T uad = qa[1 + d] * ira, ubd = qb[1 + d] * irb;
  const T pa = gm1 * (qa[4] - 0.5 * (qa[1] * qa[1] + qa[2] * qa[2] + qa[3] * qa[3]) * ira);
  const T pb = gm1 * (qb[4] - 0.5 * (qb[1] * qb[1] + qb[2] * qb[2] + qb[3] * qb[3]) * irb);
  const T wa = (vval(uad) >= 0.0 ? uad : -uad) + dsqrt(G.gamma * pa * ira);
  const T wb = (vval(ubd) >= 0.0 ? ubd : -ubd) + dsqrt(G.gamma * pb * irb);
  const T lam = vval(wa) >= vval(wb) ? wa : wb;
  const double sd = (double)s;
  for (int k = 0; k < 5; ++k) fh[k] = 0.5 * sd * (fa[k] + fb[k]) - 0.5 * lam * (qb[k] - qa[k]);
}

// The configured advective numerical flux (Geo::adv_flux: 0 Roe, 1 Lax-Friedrichs).
template <class T>
SC_HD inline void flux_adv(const Geo& G, const T qa[5], const T qb[5], int d, int s, T fh[5]) {
  if (G.adv_flux == 1)
    flux_lf(G, qa, qb, d, s, fh);
  else
    flux_roe(G, qa, qb, d, s, fh);
}

// ------------------------------------------------------------------ host context
struct Pattern {
  // Neighbour couplings of one element (identical for all elements): pair p couples
  // row node row[p] of the element to node col[p] of the neighbour in slot slot[p].
  std::vector<int> row, slot, col;
  // Row-grouped lists (CSR over the element's nodes in natural order).
  std::vector<int> ptr;  // size nn+1
  std::vector<int> ids;  // pair ids
};

struct sc_ctx {
  sc_config cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  bool has_mesh = false, has_state = false, has_dt = false, assembled = false, condensed = false;
  int bdf = 1;
  Geo G{};
  double L = 0.0;
  std::vector<double> xi;          // Gauss-Lobatto nodes
  std::vector<int> perm, iperm;    // natural node -> position (interior first), inverse
  std::vector<int> own_pairs;      // (pj << 16) | pr of the own node pairs sharing a GL index, grouped by kind
  std::vector<int> nbr;            // [K][18] neighbour element per slot
  Pattern pat;
  // device memory
  double *Q = nullptr, *Qh = nullptr, *grad = nullptr, *F = nullptr, *B = nullptr;
  double *NJ = nullptr, *RJ = nullptr, *Aown = nullptr, *X = nullptr;
  // interior penalty only: the elements' own (unlifted) gradients and the point-flux
  // Jacobians at them, same layouts as grad and NJ
  double *gloc = nullptr, *NJL = nullptr;
  int *d_nbr = nullptr, *d_perm = nullptr, *d_iperm = nullptr, *d_own_pairs = nullptr;
  double* gj_scale = nullptr;      // [K][n_i] row scaling of the blocked Gauss-Jordan (T-typed)
  double *OV = nullptr, *OZ = nullptr;  // outer FGMRES: Arnoldi basis (m+1 global vectors), preconditioned (m)
  int *d_prow = nullptr, *d_pslot = nullptr, *d_pcol = nullptr, *d_pptr = nullptr, *d_pinfo = nullptr;
  double *Ainv = nullptr, *Ytmp = nullptr, *See = nullptr;
  int *piv = nullptr, *rowperm = nullptr, *d_status = nullptr;
  // Krylov workspace (boundary space of size n1 = K*nb)
  double *V = nullptr, *Wv = nullptr, *Zv = nullptr, *Xb = nullptr, *Gb = nullptr, *Rb = nullptr;
  double *Ui = nullptr, *Tb = nullptr, *Hd = nullptr, *partial = nullptr, *Xfull = nullptr, *Rfull = nullptr;
  int restart_alloc = 0;
  // mixed-precision arm: FP32 copies of the element blocks and FP32 condensation
  float *Aown32 = nullptr, *X32 = nullptr, *Ainv32 = nullptr, *Y32 = nullptr, *See32 = nullptr;
  float *Zf = nullptr, *Xbf = nullptr, *Uf = nullptr;  // FP32 vectors of the FP32 operator
  double* Cross = nullptr;   // neighbour-coupling products of one pass, FP64 operator
  float* Cross32 = nullptr;  // same, FP32 operator
  double* Dfull = nullptr;  // refinement correction
  double* dQn = nullptr;    // Newton update of sc_newton_step
  // pattern-packed own blocks of the condensed operator (A_ib rows, [A_bi A_bb] rows)
  std::vector<int> pk_lptr, pk_list, pk_pos, pk_row_off;
  std::vector<int> pk_nint;  // per node slot: packed entries of its rows in interior columns (listed first)
  long long pk_stride = 0, pk_nnz_int = 0, pk_nnz_bnd = 0;
  int *d_pk_lptr = nullptr, *d_pk_list = nullptr, *d_pk_row_off = nullptr, *d_pk_pos = nullptr;
  int* d_pk_nint = nullptr;
  double* Apk = nullptr;   // FP64 arm
  float* Apk32 = nullptr;  // mixed arm
  // S_ee factors with partitioned inverses in the block-Jacobi solve layout
  double* Sls = nullptr;
  float* Sls32 = nullptr;
  __half* Sls16 = nullptr;  // FP16 copy of the mixed arm's layout, used when every entry is in range
  bool ls16_ok = false;
  bool packed = false;     // packed blocks match the assembled Jacobian
  // learned correction of the block-Jacobi preconditioner (mixed arm)
  std::vector<int> l_face, l_mirror;  // per boundary position: face, co-located position
  std::vector<int> l_nfaces;          // per boundary position: number of element faces containing the node
  int* d_lnfaces = nullptr;
  // per (boundary position, i-th face containing it): the face, the co-located position in
  // the neighbour across it, and that position's slot of the opposite face
  std::vector<int> l_face3, l_mirror3, l_rslot3;
  int *d_lface3 = nullptr, *d_lmirror3 = nullptr, *d_lrslot3 = nullptr;
  int *d_lface = nullptr, *d_lmirror = nullptr;
  float *Sdiag = nullptr, *Cpl = nullptr;  // [K nbn][25] [S_ee]_kk; [K nbn][3][25] S_(k,k'_f) per face of k
  float *Feat = nullptr, *Snorm = nullptr, *Ynet = nullptr, *Hbuf = nullptr, *Ck = nullptr, *Wbias = nullptr;
  uint16_t* Wbf16 = nullptr;
  bool Sdiag_valid = false, weights_set = false, learned_on = false;
  int learned_fallbacks = 0;
  // explicit Schur blocks W_e over the extended boundary sets (measured alternative)
  int ex_F = 0, ex_m = 0, ex_ldm = 0;
  std::vector<int> ex_nbpos, ex_face_idx;
  int *d_ex_nbpos = nullptr, *d_ex_face_idx = nullptr;
  float *ExIb = nullptr, *ExBi = nullptr, *ExY = nullptr, *ExW = nullptr;
  // red-black sweep over the element Schur blocks (SC_PC_RED_BLACK, SC_PC_LEARNED): the
  // elements of each colour of the checkerboard (ex + ey + ez even = red), red first
  std::vector<int> colour_list;
  int n_red = 0, n_black = 0;
  int* d_colour = nullptr;
  float* Zrb = nullptr;      // FP32 sweep vector (mixed arm)
  double* Trb = nullptr;     // (S z) on the black rows
  // learned correction of the black face blocks: uncorrected copies, corrected factors
  float *SeeB = nullptr, *SeeL = nullptr, *SlsL = nullptr;
  int *pivL = nullptr, *rowpermL = nullptr;
  bool blackL_valid = false;  // SlsL holds the factors of the corrected black blocks
  bool red_compact = false;   // SC_PC_RB_SCHUR: Sls32 / rowperm hold only the red blocks' factors,
                              // entry i for the i-th red element (the black ones are in SlsL)
  // Schur-corrected sweep (SC_PC_RB_SCHUR): the red blocks' inverses, column-major per red
  // element (Zinv[r][j][i] = (S_rr^-1)[i][j], r the red list index), red index of every
  // element (-1 for black), and per face f the (N+1)^2 boundary nodes on f with the slot of f
  // in each node's face list: face_tab[(2 f) P2 + t] = node, face_tab[(2 f + 1) P2 + t] = slot
  float* Zinv = nullptr;
  std::vector<int> red_index, face_tab;
  int *d_redidx = nullptr, *d_face_tab = nullptr;
  // dense direct solve (sc_direct_factor): n x n factors (row-major, ld = ldd), pivots
  void* Dlu = nullptr;       // double (FP64 arm) or float (mixed arm)
  int* d_dpiv = nullptr;
  double* Dcorr = nullptr;   // one refinement sweep's correction (K ne doubles)
  int direct_n = 0, direct_ld = 0, direct_which = -1;
  bool direct_valid = false;
  bool op32 = false;        // the condensed operator / preconditioner run on the FP32 copies
  cudaEvent_t ev[8] = {};
  // measurement hooks: kernel launches since creation, and optional CUDA-event timing
  // of every launch of one selected kernel (see sc_profile_kernel)
  long long launches = 0;
  int prof_kernel = -1;
  std::vector<cudaEvent_t> prof_ev;  // start/stop pairs, reused
  int prof_used = 0;
  double prof_ms = 0.0;
  long long prof_count = 0;
  long long prof_elems = 0;  // elements processed by the profiled launches
};

// Kernel ids of the measurement hook (sc_profile_kernel).
enum { SCK_COND_INTERIOR = 0, SCK_COND_BOUNDARY = 1, SCK_LU_SOLVE = 2, SCK_LU = 3, SCK_GEMM = 4,
       SCK_GJ_INV = 5, SCK_ASM_OWN = 6, SCK_GLOBAL_APPLY = 7, SCK_EXPLICIT_GEMM = 8, SCK_EXPLICIT_APPLY = 9,
       SCK_COUNT = 10 };

// Bracket one launch of kernel `id` with events when it is the profiled kernel; `elements`
// is the number of elements the launch processes (default: every element of the mesh).
struct ProfScope {
  sc_ctx* c; int id; bool on;
  ProfScope(sc_ctx* cc, int kid, int elements = -1) : c(cc), id(kid), on(cc->prof_kernel == kid) {
    c->launches++;
    if (on) {
      c->prof_elems += elements < 0 ? c->G.K : elements;
      if ((int)c->prof_ev.size() < 2 * (c->prof_used + 1)) {
        cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
        c->prof_ev.push_back(a); c->prof_ev.push_back(b);
      }
      cudaEventRecord(c->prof_ev[2 * c->prof_used], c->stream);
    }
  }
  ~ProfScope() {
    if (on) { cudaEventRecord(c->prof_ev[2 * c->prof_used + 1], c->stream); c->prof_used++; }
  }
};
// Count a launch that is never profiled.
inline void count_launch(sc_ctx* c, int n = 1) { c->launches += n; }

// kernels launchers (defined in the .cu files)
// One element of a batched condensation (elements of several systems, any order): its
// sizes and the addresses of its FP32 blocks.
struct CondItem {
  int ni, nb, lda, ldi, lds, e;  // sizes and leading dimensions; e: element index reported on failure
  const float* Aown;              // own block (ne x lda), interior columns first, boundary at cb0
  int cb0;
  float *Ainv, *Yt, *See, *Sls;   // A_ii^-1 (ni x ldi), Y^T (nb x ldi), S_ee (nb x lds), solve layout
  int *piv, *rowperm;
  int* status;
  float* dsc;                     // n_i row scales of the blocked Gauss-Jordan (n_i > 136)
};

// Status word value written by a tensor-core kernel whose bounded wait ran out (element
// indices written by the factorisations are far below it).
constexpr int SC_TC_TIMEOUT = 1 << 30;
// Status word value written by the packing kernel when an own-block entry outside the
// packed pattern is nonzero.
constexpr int SC_PACK_VIOLATION = (1 << 30) + 1;
// Status word value written when an interior row couples outside the extended boundary
// set of the explicit Schur blocks.
constexpr int SC_EXPLICIT_PATTERN = (1 << 30) + 2;

namespace sc {
// Gauss-Lobatto nodes x, weights w and differentiation matrix D[a][b] = l_b'(x_a) of order N.
void gl_basis(int N, std::vector<double>& x, std::vector<double>& w, double D[SC_MAXP][SC_MAXP]);
cudaError_t launch_residual(sc_ctx* c);
// -R(Q) with the geometry G (c0 = 0 gives -H(Q), the spatial operator alone) into out;
// uses c->grad and c->F as scratch.
cudaError_t launch_residual_geo(sc_ctx* c, const Geo& G, const double* Q, const double* Qh, double* out);
cudaError_t launch_history(sc_ctx* c, const double* Qs, const double* Qsm1);
cudaError_t launch_assembly(sc_ctx* c);
cudaError_t launch_condense(sc_ctx* c);
cudaError_t cond_interior(sc_ctx* c, const double* xb, double beta, const double* Bfull, double alpha,
                          double* u);
cudaError_t cond_boundary(sc_ctx* c, const double* xb, double delta, const double* Bfull, double gamma_,
                          const double* u, double* y);
cudaError_t precond_apply(sc_ctx* c, const double* v, double* z);
cudaError_t precond_apply32(sc_ctx* c, const double* v, double* z, float* zf);
cudaError_t cond_interior32(sc_ctx* c, const float* xb, double beta, const double* Bfull, double alpha, float* u);
cudaError_t cond_boundary32(sc_ctx* c, const float* xb, double delta, const double* Bfull, double gamma_,
                            const float* u, double* y);
cudaError_t scatter_solution32(sc_ctx* c, const double* xb, const float* xi, double* x);
cudaError_t vec_to_float(sc_ctx* c, float* y, const double* x, size_t n);
cudaError_t global_apply(sc_ctx* c, const double* x, double* y);
cudaError_t scatter_solution(sc_ctx* c, const double* xb, const double* xi, double* x);
cudaError_t multidot(sc_ctx* c, const double* V, int nvec, size_t n, const double* w, double* out_dev);
cudaError_t vec_update(sc_ctx* c, double* w, const double* V, int nvec, size_t n, const double* coef_dev,
                       double sign);
cudaError_t vec_scale_copy(sc_ctx* c, double* dst, const double* src, size_t n, const double* scal_dev,
                           int invert);
// Batched TF32 tensor-core GEMM C = alpha op(A) op(B) + beta C (row-major FP32 blocks;
// ta: A stored K x M, tb: B stored N x K).  A tensor-core wait that times out stores
// SC_TC_TIMEOUT into *status if it still holds -1.
cudaError_t gemm_tf32(cudaStream_t stream, int M, int N, int K, float alpha, const float* A, long long sA, int lda,
                      bool ta, const float* B, long long sB, int ldb, bool tb, float beta, float* C, long long sC,
                      int ldc, int batch, int* status);
size_t solve_layout_elems(const Geo& G);
void build_packed_pattern(sc_ctx* c);
long long solve_layout_stride(const Geo& G);
cudaError_t factor_batch32(sc_ctx* c, float* A, int n, int lda, long long stride, int batch, int* piv, int* rowperm,
                           float* LS, int* status);
void build_learned_tables(sc_ctx* c);
void build_explicit_tables(sc_ctx* c);
cudaError_t upload_explicit_tables(sc_ctx* c);
size_t explicit_elems_W(const Geo& G, const sc_ctx* c);
cudaError_t explicit_build(sc_ctx* c);
cudaError_t explicit_matvec32(sc_ctx* c, const float* x, double* y);
// Items are sorted by decreasing block size; the first nbig of them take the large-block
// kernels (blocked Gauss-Jordan for n_i > 136, shared-memory panels for n_b > 496).
cudaError_t grouped_gj(cudaStream_t st, const CondItem* items, int n, int nbig, int max_ni);
int grouped_gj_launches(int nbig, int n, int max_ni);
bool gj_blocked_item(int ni);
bool lu_panel_smem_item(int nb);
cudaError_t grouped_copy_bb(cudaStream_t st, const CondItem* items, int n);
cudaError_t grouped_lu_panel(cudaStream_t st, const CondItem* items, int n, int nbig, int k0, int max_nb);
cudaError_t grouped_finish(cudaStream_t st, const CondItem* items, int n, int max_nb);
cudaError_t to_float(sc_ctx* c, const double* a, float* b, size_t n);
cudaError_t gemm_tf32_ptrs(cudaStream_t stream, int M, int N, int K, float alpha, const float* const* Ap, int lda,
                           bool ta, const float* const* Bp, int ldb, bool tb, float beta, float* const* Cp, int ldc,
                           int batch, int bn, int* status);
cudaError_t gemm_fp32(sc_ctx* c, int M, int N, int K, const float* A, long long sA, int lda, const float* B,
                      long long sB, int ldb, float* C, long long sC, int ldc, int batch);
cudaError_t extract_sdiag(sc_ctx* c, const float* See);
cudaError_t learned_features(sc_ctx* c, float* F, float* snorm);
cudaError_t learned_correction(sc_ctx* c);
cudaError_t assemble_correction(sc_ctx* c, const float* Y, float scale);
// FP32 interior inverses up to this n_i run register-resident (k_gj_inv_reg); larger ones blocked
constexpr int kGjRegRows = 136;
constexpr int kMlpInputs = 128;
constexpr int kMlpWeights = 256 * kMlpInputs + 256 * 256 + 25 * 256, kMlpBiases = 2 * 256 + 25;
cudaError_t mlp_forward(cudaStream_t st, const uint16_t* Wbf16, const float* bias, const float* X, int n, float* Y,
                        float* h1, float* h2);
cudaError_t upload_packed_pattern(sc_ctx* c);
cudaError_t pack_own(sc_ctx* c);
template <class T>
cudaError_t cond_interior_pk(sc_ctx* c, const T* Apk, const T* X, const T* Ainv, const T* xb, double beta,
                             const double* Bfull, double alpha, T* u, int black_zero);
cudaError_t cond_interior_sweep(sc_ctx* c, const double* xb, double* u);
cudaError_t cond_interior_sweep32(sc_ctx* c, const float* xb, float* u);
template <class T>
cudaError_t cond_boundary_pk(sc_ctx* c, const T* Apk, const T* X, const T* xb, double delta, const double* Bfull,
                             double gamma_, const T* u, double* y);
cudaError_t vec_axpby(sc_ctx* c, double* y, double a, const double* x, double b, size_t n);
// block solves of a list of elements (factors by element, or compact by list position), vsub
// subtracted from the right-hand side
cudaError_t lu_solve_list(sc_ctx* c, const double* LS, const int* rowperm, int compact, const int* elist, int nlist,
                          const double* v, const double* vsub, double* z);
cudaError_t lu_solve_list32(sc_ctx* c, const float* LS, const int* rowperm, int compact, const int* elist, int nlist,
                            const double* v, const double* vsub, double* z, float* zt);
template <class T>
cudaError_t cond_boundary_pk_list(sc_ctx* c, const T* Apk, const T* X, const T* xb, const T* u, double* y,
                                  const int* elist, int nlist);
// red-black sweep (precond SC_PC_RED_BLACK, or SC_PC_LEARNED while the learned correction is on)
void build_colours(sc_ctx* c);
bool rb_active(const sc_ctx* c);
cudaError_t precond_rb(sc_ctx* c, const double* v, double* z);
cudaError_t precond_rb32(sc_ctx* c, const double* v, double* z, float* zf);
cudaError_t learned_black_factor(sc_ctx* c, const float* Ck, float scale);
cudaError_t learned_couplings(sc_ctx* c);
void build_face_tables(sc_ctx* c);
cudaError_t schur_black_factor(sc_ctx* c);
cudaError_t red_factor32(sc_ctx* c, const float* See);
cudaError_t plain_black_factor(sc_ctx* c);
cudaError_t inverse_columns32(sc_ctx* c, const int* list, int nlist, float* out);
cudaError_t gather_black_see(sc_ctx* c, const float* See);
template <class T>
cudaError_t gemm_update(sc_ctx* c, int M, int N, int K, const T* A, int lda, const T* B, int ldb, T* C, int ldc);
void free_direct_factors(sc_ctx* c);
// [S_ee^-1]_kk for every (element, boundary node) sample from the condensation's factors
cudaError_t inverse_node_blocks32(sc_ctx* c, float* out);
}  // namespace sc
