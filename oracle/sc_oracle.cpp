// FP64 CPU oracle for the statically condensed GL-DGSEM Newton system.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls this
// file; only the tests, the smoke check and the CPU-baseline leg of the benchmark
// load it.  It shares no code, header or table with the CUDA path.
//
// What it computes (all in double precision, straight from the paper's equations):
//   * Gauss-Lobatto nodes and weights and the Lagrange basis (App. C, eqs. mapping,
//     quadRule; discrete orthogonality l_i(xi_j) = delta_ij).
//   * The weak-form GL-DGSEM residual of Sec. 2.1, eq. DGSEMsystem:
//       lifting   J_m w_m g_m = - sum_n J w_n q_n grad phi_m(x_n) + int phi_m qhat n dS
//       outer eq  R_j = J_j w_j dQ/dt - sum_m J w_m F(q_m, g_m) . grad phi_j(x_m)
//                       + int fhat phi_j dS
//     with F = f^a - f^nu (App. B), fhat = Roe(q+, q-, n) - BR1 average of f^nu . n,
//     qhat = (q+ + q-)/2 (BR1), and a BDF1/BDF2 time term (eqs. ImplicitDisc,
//     NeqtonEq).
//   * The Jacobian A = dR/dQ of eq. NewtonLinSys1 by forward-mode dual numbers
//     (exact to rounding), column node by column node, and the Jacobian-vector
//     product A x with a one-direction dual.
// The condensation itself (Sec. 2.2 eqs. StaticCondBlock, SC_step1, SC_step2) lives
// in oracle/linalg.py on top of these matrices.
//
// Readings of the paper used here:
//   * nondimensionalisation rho_inf = V_inf = L_inf = T_inf = 1, p_inf = 1/(gamma Ma^2),
//     T = gamma Ma^2 p / rho, kappa = mu / ((gamma-1) Pr Ma^2)  (App. B, kappa);
//   * Stokes stress tau = mu (grad v + grad v^T) - (2/3) mu (div v) I (App. B);
//   * Sutherland mu = (1+S)/(T+S) T^(3/2), S = T_suth / T_inf (App. B);
//   * Roe flux with Roe averages and Harten's entropy fix on every wave,
//     |lambda| -> (lambda^2 + delta^2)/(2 delta) for |lambda| < delta,
//     delta = roe_delta * c_roe (the paper names Roe without details);
//   * or (adv_flux = 1) the Lax-Friedrichs flux of the paper's experiment (Sec. 4), read as
//     the local one: fhat = (f(q+) + f(q-)) . n / 2 - lambda (q- - q+) / 2 with
//     lambda = max over the two states of |u . n| + c;
//   * or (visc_flux = 1) the symmetric interior-penalty viscous flux of the paper's
//     experiment (Sec. 4), read inside the paper's mixed form: the volume term keeps the
//     lifted gradient with qhat = (q+ + q-)/2, and the face flux becomes the compact
//     f^nu_hat . n = (f^nu(q+, grad q+) + f^nu(q-, grad q-)) . n / 2 + sigma (q- - q+) with
//     the elements' own (unlifted) gradients, sigma = C_IP (N+1)^2 nu_ref / h on all five
//     variables.  For linear diffusion this is the SIPG bilinear form with Gauss-Lobatto
//     quadrature: the lifted volume gradient supplies the symmetrising term.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- dual numbers
template <int ND>
struct Dual {
  double v;
  double d[ND];
  Dual() : v(0.0) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < ND; ++i) d[i] = 0.0; }
};

template <int ND> inline Dual<ND> operator+(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v + b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int ND> inline Dual<ND> operator-(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v - b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int ND> inline Dual<ND> operator-(const Dual<ND>& a) {
  Dual<ND> r; r.v = -a.v; for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r; }
template <int ND> inline Dual<ND> operator*(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v * b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int ND> inline Dual<ND> operator/(const Dual<ND>& a, const Dual<ND>& b) {
  Dual<ND> r; r.v = a.v / b.v; const double ib = 1.0 / (b.v * b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) * ib;
  return r; }
template <int ND> inline Dual<ND> operator+(const Dual<ND>& a, double b) { Dual<ND> r = a; r.v += b; return r; }
template <int ND> inline Dual<ND> operator+(double b, const Dual<ND>& a) { return a + b; }
template <int ND> inline Dual<ND> operator-(const Dual<ND>& a, double b) { Dual<ND> r = a; r.v -= b; return r; }
template <int ND> inline Dual<ND> operator-(double b, const Dual<ND>& a) { return (-a) + b; }
template <int ND> inline Dual<ND> operator*(const Dual<ND>& a, double b) {
  Dual<ND> r; r.v = a.v * b; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b; return r; }
template <int ND> inline Dual<ND> operator*(double b, const Dual<ND>& a) { return a * b; }
template <int ND> inline Dual<ND> operator/(const Dual<ND>& a, double b) { return a * (1.0 / b); }
template <int ND> inline Dual<ND> operator/(double a, const Dual<ND>& b) { return Dual<ND>(a) / b; }
template <int ND> inline Dual<ND>& operator+=(Dual<ND>& a, const Dual<ND>& b) { a = a + b; return a; }
template <int ND> inline Dual<ND>& operator-=(Dual<ND>& a, const Dual<ND>& b) { a = a - b; return a; }
template <int ND> inline Dual<ND> sqrt(const Dual<ND>& a) {
  Dual<ND> r; r.v = std::sqrt(a.v); const double s = 0.5 / r.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * s;
  return r; }

inline double val(double x) { return x; }
template <int ND> inline double val(const Dual<ND>& x) { return x.v; }
using std::sqrt;

}  // namespace

extern "C" {
struct or_params {
  int n;            // elements per direction (periodic n^3 mesh)
  int N;            // polynomial order
  double L;         // box side
  double dt;        // time step
  int bdf;          // 1 or 2
  double gamma, Pr, Re, Ma, Ts;  // Ts = T_sutherland / T_inf
  int sutherland;   // 1: Sutherland viscosity, 0: mu = 1
  int model;        // 0: Navier-Stokes; 1: five copies of linear advection-diffusion
  int viscous;      // 0 drops the viscous flux (Euler / pure advection)
  double adv[3];    // advection speed of model 1
  double nu;        // diffusivity of model 1
  double roe_delta; // entropy-fix width as a fraction of the Roe sound speed
  int with_time;    // 0 drops the time term (spatial operator H only)
  int adv_flux;     // 0: Roe with entropy fix; 1: local Lax-Friedrichs (the paper's experiment, Sec. 4)
  int visc_flux;    // 0: BR1 (non-compact); 1: symmetric interior penalty (compact, Sec. 4)
  double ip_penalty;  // C_IP of the interior-penalty coefficient sigma = C_IP (N+1)^2 nu_ref / h
};
}

namespace {

constexpr int NV = 5;

// Gauss-Lobatto nodes/weights by Newton iteration on P_N' (App. C), Lagrange basis
// values and derivatives from the product formula.
struct Basis {
  int N = 0, p = 0;
  std::vector<double> xi, w;
  std::vector<double> ell;   // ell[i*p + a] = l_i(xi_a)
  std::vector<double> dell;  // dell[i*p + a] = l_i'(xi_a)
  std::vector<double> eL, eR;  // l_i(-1), l_i(+1)
};

void legendre(int N, double x, double& P, double& dP, double& d2P) {
  // Three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; the derivatives
  // follow from P'_{k+1} = P'_{k-1} + (2k+1) P_k and its derivative.
  double p0 = 1.0, p1 = x, dp0 = 0.0, dp1 = 1.0, d2p0 = 0.0, d2p1 = 0.0;
  if (N == 0) { P = 1.0; dP = 0.0; d2P = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    double dp2 = dp0 + (2 * k + 1) * p1;
    double d2p2 = d2p0 + (2 * k + 1) * dp1;
    p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2; d2p0 = d2p1; d2p1 = d2p2;
  }
  P = p1; dP = dp1; d2P = d2p1;
}

double lagrange(const std::vector<double>& xi, int i, double x) {
  double r = 1.0;
  for (size_t m = 0; m < xi.size(); ++m)
    if ((int)m != i) r *= (x - xi[m]) / (xi[i] - xi[m]);
  return r;
}

double lagrange_deriv(const std::vector<double>& xi, int i, double x) {
  // d/dx prod_{m != i} (x - xi_m)/(xi_i - xi_m) by the product rule.
  double s = 0.0;
  for (size_t k = 0; k < xi.size(); ++k) {
    if ((int)k == i) continue;
    double t = 1.0 / (xi[i] - xi[k]);
    for (size_t m = 0; m < xi.size(); ++m)
      if ((int)m != i && m != k) t *= (x - xi[m]) / (xi[i] - xi[m]);
    s += t;
  }
  return s;
}

Basis make_basis(int N) {
  Basis b; b.N = N; b.p = N + 1;
  b.xi.assign(N + 1, 0.0); b.w.assign(N + 1, 0.0);
  b.xi[0] = -1.0; b.xi[N] = 1.0;
  const double pi = 3.14159265358979323846;
  for (int k = 1; k < N; ++k) {
    double x = -std::cos(pi * k / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P; legendre(N, x, P, dP, d2P);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    b.xi[k] = x;
  }
  for (int k = 0; k <= N / 2; ++k) {  // symmetrise
    double a = 0.5 * (b.xi[N - k] - b.xi[k]);
    b.xi[k] = -a; b.xi[N - k] = a;
  }
  if (N % 2 == 0) b.xi[N / 2] = 0.0;
  for (int k = 0; k <= N; ++k) {
    double P, dP, d2P; legendre(N, b.xi[k], P, dP, d2P);
    b.w[k] = 2.0 / (N * (N + 1) * P * P);
  }
  const int p = b.p;
  b.ell.resize(p * p); b.dell.resize(p * p); b.eL.resize(p); b.eR.resize(p);
  for (int i = 0; i < p; ++i) {
    for (int a = 0; a < p; ++a) {
      b.ell[i * p + a] = lagrange(b.xi, i, b.xi[a]);
      b.dell[i * p + a] = lagrange_deriv(b.xi, i, b.xi[a]);
    }
    b.eL[i] = lagrange(b.xi, i, -1.0);
    b.eR[i] = lagrange(b.xi, i, 1.0);
  }
  return b;
}

// ---------------------------------------------------------------- physics (App. B)
template <class T>
void adv_flux(const or_params& P, const T* q, int d, T* f) {
  if (P.model == 1) {
    for (int k = 0; k < NV; ++k) f[k] = q[k] * P.adv[d];
    return;
  }
  const double g = P.gamma;
  T rho = q[0];
  T vel[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  T p = (g - 1.0) * (q[4] - 0.5 * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]));
  f[0] = q[1 + d];
  for (int i = 0; i < 3; ++i) f[1 + i] = q[1 + i] * vel[d];
  f[1 + d] += p;
  f[4] = vel[d] * (q[4] + p);
}

template <class T>
T viscosity(const or_params& P, const T& Tmp) {
  if (!P.sutherland) return T(1.0);
  const double S = P.Ts;
  return (1.0 + S) / (Tmp + S) * Tmp * sqrt(Tmp);
}

// Viscous flux f^nu_d(q, g), g[a*NV + k] = d q_k / d x_a.
template <class T>
void visc_flux(const or_params& P, const T* q, const T* g, int d, T* f) {
  if (!P.viscous) { for (int k = 0; k < NV; ++k) f[k] = T(0.0); return; }
  if (P.model == 1) {
    for (int k = 0; k < NV; ++k) f[k] = P.nu * g[d * NV + k];
    return;
  }
  const double gm = P.gamma;
  T rho = q[0];
  T vel[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  T E = q[4] / rho;
  // gradients of primitive quantities from gradients of conserved ones
  T dv[3][3];  // dv[a][i] = d u_i / d x_a
  T dE[3];
  for (int a = 0; a < 3; ++a) {
    for (int i = 0; i < 3; ++i) dv[a][i] = (g[a * NV + 1 + i] - vel[i] * g[a * NV + 0]) / rho;
    dE[a] = (g[a * NV + 4] - E * g[a * NV + 0]) / rho;
  }
  T e = E - 0.5 * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]);
  // T = gamma Ma^2 p / rho with p = (gamma-1) rho e
  T Tmp = gm * (gm - 1.0) * P.Ma * P.Ma * e;
  T mu = viscosity(P, Tmp);
  T dT[3];
  for (int a = 0; a < 3; ++a) {
    T de = dE[a] - (vel[0] * dv[a][0] + vel[1] * dv[a][1] + vel[2] * dv[a][2]);
    dT[a] = gm * (gm - 1.0) * P.Ma * P.Ma * de;
  }
  T kappa = mu / ((gm - 1.0) * P.Pr * P.Ma * P.Ma);
  T div = dv[0][0] + dv[1][1] + dv[2][2];
  T tau[3];  // tau_{d i}
  for (int i = 0; i < 3; ++i) {
    tau[i] = mu * (dv[d][i] + dv[i][d]);
    if (i == d) tau[i] = tau[i] - (2.0 / 3.0) * mu * div;
  }
  const double iRe = 1.0 / P.Re;
  f[0] = T(0.0);
  for (int i = 0; i < 3; ++i) f[1 + i] = iRe * tau[i];
  f[4] = iRe * (vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2] + kappa * dT[d]);
}

template <class T>
T abs_fixed(const T& lam, const T& delta) {
  // Harten's entropy fix: |lambda| below delta is replaced by a parabola.
  if (std::fabs(val(lam)) >= val(delta)) return val(lam) >= 0 ? lam : -lam;
  return (lam * lam + delta * delta) / (2.0 * delta);
}

// Advective numerical flux fhat^a(q+, q-, n) . n with n = s e_d (outward for q+).
template <class T>
void num_flux_adv(const or_params& P, const T* qL, const T* qR, int d, int s, T* fh) {
  T fL[NV], fR[NV];
  adv_flux(P, qL, d, fL);
  adv_flux(P, qR, d, fR);
  if (P.model == 1) {
    double an = P.adv[d] * s;
    for (int k = 0; k < NV; ++k)
      fh[k] = 0.5 * (double)s * (fL[k] + fR[k]) - 0.5 * std::fabs(an) * (qR[k] - qL[k]);
    return;
  }
  const double g = P.gamma;
  T rL = qL[0], rR = qR[0];
  T uL[3] = {qL[1] / rL, qL[2] / rL, qL[3] / rL};
  T uR[3] = {qR[1] / rR, qR[2] / rR, qR[3] / rR};
  T pL = (g - 1.0) * (qL[4] - 0.5 * rL * (uL[0] * uL[0] + uL[1] * uL[1] + uL[2] * uL[2]));
  T pR = (g - 1.0) * (qR[4] - 0.5 * rR * (uR[0] * uR[0] + uR[1] * uR[1] + uR[2] * uR[2]));
  if (P.adv_flux == 1) {
    // local Lax-Friedrichs: the central flux minus half the larger of the two states' fastest
    // wave speeds |u.n| + c times the jump
    T sL = sqrt(g * pL / rL), sR = sqrt(g * pR / rR);
    T wL = (val(uL[d]) >= 0 ? uL[d] : -uL[d]) + sL;
    T wR = (val(uR[d]) >= 0 ? uR[d] : -uR[d]) + sR;
    T lam = val(wL) >= val(wR) ? wL : wR;
    for (int k = 0; k < NV; ++k) fh[k] = 0.5 * (double)s * (fL[k] + fR[k]) - 0.5 * lam * (qR[k] - qL[k]);
    return;
  }
  T HL = (qL[4] + pL) / rL, HR = (qR[4] + pR) / rR;
  T sL = sqrt(rL), sR = sqrt(rR);
  T den = sL + sR;
  T ut[3];
  for (int i = 0; i < 3; ++i) ut[i] = (sL * uL[i] + sR * uR[i]) / den;
  T Ht = (sL * HL + sR * HR) / den;
  T q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  T ct = sqrt((g - 1.0) * (Ht - 0.5 * q2));
  T rt = sL * sR;
  T unt = ut[d] * (double)s;
  T drho = rR - rL, dp = pR - pL;
  T du[3] = {uR[0] - uL[0], uR[1] - uL[1], uR[2] - uL[2]};
  T dun = du[d] * (double)s;
  T c2 = ct * ct;
  T a1 = (dp - rt * ct * dun) / (2.0 * c2);
  T a2 = drho - dp / c2;
  T a5 = (dp + rt * ct * dun) / (2.0 * c2);
  T delta = P.roe_delta * ct;
  T l1 = abs_fixed(unt - ct, delta);
  T l2 = abs_fixed(unt, delta);
  T l5 = abs_fixed(unt + ct, delta);
  double n[3] = {0.0, 0.0, 0.0}; n[d] = (double)s;
  T dut[3];  // tangential velocity jump
  for (int i = 0; i < 3; ++i) dut[i] = du[i] - dun * n[i];
  T utdut = ut[0] * dut[0] + ut[1] * dut[1] + ut[2] * dut[2];
  T diss[NV];
  // acoustic wave u - c
  diss[0] = l1 * a1;
  for (int i = 0; i < 3; ++i) diss[1 + i] = l1 * a1 * (ut[i] - ct * n[i]);
  diss[4] = l1 * a1 * (Ht - ct * unt);
  // entropy wave
  diss[0] += l2 * a2;
  for (int i = 0; i < 3; ++i) diss[1 + i] += l2 * a2 * ut[i];
  diss[4] += l2 * a2 * (0.5 * q2);
  // shear waves
  for (int i = 0; i < 3; ++i) diss[1 + i] += l2 * rt * dut[i];
  diss[4] += l2 * rt * utdut;
  // acoustic wave u + c
  diss[0] += l5 * a5;
  for (int i = 0; i < 3; ++i) diss[1 + i] += l5 * a5 * (ut[i] + ct * n[i]);
  diss[4] += l5 * a5 * (Ht + ct * unt);
  for (int k = 0; k < NV; ++k) fh[k] = 0.5 * (double)s * (fL[k] + fR[k]) - 0.5 * diss[k];
}

// ---------------------------------------------------------------- mesh + discretisation
struct Disc {
  or_params P;
  Basis B;
  int n, N, p, nn, K;
  double h, J, Jf, dx;  // J = (h/2)^3 volume Jacobian, Jf = (h/2)^2 face Jacobian, dx = 2/h metric
  explicit Disc(const or_params& pp) : P(pp) {
    n = P.n; N = P.N; p = N + 1; nn = p * p * p; K = n * n * n;
    B = make_basis(N);
    h = P.L / n; J = std::pow(0.5 * h, 3); Jf = std::pow(0.5 * h, 2); dx = 2.0 / h;
  }
  int node(int i, int j, int k) const { return i + p * (j + p * k); }
  void coords(int m, int c[3]) const { c[0] = m % p; c[1] = (m / p) % p; c[2] = m / (p * p); }
  int elem(int ex, int ey, int ez) const {
    ex = ((ex % n) + n) % n; ey = ((ey % n) + n) % n; ez = ((ez % n) + n) % n;
    return ex + n * (ey + n * ez);
  }
  void ecoords(int e, int c[3]) const { c[0] = e % n; c[1] = (e / n) % n; c[2] = e / (n * n); }
  int neighbor(int e, int d, int s) const {
    int c[3]; ecoords(e, c); c[d] += s; return elem(c[0], c[1], c[2]);
  }
};

// State accessor: the global double-precision state, with the five variables of one
// node seeded as the dual directions (Jacobian columns) or a direction vector (JVP).
template <class T>
struct Access {
  const Disc* D; const double* Q; int se = -1, sn = -1;
  T get(int e, int m, int k) const { return T(Q[((size_t)e * D->nn + m) * NV + k]); }
};
template <int ND>
struct Access<Dual<ND>> {
  const Disc* D; const double* Q; int se = -1, sn = -1; const double* dir = nullptr;
  Dual<ND> get(int e, int m, int k) const {
    Dual<ND> t(Q[((size_t)e * D->nn + m) * NV + k]);
    if (dir) { t.d[0] = dir[((size_t)e * D->nn + m) * NV + k]; }
    else if (e == se && m == sn && k < ND) t.d[k] = 1.0;
    return t;
  }
};

// Value of the element's polynomial at a face point (face d, side s, in-face node
// indices fb, fc): sum over nodes of q_n phi_n(x), reduced with l_i(xi_j) = delta_ij
// in the two in-face directions.
template <class T, class A>
void trace(const Disc& D, const A& acc, int e, int d, int s, int fb, int fc, T* out) {
  const std::vector<double>& edge = (s > 0) ? D.B.eR : D.B.eL;
  for (int k = 0; k < NV; ++k) out[k] = T(0.0);
  int db = (d + 1) % 3, dc = (d + 2) % 3;
  for (int a = 0; a < D.p; ++a) {
    double phi = edge[a];
    if (phi == 0.0) continue;
    int c[3]; c[d] = a; c[db] = fb; c[dc] = fc;
    int m = D.node(c[0], c[1], c[2]);
    for (int k = 0; k < NV; ++k) out[k] += phi * acc.get(e, m, k);
  }
}

// Gradient of the element's own polynomial (no lifting) at the same face point:
// out[a*NV + k] = d/dx_a sum_n q_n phi_n(x).  This is the local gradient that a compact
// viscous flux takes on each side of a face (Sec. 2.1, compact fluxes).
template <class T, class A>
void trace_grad(const Disc& D, const A& acc, int e, int d, int s, int fb, int fc, T* out) {
  const Basis& B = D.B;
  const std::vector<double>& edge = (s > 0) ? B.eR : B.eL;
  const int xf = (s > 0) ? D.N : 0;  // xi = +-1 is the Gauss-Lobatto node 0 or N
  for (int x = 0; x < 3 * NV; ++x) out[x] = T(0.0);
  int db = (d + 1) % 3, dc = (d + 2) % 3;
  for (int a = 0; a < D.p; ++a)
    for (int b = 0; b < D.p; ++b)
      for (int cc = 0; cc < D.p; ++cc) {
        // phi = l_a(xi_d) l_b(xi_db) l_cc(xi_dc) evaluated / differentiated at the point
        double v_d = edge[a], dv_d = B.dell[a * D.p + xf];
        double v_b = (b == fb) ? 1.0 : 0.0, dv_b = B.dell[b * D.p + fb];
        double v_c = (cc == fc) ? 1.0 : 0.0, dv_c = B.dell[cc * D.p + fc];
        double gd[3];
        gd[d] = D.dx * dv_d * v_b * v_c;
        gd[db] = D.dx * v_d * dv_b * v_c;
        gd[dc] = D.dx * v_d * v_b * dv_c;
        if (gd[0] == 0.0 && gd[1] == 0.0 && gd[2] == 0.0) continue;
        int c[3]; c[d] = a; c[db] = b; c[dc] = cc;
        int m = D.node(c[0], c[1], c[2]);
        for (int k = 0; k < NV; ++k) {
          T qm = acc.get(e, m, k);
          for (int x = 0; x < 3; ++x)
            if (gd[x] != 0.0) out[x * NV + k] += gd[x] * qm;
        }
      }
}

// Interior-penalty coefficient (reading of the unstated constant): sigma = C_IP (N+1)^2
// nu_ref / h with nu_ref the reference diffusivity, 1/Re for Navier-Stokes (mu = 1 at the
// free-stream temperature) and nu for the advection-diffusion model.
double ip_sigma(const or_params& P, int N, double h) {
  if (!P.viscous) return 0.0;
  const double nu_ref = (P.model == 1) ? P.nu : 1.0 / P.Re;
  return P.ip_penalty * (N + 1.0) * (N + 1.0) * nu_ref / h;
}

// Weak-form lifting (eq. DGSEMsystem:2): g[m][a][k] for every node m of element e.
template <class T, class A>
void lifting(const Disc& D, const A& acc, int e, T* g /* nn*3*NV */) {
  const Basis& B = D.B;
  const int p = D.p;
  for (int m = 0; m < D.nn; ++m) {
    int cm[3]; D.coords(m, cm);
    T s3[3][NV];
    for (int a = 0; a < 3; ++a) for (int k = 0; k < NV; ++k) s3[a][k] = T(0.0);
    // volume: - sum_n J w_n q_n d_a phi_m(x_n)
    for (int nidx = 0; nidx < D.nn; ++nidx) {
      int cn[3]; D.coords(nidx, cn);
      double wn = B.w[cn[0]] * B.w[cn[1]] * B.w[cn[2]];
      double e0 = B.ell[cm[0] * p + cn[0]], e1 = B.ell[cm[1] * p + cn[1]], e2 = B.ell[cm[2] * p + cn[2]];
      double d0 = B.dell[cm[0] * p + cn[0]], d1 = B.dell[cm[1] * p + cn[1]], d2 = B.dell[cm[2] * p + cn[2]];
      double gp[3] = {D.dx * d0 * e1 * e2, D.dx * e0 * d1 * e2, D.dx * e0 * e1 * d2};
      if (gp[0] == 0.0 && gp[1] == 0.0 && gp[2] == 0.0) continue;
      for (int k = 0; k < NV; ++k) {
        T qn = acc.get(e, nidx, k);
        for (int a = 0; a < 3; ++a)
          if (gp[a] != 0.0) s3[a][k] -= (D.J * wn * gp[a]) * qn;
      }
    }
    // surface: int phi_m qhat n dS over the six faces
    for (int d = 0; d < 3; ++d) {
      int db = (d + 1) % 3, dc = (d + 2) % 3;
      for (int s = -1; s <= 1; s += 2) {
        const std::vector<double>& edge = (s > 0) ? B.eR : B.eL;
        double phin = edge[cm[d]];
        if (phin == 0.0) continue;
        int fb = cm[db], fc = cm[dc];  // face point co-located with m in-face
        double wf = B.w[fb] * B.w[fc];
        T qp[NV], qm[NV];
        trace(D, acc, e, d, s, fb, fc, qp);
        int nb = D.neighbor(e, d, s);
        trace(D, acc, nb, d, -s, fb, fc, qm);
        for (int k = 0; k < NV; ++k) {
          T qhat = 0.5 * (qp[k] + qm[k]);
          s3[d][k] += (D.Jf * wf * phin * (double)s) * qhat;
        }
      }
    }
    double wm = B.w[cm[0]] * B.w[cm[1]] * B.w[cm[2]];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < NV; ++k) g[((size_t)m * 3 + a) * NV + k] = s3[a][k] / (D.J * wm);
  }
}

// Residual rows of element e (eq. DGSEMsystem:1 plus the time term).  gsrc(e') must
// return the lifted gradient array of element e'.
template <class T, class A, class G>
void elem_residual(const Disc& D, const A& acc, int e, const G& gsrc,
                   const double* Qs, const double* Qsm1, T* R /* nn*NV */) {
  const Basis& B = D.B;
  const int p = D.p;
  const size_t gsz = (size_t)D.nn * 3 * NV;
  std::vector<T> g(gsz);
  { const T* gp = gsrc(e); for (size_t x = 0; x < gsz; ++x) g[x] = gp[x]; }
  // fluxes F_d = f^a_d - f^nu_d at every node
  std::vector<T> F((size_t)D.nn * 3 * NV);
  for (int m = 0; m < D.nn; ++m) {
    T q[NV];
    for (int k = 0; k < NV; ++k) q[k] = acc.get(e, m, k);
    for (int d = 0; d < 3; ++d) {
      T fa[NV], fv[NV];
      adv_flux(D.P, q, d, fa);
      visc_flux(D.P, q, &g[(size_t)m * 3 * NV], d, fv);
      for (int k = 0; k < NV; ++k) F[((size_t)m * 3 + d) * NV + k] = fa[k] - fv[k];
    }
  }
  for (int j = 0; j < D.nn; ++j) {
    int cj[3]; D.coords(j, cj);
    double wj = B.w[cj[0]] * B.w[cj[1]] * B.w[cj[2]];
    T r[NV];
    for (int k = 0; k < NV; ++k) r[k] = T(0.0);
    if (D.P.with_time) {
      for (int k = 0; k < NV; ++k) {
        size_t idx = ((size_t)e * D.nn + j) * NV + k;
        T qj = acc.get(e, j, k);
        if (D.P.bdf == 2)
          r[k] = (D.J * wj / D.P.dt) * (1.5 * qj - 2.0 * Qs[idx] + 0.5 * Qsm1[idx]);
        else
          r[k] = (D.J * wj / D.P.dt) * (qj - Qs[idx]);
      }
    }
    // volume: - sum_m J w_m F(m) . grad phi_j(x_m)
    for (int m = 0; m < D.nn; ++m) {
      int cm[3]; D.coords(m, cm);
      double e0 = B.ell[cj[0] * p + cm[0]], e1 = B.ell[cj[1] * p + cm[1]], e2 = B.ell[cj[2] * p + cm[2]];
      double d0 = B.dell[cj[0] * p + cm[0]], d1 = B.dell[cj[1] * p + cm[1]], d2 = B.dell[cj[2] * p + cm[2]];
      double gp[3] = {D.dx * d0 * e1 * e2, D.dx * e0 * d1 * e2, D.dx * e0 * e1 * d2};
      if (gp[0] == 0.0 && gp[1] == 0.0 && gp[2] == 0.0) continue;
      double wm = B.w[cm[0]] * B.w[cm[1]] * B.w[cm[2]];
      for (int d = 0; d < 3; ++d) {
        if (gp[d] == 0.0) continue;
        for (int k = 0; k < NV; ++k) r[k] -= (D.J * wm * gp[d]) * F[((size_t)m * 3 + d) * NV + k];
      }
    }
    // surface: int fhat phi_j dS
    for (int d = 0; d < 3; ++d) {
      int db = (d + 1) % 3, dc = (d + 2) % 3;
      for (int s = -1; s <= 1; s += 2) {
        const std::vector<double>& edge = (s > 0) ? B.eR : B.eL;
        const std::vector<double>& edgeo = (s > 0) ? B.eL : B.eR;
        double phin = edge[cj[d]];
        if (phin == 0.0) continue;
        int fb = cj[db], fc = cj[dc];
        double wf = B.w[fb] * B.w[fc];
        int nb = D.neighbor(e, d, s);
        T qp[NV], qm[NV];
        trace(D, acc, e, d, s, fb, fc, qp);
        trace(D, acc, nb, d, -s, fb, fc, qm);
        T gpl[3 * NV], gmi[3 * NV];
        double sigma = 0.0;
        if (D.P.visc_flux == 1) {
          // interior penalty: the average of the viscous fluxes at the local gradients of
          // both sides, minus sigma times the jump of q (penalising q+ - q-)
          trace_grad(D, acc, e, d, s, fb, fc, gpl);
          trace_grad(D, acc, nb, d, -s, fb, fc, gmi);
          sigma = ip_sigma(D.P, D.N, D.h);
        } else {
          // BR1: lifted gradients are nodal polynomials too; trace them the same way
          for (int x = 0; x < 3 * NV; ++x) { gpl[x] = T(0.0); gmi[x] = T(0.0); }
          const T* gn = gsrc(nb);
          for (int a = 0; a < p; ++a) {
            int c[3]; c[db] = fb; c[dc] = fc; c[d] = a;
            int m = D.node(c[0], c[1], c[2]);
            if (edge[a] != 0.0)
              for (int x = 0; x < 3 * NV; ++x) gpl[x] += edge[a] * g[(size_t)m * 3 * NV + x];
            if (edgeo[a] != 0.0)
              for (int x = 0; x < 3 * NV; ++x) gmi[x] += edgeo[a] * gn[(size_t)m * 3 * NV + x];
          }
        }
        T fa[NV], fvp[NV], fvm[NV];
        num_flux_adv(D.P, qp, qm, d, s, fa);
        visc_flux(D.P, qp, gpl, d, fvp);
        visc_flux(D.P, qm, gmi, d, fvm);
        for (int k = 0; k < NV; ++k) {
          T fhat = fa[k] - 0.5 * (double)s * (fvp[k] + fvm[k]) + sigma * (qp[k] - qm[k]);
          r[k] += (D.Jf * wf * phin) * fhat;
        }
      }
    }
    for (int k = 0; k < NV; ++k) R[(size_t)j * NV + k] = r[k];
  }
}

// Distinct elements of the 3x3x3 block of elements around e (periodic wrap).
int neighborhood(const Disc& D, int e, int* out) {
  int c[3]; D.ecoords(e, c); int cnt = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dxx = -1; dxx <= 1; ++dxx) {
        int x = D.elem(c[0] + dxx, c[1] + dy, c[2] + dz);
        bool seen = false;
        for (int i = 0; i < cnt; ++i) seen |= (out[i] == x);
        if (!seen) out[cnt++] = x;
      }
  return cnt;
}

// Derivatives of the rows of the elements rows_e[0..nrow) with respect to the five
// variables of node r of element c: out[i] holds dR_{rows_e[i]}/dq_{c,r} as duals.
void column_node(const Disc& D, const double* Q, const std::vector<double>& g0,
                 int c, int r, const int* rows_e, int nrow,
                 std::vector<std::vector<Dual<5>>>& out) {
  using T = Dual<5>;
  Access<T> acc{&D, Q}; acc.se = c; acc.sn = r;
  // Lifted gradients depend on the seed only in c and its face neighbours.
  int N1[7]; int cnt = 0; N1[cnt++] = c;
  for (int d = 0; d < 3; ++d)
    for (int s = -1; s <= 1; s += 2) {
      int nb = D.neighbor(c, d, s); bool seen = false;
      for (int i = 0; i < cnt; ++i) seen |= (N1[i] == nb);
      if (!seen) N1[cnt++] = nb;
    }
  const size_t gsz = (size_t)D.nn * 3 * NV;
  std::vector<T> gseed((size_t)cnt * gsz);
  for (int i = 0; i < cnt; ++i) lifting<T>(D, acc, N1[i], gseed.data() + (size_t)i * gsz);
  // Unseeded elements carry the base gradients with zero derivative.  elem_residual
  // copies its own element's gradients first and then asks for one neighbour at a
  // time, so one promotion buffer suffices.
  std::vector<T> slot(gsz);
  auto gsrc = [&](int ee) -> const T* {
    for (int t = 0; t < cnt; ++t) if (N1[t] == ee) return gseed.data() + (size_t)t * gsz;
    for (size_t x = 0; x < gsz; ++x) slot[x] = T(g0[(size_t)ee * gsz + x]);
    return slot.data();
  };
  out.resize(nrow);
  for (int i = 0; i < nrow; ++i) {
    out[i].resize((size_t)D.nn * NV);
    elem_residual<T>(D, acc, rows_e[i], gsrc, Q, Q, out[i].data());
  }
}

}  // namespace

extern "C" {

int or_gl(int N, double* xi, double* w, double* Dm) {
  if (N < 1 || N > 16) return 1;
  Basis b = make_basis(N);
  int p = N + 1;
  for (int i = 0; i < p; ++i) { xi[i] = b.xi[i]; w[i] = b.w[i]; }
  if (Dm)
    for (int a = 0; a < p; ++a)
      for (int i = 0; i < p; ++i) Dm[a * p + i] = b.dell[i * p + a];  // D[a][i] = l_i'(xi_a)
  return 0;
}

int or_lagrange(int N, int i, double x, double* value, double* deriv) {
  if (N < 1 || i < 0 || i > N) return 1;
  Basis b = make_basis(N);
  *value = lagrange(b.xi, i, x);
  *deriv = lagrange_deriv(b.xi, i, x);
  return 0;
}

// Lifted gradients of every element: g[K][nn][3][5].
int or_lifting(const or_params* P, const double* Q, double* g) {
  Disc D(*P);
  Access<double> acc{&D, Q};
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < D.K; ++e) lifting<double>(D, acc, e, g + (size_t)e * D.nn * 3 * NV);
  return 0;
}

// Residual R(Q) of every element: R[K][nn][5].
int or_residual(const or_params* P, const double* Q, const double* Qs, const double* Qsm1, double* R) {
  Disc D(*P);
  Access<double> acc{&D, Q};
  std::vector<double> g((size_t)D.K * D.nn * 3 * NV);
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < D.K; ++e) lifting<double>(D, acc, e, g.data() + (size_t)e * D.nn * 3 * NV);
  auto gsrc = [&](int ee) { return (const double*)(g.data() + (size_t)ee * D.nn * 3 * NV); };
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < D.K; ++e)
    elem_residual<double>(D, acc, e, gsrc, Qs, Qsm1 ? Qsm1 : Qs, R + (size_t)e * D.nn * NV);
  return 0;
}

// Jacobian-vector product y = (dR/dQ) x with a one-direction dual.
int or_jvp(const or_params* P, const double* Q, const double* x, double* y) {
  Disc D(*P);
  using T = Dual<1>;
  Access<T> acc{&D, Q}; acc.dir = x;
  std::vector<T> g((size_t)D.K * D.nn * 3 * NV);
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < D.K; ++e) lifting<T>(D, acc, e, g.data() + (size_t)e * D.nn * 3 * NV);
  auto gsrc = [&](int ee) { return (const T*)(g.data() + (size_t)ee * D.nn * 3 * NV); };
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < D.K; ++e) {
    std::vector<T> R((size_t)D.nn * NV);
    elem_residual<T>(D, acc, e, gsrc, Q, Q, R.data());
    for (size_t i = 0; i < R.size(); ++i) y[(size_t)e * D.nn * NV + i] = R[i].d[0];
  }
  return 0;
}

// Full Jacobian in COO form: rows/cols are global dof indices (e*nn + node)*5 + var.
// Returns the number of non-zeros; nothing beyond cap is written.
long or_jacobian_coo(const or_params* P, const double* Q, long cap, int* rows, int* cols, double* vals) {
  Disc D(*P);
  std::vector<double> g0((size_t)D.K * D.nn * 3 * NV);
  or_lifting(P, Q, g0.data());
  std::vector<std::vector<long>> R_(D.K), C_(D.K);
  std::vector<std::vector<double>> V_(D.K);
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < D.K; ++c) {
    int nbh[27]; int cnt = neighborhood(D, c, nbh);
    std::vector<std::vector<Dual<5>>> Rr;
    for (int r = 0; r < D.nn; ++r) {
      column_node(D, Q, g0, c, r, nbh, cnt, Rr);
      for (int i = 0; i < cnt; ++i) {
        int e = nbh[i];
        for (int j = 0; j < D.nn; ++j)
          for (int v = 0; v < NV; ++v)
            for (int k = 0; k < NV; ++k) {
              double a = Rr[i][(size_t)j * NV + v].d[k];
              if (a == 0.0) continue;
              R_[c].push_back(((long)e * D.nn + j) * NV + v);
              C_[c].push_back(((long)c * D.nn + r) * NV + k);
              V_[c].push_back(a);
            }
      }
    }
  }
  long total = 0;
  for (int c = 0; c < D.K; ++c)
    for (size_t i = 0; i < R_[c].size(); ++i) {
      if (total < cap) { rows[total] = (int)R_[c][i]; cols[total] = (int)C_[c][i]; vals[total] = V_[c][i]; }
      ++total;
    }
  return total;
}

// Rows of element e only: for each distinct element c of the 3x3x3 neighbourhood,
// the dense block dR_e/dQ_c (nn*5 x nn*5, natural order, row-major).
// Returns the number of blocks written (<= 27); col_elems receives their elements.
int or_jacobian_elem_rows(const or_params* P, const double* Q, int e, int* col_elems, double* blocks) {
  Disc D(*P);
  std::vector<double> g0((size_t)D.K * D.nn * 3 * NV);
  or_lifting(P, Q, g0.data());
  int nbh[27]; int cnt = neighborhood(D, e, nbh);
  const int ne = D.nn * NV;
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < cnt; ++i) {
    int c = nbh[i];
    col_elems[i] = c;
    double* blk = blocks + (size_t)i * ne * ne;
    std::vector<std::vector<Dual<5>>> Rr;
    for (int r = 0; r < D.nn; ++r) {
      column_node(D, Q, g0, c, r, &e, 1, Rr);
      for (int j = 0; j < D.nn; ++j)
        for (int v = 0; v < NV; ++v)
          for (int k = 0; k < NV; ++k)
            blk[(size_t)(j * NV + v) * ne + r * NV + k] = Rr[0][(size_t)j * NV + v].d[k];
    }
  }
  return cnt;
}

// The fluxes on their own, for the flux pins.
int or_num_flux(const or_params* P, const double* qL, const double* qR, int d, int s, double* fa) {
  num_flux_adv<double>(*P, qL, qR, d, s, fa);
  return 0;
}
int or_phys_flux(const or_params* P, const double* q, const double* g, int d, double* fa, double* fv) {
  adv_flux<double>(*P, q, d, fa);
  visc_flux<double>(*P, q, g, d, fv);
  return 0;
}
int or_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"

// ============================================================ meshes of mixed order
// Element e carries its own order N_e (periodic n^3 mesh, same Cartesian cells).  A face
// between two orders is a mortar (the survey's reading of an unstated case): both
// traces, of the state and of the lifted gradient, are interpolated to the Gauss-Lobatto
// nodes of order M = max(N_L, N_R) on the face; qhat (BR1) and fhat are formed there
// point by point, exactly as on a conforming face, and each side takes the L2 projection
// of them onto its own face polynomials (degree N_e in each in-face direction), with a
// Gauss rule of M + 1 points (exact to degree 2M + 1).  The element's weak form then
// integrates the projected values with its own Gauss-Lobatto face quadrature.  Faces
// between equal orders are conforming unless force_mortar is set; the mortar of equal
// orders reduces to the conforming face, which is what the pins check.
namespace {

struct MDisc {
  or_params P;
  int n, K, force_mortar;
  double h, J, Jf, dx;
  std::vector<int> ord, off;  // order and first node of every element
  std::vector<Basis> B;       // B[N], N = 1..7
  MDisc(const or_params& pp, const int* orders, int fm) : P(pp), force_mortar(fm) {
    n = P.n; K = n * n * n;
    h = P.L / n; J = std::pow(0.5 * h, 3); Jf = std::pow(0.5 * h, 2); dx = 2.0 / h;
    ord.assign(orders, orders + K);
    off.assign(K + 1, 0);
    for (int e = 0; e < K; ++e) off[e + 1] = off[e] + (ord[e] + 1) * (ord[e] + 1) * (ord[e] + 1);
    B.resize(8);
    for (int N = 1; N <= 7; ++N) B[N] = make_basis(N);
  }
  int p(int e) const { return ord[e] + 1; }
  int nn(int e) const { return p(e) * p(e) * p(e); }
  int node(int e, int i, int j, int k) const { const int q = p(e); return i + q * (j + q * k); }
  void coords(int e, int m, int c[3]) const { const int q = p(e); c[0] = m % q; c[1] = (m / q) % q; c[2] = m / (q * q); }
  int elem(int ex, int ey, int ez) const {
    ex = ((ex % n) + n) % n; ey = ((ey % n) + n) % n; ez = ((ez % n) + n) % n;
    return ex + n * (ey + n * ez);
  }
  int neighbor(int e, int d, int s) const {
    int c[3] = {e % n, (e / n) % n, e / (n * n)}; c[d] += s; return elem(c[0], c[1], c[2]);
  }
  size_t nodes() const { return (size_t)off[K]; }
};

template <class T> struct IsDual { static constexpr bool v = false; };
template <int ND> struct IsDual<Dual<ND>> { static constexpr bool v = true; };

// Ragged state accessor, with the same seeding rules as Access.
template <class T>
struct MAccess {
  const MDisc* D; const double* Q; int se = -1, sn = -1; const double* dir = nullptr;
  T get(int e, int m, int k) const {
    const size_t i = ((size_t)D->off[e] + m) * NV + k;
    T t(Q[i]);
    if constexpr (IsDual<T>::v) {
      if (dir) t.d[0] = dir[i];
      else if (e == se && m == sn && k < (int)(sizeof(t.d) / sizeof(double))) t.d[k] = 1.0;
    }
    return t;
  }
};

// Gauss-Legendre points and weights (Newton on P_m from the Chebyshev guesses).
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0); w.assign(m, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < m; ++i) {
    double z = -std::cos(pi * (i + 0.75) / (m + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P; legendre(m, z, P, dP, d2P);
      const double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP, d2P; legendre(m, z, P, dP, d2P);
    x[i] = z; w[i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

// 1-D transfer matrices of a mortar: interpolation from order a to order b nodes
// (rows: b nodes) and L2 projection from order M mortar nodes to order Ne (rows: Ne nodes).
struct Mortar1D {
  std::vector<double> interp[8][8];  // interp[a][b][(b nodes) x (a+1)]
  std::vector<double> proj[8][8];    // proj[M][Ne][(Ne+1) x (M+1)]
  explicit Mortar1D(const std::vector<Basis>& B) {
    for (int a = 1; a <= 7; ++a)
      for (int b = 1; b <= 7; ++b) {
        interp[a][b].assign((size_t)(b + 1) * (a + 1), 0.0);
        for (int g = 0; g <= b; ++g)
          for (int i = 0; i <= a; ++i) interp[a][b][(size_t)g * (a + 1) + i] = lagrange(B[a].xi, i, B[b].xi[g]);
      }
    for (int M = 1; M <= 7; ++M)
      for (int Ne = 1; Ne <= M; ++Ne) {
        std::vector<double> gx, gw;
        gauss_legendre(M + 1, gx, gw);
        const int pe = Ne + 1, pm = M + 1;
        std::vector<double> Mm((size_t)pe * pe, 0.0), Bm((size_t)pe * pm, 0.0);
        for (size_t q = 0; q < gx.size(); ++q) {
          std::vector<double> le(pe), lm(pm);
          for (int i = 0; i < pe; ++i) le[i] = lagrange(B[Ne].xi, i, gx[q]);
          for (int i = 0; i < pm; ++i) lm[i] = lagrange(B[M].xi, i, gx[q]);
          for (int i = 0; i < pe; ++i) {
            for (int j = 0; j < pe; ++j) Mm[(size_t)i * pe + j] += gw[q] * le[i] * le[j];
            for (int j = 0; j < pm; ++j) Bm[(size_t)i * pm + j] += gw[q] * le[i] * lm[j];
          }
        }
        // proj = Mm^-1 Bm by Gauss-Jordan on the small symmetric positive mass matrix
        std::vector<double> A = Mm, X = Bm;
        for (int c = 0; c < pe; ++c) {
          int piv = c;
          for (int r = c + 1; r < pe; ++r)
            if (std::fabs(A[(size_t)r * pe + c]) > std::fabs(A[(size_t)piv * pe + c])) piv = r;
          for (int j = 0; j < pe; ++j) std::swap(A[(size_t)c * pe + j], A[(size_t)piv * pe + j]);
          for (int j = 0; j < pm; ++j) std::swap(X[(size_t)c * pm + j], X[(size_t)piv * pm + j]);
          const double d = A[(size_t)c * pe + c];
          for (int j = 0; j < pe; ++j) A[(size_t)c * pe + j] /= d;
          for (int j = 0; j < pm; ++j) X[(size_t)c * pm + j] /= d;
          for (int r = 0; r < pe; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * pe + c];
            for (int j = 0; j < pe; ++j) A[(size_t)r * pe + j] -= f * A[(size_t)c * pe + j];
            for (int j = 0; j < pm; ++j) X[(size_t)r * pm + j] -= f * X[(size_t)c * pm + j];
          }
        }
        proj[M][Ne] = X;
      }
  }
};

// out[a][b] = sum_{i,j} T[a][i] T[b][j] in[i][j] for nc components per point
// (T rows: ro, cols: ci).
template <class T>
void tensor2(const std::vector<double>& Tm, int ro, int ci, const T* in, T* out, int nc) {
  std::vector<T> tmp((size_t)ro * ci * nc, T(0.0));
  for (int a = 0; a < ro; ++a)
    for (int i = 0; i < ci; ++i) {
      const double t = Tm[(size_t)a * ci + i];
      if (t == 0.0) continue;
      for (int j = 0; j < ci; ++j)
        for (int k = 0; k < nc; ++k) tmp[((size_t)a * ci + j) * nc + k] += t * in[((size_t)i * ci + j) * nc + k];
    }
  for (size_t x = 0; x < (size_t)ro * ro * nc; ++x) out[x] = T(0.0);
  for (int b = 0; b < ro; ++b)
    for (int j = 0; j < ci; ++j) {
      const double t = Tm[(size_t)b * ci + j];
      if (t == 0.0) continue;
      for (int a = 0; a < ro; ++a)
        for (int k = 0; k < nc; ++k) out[((size_t)a * ro + b) * nc + k] += t * tmp[((size_t)a * ci + j) * nc + k];
    }
}

// Face values of element e on face (d, s): the state (5) and, with g, the lifted gradient
// (15) at its face nodes [fb + p fc], fb / fc the in-face indices along (d+1)%3, (d+2)%3.
template <class T, class A>
void face_values(const MDisc& D, const A& acc, int e, int d, int s, const T* g, T* q, T* gf) {
  const int p = D.p(e), N = D.ord[e], db = (d + 1) % 3, dc = (d + 2) % 3;
  for (int fc = 0; fc < p; ++fc)
    for (int fb = 0; fb < p; ++fb) {
      int c[3]; c[d] = s > 0 ? N : 0; c[db] = fb; c[dc] = fc;
      const int m = D.node(e, c[0], c[1], c[2]);
      for (int k = 0; k < NV; ++k) q[((size_t)fc * p + fb) * NV + k] = acc.get(e, m, k);
      if (g && gf)
        for (int x = 0; x < 3 * NV; ++x) gf[((size_t)fc * p + fb) * 3 * NV + x] = g[(size_t)m * 3 * NV + x];
    }
}

// qhat (lifting) or fhat (with gradients) at element e's face nodes on face (d, s).
template <class T, class A>
void face_flux(const MDisc& D, const Mortar1D& Mo, const A& acc, int e, int d, int s,
               const std::vector<std::vector<T>>* G, bool want_f, T* out /* p*p*NV */) {
  const int nb = D.neighbor(e, d, s);
  const int Ne = D.ord[e], Nn = D.ord[nb], pe = Ne + 1, pn = Nn + 1;
  const bool mortar = Ne != Nn || D.force_mortar;
  const int M = std::max(Ne, Nn), pm = M + 1;
  std::vector<T> qp((size_t)pe * pe * NV), qm((size_t)pn * pn * NV);
  std::vector<T> gp, gm;
  if (want_f) { gp.resize((size_t)pe * pe * 3 * NV); gm.resize((size_t)pn * pn * 3 * NV); }
  face_values<T>(D, acc, e, d, s, want_f ? (*G)[e].data() : nullptr, qp.data(), want_f ? gp.data() : nullptr);
  face_values<T>(D, acc, nb, d, -s, want_f ? (*G)[nb].data() : nullptr, qm.data(), want_f ? gm.data() : nullptr);
  // values on the mortar points (the element's own face nodes when conforming)
  const int pt = mortar ? pm : pe;
  std::vector<T> QP, QM, GP, GM;
  if (mortar) {
    QP.resize((size_t)pm * pm * NV); QM.resize((size_t)pm * pm * NV);
    tensor2<T>(Mo.interp[Ne][M], pm, pe, qp.data(), QP.data(), NV);
    tensor2<T>(Mo.interp[Nn][M], pm, pn, qm.data(), QM.data(), NV);
    if (want_f) {
      GP.resize((size_t)pm * pm * 3 * NV); GM.resize((size_t)pm * pm * 3 * NV);
      tensor2<T>(Mo.interp[Ne][M], pm, pe, gp.data(), GP.data(), 3 * NV);
      tensor2<T>(Mo.interp[Nn][M], pm, pn, gm.data(), GM.data(), 3 * NV);
    }
  } else {
    QP = qp; QM = qm; GP = gp; GM = gm;
  }
  std::vector<T> F((size_t)pt * pt * NV);
  for (int x = 0; x < pt * pt; ++x) {
    const T* a = &QP[(size_t)x * NV];
    const T* b = &QM[(size_t)x * NV];
    if (!want_f) {
      for (int k = 0; k < NV; ++k) F[(size_t)x * NV + k] = 0.5 * (a[k] + b[k]);
    } else {
      T fa[NV], fvp[NV], fvm[NV];
      num_flux_adv(D.P, a, b, d, s, fa);
      visc_flux(D.P, a, &GP[(size_t)x * 3 * NV], d, fvp);
      visc_flux(D.P, b, &GM[(size_t)x * 3 * NV], d, fvm);
      for (int k = 0; k < NV; ++k) F[(size_t)x * NV + k] = fa[k] - 0.5 * (double)s * (fvp[k] + fvm[k]);
    }
  }
  if (mortar) tensor2<T>(Mo.proj[M][Ne], pe, pm, F.data(), out, NV);
  else for (size_t x = 0; x < F.size(); ++x) out[x] = F[x];
}

// Lifted gradient of element e (as `lifting`, with the face qhat of face_flux).
template <class T, class A>
void mlifting(const MDisc& D, const Mortar1D& Mo, const A& acc, int e, T* g) {
  const Basis& B = D.B[D.ord[e]];
  const int p = D.p(e), nn = D.nn(e);
  std::vector<T> qh[6];
  for (int f = 0; f < 6; ++f) {
    qh[f].resize((size_t)p * p * NV);
    face_flux<T>(D, Mo, acc, e, f / 2, (f & 1) ? 1 : -1, nullptr, false, qh[f].data());
  }
  for (int m = 0; m < nn; ++m) {
    int cm[3]; D.coords(e, m, cm);
    T s3[3][NV];
    for (int a = 0; a < 3; ++a) for (int k = 0; k < NV; ++k) s3[a][k] = T(0.0);
    for (int nidx = 0; nidx < nn; ++nidx) {
      int cn[3]; D.coords(e, nidx, cn);
      const double wn = B.w[cn[0]] * B.w[cn[1]] * B.w[cn[2]];
      const double e0 = B.ell[cm[0] * p + cn[0]], e1 = B.ell[cm[1] * p + cn[1]], e2 = B.ell[cm[2] * p + cn[2]];
      const double d0 = B.dell[cm[0] * p + cn[0]], d1 = B.dell[cm[1] * p + cn[1]], d2 = B.dell[cm[2] * p + cn[2]];
      const double gp[3] = {D.dx * d0 * e1 * e2, D.dx * e0 * d1 * e2, D.dx * e0 * e1 * d2};
      for (int k = 0; k < NV; ++k) {
        const T qn = acc.get(e, nidx, k);
        for (int a = 0; a < 3; ++a)
          if (gp[a] != 0.0) s3[a][k] -= (D.J * wn * gp[a]) * qn;
      }
    }
    for (int d = 0; d < 3; ++d) {
      const int db = (d + 1) % 3, dc = (d + 2) % 3;
      for (int s = -1; s <= 1; s += 2) {
        const double phin = ((s > 0) ? B.eR : B.eL)[cm[d]];
        if (phin == 0.0) continue;
        const int fb = cm[db], fc = cm[dc];
        const double wf = B.w[fb] * B.w[fc];
        const T* qhat = &qh[2 * d + (s > 0 ? 1 : 0)][((size_t)fc * p + fb) * NV];
        for (int k = 0; k < NV; ++k) s3[d][k] += (D.Jf * wf * phin * (double)s) * qhat[k];
      }
    }
    const double wm = B.w[cm[0]] * B.w[cm[1]] * B.w[cm[2]];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < NV; ++k) g[((size_t)m * 3 + a) * NV + k] = s3[a][k] / (D.J * wm);
  }
}

// Residual rows of element e (as elem_residual, with the face fhat of face_flux).
template <class T, class A>
void melem_residual(const MDisc& D, const Mortar1D& Mo, const A& acc, int e, const std::vector<std::vector<T>>& G,
                    const double* Qs, const double* Qsm1, T* R) {
  const Basis& B = D.B[D.ord[e]];
  const int p = D.p(e), nn = D.nn(e);
  const std::vector<T>& g = G[e];
  std::vector<T> F((size_t)nn * 3 * NV);
  for (int m = 0; m < nn; ++m) {
    T q[NV];
    for (int k = 0; k < NV; ++k) q[k] = acc.get(e, m, k);
    for (int d = 0; d < 3; ++d) {
      T fa[NV], fv[NV];
      adv_flux(D.P, q, d, fa);
      visc_flux(D.P, q, &g[(size_t)m * 3 * NV], d, fv);
      for (int k = 0; k < NV; ++k) F[((size_t)m * 3 + d) * NV + k] = fa[k] - fv[k];
    }
  }
  std::vector<T> fh[6];
  for (int f = 0; f < 6; ++f) {
    fh[f].resize((size_t)p * p * NV);
    face_flux<T>(D, Mo, acc, e, f / 2, (f & 1) ? 1 : -1, &G, true, fh[f].data());
  }
  for (int j = 0; j < nn; ++j) {
    int cj[3]; D.coords(e, j, cj);
    const double wj = B.w[cj[0]] * B.w[cj[1]] * B.w[cj[2]];
    T r[NV];
    for (int k = 0; k < NV; ++k) r[k] = T(0.0);
    if (D.P.with_time) {
      for (int k = 0; k < NV; ++k) {
        const size_t idx = ((size_t)D.off[e] + j) * NV + k;
        const T qj = acc.get(e, j, k);
        if (D.P.bdf == 2) r[k] = (D.J * wj / D.P.dt) * (1.5 * qj - 2.0 * Qs[idx] + 0.5 * Qsm1[idx]);
        else r[k] = (D.J * wj / D.P.dt) * (qj - Qs[idx]);
      }
    }
    for (int m = 0; m < nn; ++m) {
      int cm[3]; D.coords(e, m, cm);
      const double e0 = B.ell[cj[0] * p + cm[0]], e1 = B.ell[cj[1] * p + cm[1]], e2 = B.ell[cj[2] * p + cm[2]];
      const double d0 = B.dell[cj[0] * p + cm[0]], d1 = B.dell[cj[1] * p + cm[1]], d2 = B.dell[cj[2] * p + cm[2]];
      const double gp[3] = {D.dx * d0 * e1 * e2, D.dx * e0 * d1 * e2, D.dx * e0 * e1 * d2};
      const double wm = B.w[cm[0]] * B.w[cm[1]] * B.w[cm[2]];
      for (int d = 0; d < 3; ++d) {
        if (gp[d] == 0.0) continue;
        for (int k = 0; k < NV; ++k) r[k] -= (D.J * wm * gp[d]) * F[((size_t)m * 3 + d) * NV + k];
      }
    }
    for (int d = 0; d < 3; ++d) {
      const int db = (d + 1) % 3, dc = (d + 2) % 3;
      for (int s = -1; s <= 1; s += 2) {
        const double phin = ((s > 0) ? B.eR : B.eL)[cj[d]];
        if (phin == 0.0) continue;
        const int fb = cj[db], fc = cj[dc];
        const double wf = B.w[fb] * B.w[fc];
        const T* fhat = &fh[2 * d + (s > 0 ? 1 : 0)][((size_t)fc * p + fb) * NV];
        for (int k = 0; k < NV; ++k) r[k] += (D.Jf * wf * phin) * fhat[k];
      }
    }
    for (int k = 0; k < NV; ++k) R[(size_t)j * NV + k] = r[k];
  }
}

// The whole residual of a mixed-order mesh in type T.
// (Element loops in parallel: every iteration writes its own element's arrays; inside
// the column loop of or_jacobian_mixed the nested regions run on one thread.)
template <class T, class A>
void mresidual(const MDisc& D, const Mortar1D& Mo, const A& acc, const double* Qs, const double* Qsm1, T* R) {
  std::vector<std::vector<T>> G(D.K);
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < D.K; ++e) {
    G[e].resize((size_t)D.nn(e) * 3 * NV);
    mlifting<T>(D, Mo, acc, e, G[e].data());
  }
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < D.K; ++e) melem_residual<T>(D, Mo, acc, e, G, Qs, Qsm1, R + (size_t)D.off[e] * NV);
}

// Meshes of mixed order take BR1 only: the interior-penalty flux is defined here on
// conforming faces.
bool orders_ok(const or_params* P, const int* orders) {
  if (P->visc_flux != 0) return false;
  const int K = P->n * P->n * P->n;
  for (int e = 0; e < K; ++e)
    if (orders[e] < 1 || orders[e] > 7) return false;
  return true;
}

}  // namespace

extern "C" {

// Residual of a mixed-order mesh: Q, Qs, Qsm1, R are flat [sum_e (N_e+1)^3][5] (element by
// element, nodes in natural order).  Returns 1 for an order outside 1..7.
int or_residual_mixed(const or_params* P, const int* orders, int force_mortar, const double* Q, const double* Qs,
                      const double* Qsm1, double* R) {
  if (!orders_ok(P, orders)) return 1;
  MDisc D(*P, orders, force_mortar);
  Mortar1D Mo(D.B);
  MAccess<double> acc{&D, Q};
  mresidual<double>(D, Mo, acc, Qs, Qsm1 ? Qsm1 : Qs, R);
  return 0;
}

// y = (dR/dQ) x on a mixed-order mesh (one-direction dual).
int or_jvp_mixed(const or_params* P, const int* orders, int force_mortar, const double* Q, const double* x,
                 double* y) {
  if (!orders_ok(P, orders)) return 1;
  MDisc D(*P, orders, force_mortar);
  Mortar1D Mo(D.B);
  using T = Dual<1>;
  MAccess<T> acc{&D, Q}; acc.dir = x;
  std::vector<T> R(D.nodes() * NV);
  mresidual<T>(D, Mo, acc, Q, Q, R.data());
  for (size_t i = 0; i < R.size(); ++i) y[i] = R[i].d[0];
  return 0;
}

// Sparse Jacobian of a mixed-order mesh in COO form (global dof rows / columns, flat
// ragged order).  For each column node only the rows of the 3x3x3 block of elements
// around it are evaluated: the seed changes the lifted gradients of its own element and
// of its face neighbours only, and the other gradients those rows read are the base
// ones.  Returns the number of non-zeros; nothing beyond cap is written.
long or_jacobian_mixed_coo(const or_params* P, const int* orders, int force_mortar, const double* Q, long cap,
                           int* rows, int* cols, double* vals) {
  if (!orders_ok(P, orders)) return -1;
  MDisc D(*P, orders, force_mortar);
  Mortar1D Mo(D.B);
  std::vector<std::vector<double>> G0(D.K);
  {
    MAccess<double> acc0{&D, Q};
#pragma omp parallel for schedule(dynamic)
    for (int e = 0; e < D.K; ++e) {
      G0[e].resize((size_t)D.nn(e) * 3 * NV);
      mlifting<double>(D, Mo, acc0, e, G0[e].data());
    }
  }
  std::vector<std::vector<long>> R_(D.K), C_(D.K);
  std::vector<std::vector<double>> V_(D.K);
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < D.K; ++c) {
    using T = Dual<5>;
    // rows: the distinct elements of the 3x3x3 block around c
    std::vector<int> nbh;
    const int cx = c % D.n, cy = (c / D.n) % D.n, cz = c / (D.n * D.n);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dxx = -1; dxx <= 1; ++dxx) {
          const int x = D.elem(cx + dxx, cy + dy, cz + dz);
          if (std::find(nbh.begin(), nbh.end(), x) == nbh.end()) nbh.push_back(x);
        }
    // gradients those rows read: their elements and face neighbours
    std::vector<int> ring = nbh;
    for (int e : nbh)
      for (int f = 0; f < 6; ++f) {
        const int x = D.neighbor(e, f / 2, (f & 1) ? 1 : -1);
        if (std::find(ring.begin(), ring.end(), x) == ring.end()) ring.push_back(x);
      }
    std::vector<int> seeded(1, c);
    for (int f = 0; f < 6; ++f) {
      const int x = D.neighbor(c, f / 2, (f & 1) ? 1 : -1);
      if (std::find(seeded.begin(), seeded.end(), x) == seeded.end()) seeded.push_back(x);
    }
    std::vector<std::vector<T>> G(D.K);
    for (int x : ring) G[x].resize((size_t)D.nn(x) * 3 * NV);
    std::vector<T> Rb;
    for (int r = 0; r < D.nn(c); ++r) {
      MAccess<T> acc{&D, Q}; acc.se = c; acc.sn = r;
      for (int x : ring) {
        if (std::find(seeded.begin(), seeded.end(), x) != seeded.end()) {
          mlifting<T>(D, Mo, acc, x, G[x].data());
        } else {
          for (size_t i = 0; i < G[x].size(); ++i) G[x][i] = T(G0[x][i]);
        }
      }
      const long col0 = ((long)D.off[c] + r) * NV;
      for (int e : nbh) {
        Rb.assign((size_t)D.nn(e) * NV, T(0.0));
        melem_residual<T>(D, Mo, acc, e, G, Q, Q, Rb.data());
        for (int j = 0; j < D.nn(e); ++j)
          for (int v = 0; v < NV; ++v)
            for (int k = 0; k < NV; ++k) {
              const double a = Rb[(size_t)j * NV + v].d[k];
              if (a == 0.0) continue;
              R_[c].push_back(((long)D.off[e] + j) * NV + v);
              C_[c].push_back(col0 + k);
              V_[c].push_back(a);
            }
      }
    }
  }
  long total = 0;
  for (int c = 0; c < D.K; ++c)
    for (size_t i = 0; i < R_[c].size(); ++i) {
      if (total < cap) { rows[total] = (int)R_[c][i]; cols[total] = (int)C_[c][i]; vals[total] = V_[c][i]; }
      ++total;
    }
  return total;
}

// Rows of element e only (mixed orders): for each distinct element c of the 3x3x3 block
// around e, the dense block dR_e/dQ_c ((N_e+1)^3 5 x (N_c+1)^3 5, row-major), written one
// after the other into blocks; col_elems receives the elements.  Returns their number.
int or_jacobian_mixed_elem_rows(const or_params* P, const int* orders, int force_mortar, const double* Q, int e,
                                int* col_elems, double* blocks) {
  if (!orders_ok(P, orders)) return -1;
  MDisc D(*P, orders, force_mortar);
  Mortar1D Mo(D.B);
  std::vector<int> nbh;
  const int ex = e % D.n, ey = (e / D.n) % D.n, ez = e / (D.n * D.n);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dxx = -1; dxx <= 1; ++dxx) {
        const int x = D.elem(ex + dxx, ey + dy, ez + dz);
        if (std::find(nbh.begin(), nbh.end(), x) == nbh.end()) nbh.push_back(x);
      }
  // gradients row e reads: e and its face neighbours
  std::vector<int> need(1, e);
  for (int f = 0; f < 6; ++f) {
    const int x = D.neighbor(e, f / 2, (f & 1) ? 1 : -1);
    if (std::find(need.begin(), need.end(), x) == need.end()) need.push_back(x);
  }
  std::vector<std::vector<double>> G0(D.K);
  {
    MAccess<double> acc0{&D, Q};
    for (int x : need) {
      G0[x].resize((size_t)D.nn(x) * 3 * NV);
      mlifting<double>(D, Mo, acc0, x, G0[x].data());
    }
  }
  std::vector<size_t> boff(nbh.size() + 1, 0);
  const size_t rows_e = (size_t)D.nn(e) * NV;
  for (size_t i = 0; i < nbh.size(); ++i) boff[i + 1] = boff[i] + rows_e * (size_t)D.nn(nbh[i]) * NV;
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < (int)nbh.size(); ++i) {
    using T = Dual<5>;
    const int c = nbh[i];
    col_elems[i] = c;
    double* blk = blocks + boff[i];
    const size_t cols = (size_t)D.nn(c) * NV;
    std::vector<std::vector<T>> G(D.K);
    for (int x : need) G[x].resize((size_t)D.nn(x) * 3 * NV);
    std::vector<T> Rb(rows_e);
    for (int r = 0; r < D.nn(c); ++r) {
      MAccess<T> acc{&D, Q}; acc.se = c; acc.sn = r;
      for (int x : need) {
        // the seed reaches the gradient of x only if c is x or one of its face neighbours
        bool touched = x == c;
        for (int f = 0; f < 6 && !touched; ++f) touched = D.neighbor(x, f / 2, (f & 1) ? 1 : -1) == c;
        if (touched) mlifting<T>(D, Mo, acc, x, G[x].data());
        else for (size_t t = 0; t < G[x].size(); ++t) G[x][t] = T(G0[x][t]);
      }
      melem_residual<T>(D, Mo, acc, e, G, Q, Q, Rb.data());
      for (size_t row = 0; row < rows_e; ++row)
        for (int k = 0; k < NV; ++k) blk[row * cols + (size_t)r * NV + k] = Rb[row].d[k];
    }
  }
  return (int)nbh.size();
}

// Dense Jacobian of a mixed-order mesh, A[row][col] (dofs x dofs, row-major), column
// node by column node with a five-direction dual (small meshes only).
int or_jacobian_mixed(const or_params* P, const int* orders, int force_mortar, const double* Q, double* A) {
  if (!orders_ok(P, orders)) return 1;
  MDisc D(*P, orders, force_mortar);
  Mortar1D Mo(D.B);
  const size_t dofs = D.nodes() * NV;
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < D.K; ++c) {
    using T = Dual<5>;
    std::vector<T> R(dofs);
    for (int r = 0; r < D.nn(c); ++r) {
      MAccess<T> acc{&D, Q}; acc.se = c; acc.sn = r;
      mresidual<T>(D, Mo, acc, Q, Q, R.data());
      const size_t col0 = ((size_t)D.off[c] + r) * NV;
      for (size_t i = 0; i < dofs; ++i)
        for (int k = 0; k < NV; ++k) A[i * dofs + col0 + k] = R[i].d[k];
    }
  }
  return 0;
}

}  // extern "C"
