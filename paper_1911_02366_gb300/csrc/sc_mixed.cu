// One periodic mesh whose elements carry different polynomial orders (2..6), on the GPU.
//
// The residual is the GL-DGSEM of Sec. 2.1 (eq. DGSEMsystem) with BR1 and the Roe or
// local Lax-Friedrichs flux.  A face between two orders is a mortar (the paper does not
// treat uneven orders): the traces of both sides, state and lifted gradient, are
// interpolated to the Gauss-Lobatto nodes of order M = max(N_L, N_R); qhat (BR1) and fhat
// are formed there point by point; each side takes the L2 projection of them onto its own
// face polynomials, computed with the Gauss rule of M + 1 points.  Faces between equal
// orders are conforming (or mortars when force_mortar is set).
//
// Every evaluation runs in one scalar type T: double for the residual, a one-direction
// dual number for the Jacobian-vector product A x (exact forward-mode derivative; FP64 for
// the refinement residual, FP32 inside the condensed operator of the inner solve), and a
// five-direction dual for the element blocks dR_e/dQ_e (one CTA per element, seeding the
// five variables of one node at a time).
//
// Static condensation (Sec. 2.2, eqs. StaticCondBlock, SC_step1, SC_step2): the own blocks
// are written in FP32 in the layout of the batched condensation, whose grouped kernels
// (A_ii^-1 by Gauss-Jordan, Y^T = A_ib^T A_ii^-T and S_ee = A_bb - A_bi Y on the TF32
// tensor cores, blocked LU of S_ee) run over all elements of every order at once.  The
// condensed operator S x_b = A_bb x_b - A_bi A_ii^-1 A_ib x_b is applied through two
// Jacobian-vector products per application (the couplings across mortar faces are never
// stored), A_ii^-1 from the FP32 inverses; GMRES runs on it, preconditioned by the block
// LU of S_ee, inside FP64 iterative refinement of the global system.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "sc_internal.cuh"

// ------------------------------------------------------------------ dual numbers over R
template <class R, int ND>
struct DualN {
  R v, d[ND];
  __host__ __device__ DualN() : v(R(0)) {
    for (int i = 0; i < ND; ++i) d[i] = R(0);
  }
  __host__ __device__ DualN(double x) : v(R(x)) {
    for (int i = 0; i < ND; ++i) d[i] = R(0);
  }
};
template <class R, int ND>
SC_HD inline DualN<R, ND> operator+(const DualN<R, ND>& a, const DualN<R, ND>& b) {
  DualN<R, ND> r; r.v = a.v + b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class R, int ND>
SC_HD inline DualN<R, ND> operator-(const DualN<R, ND>& a, const DualN<R, ND>& b) {
  DualN<R, ND> r; r.v = a.v - b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class R, int ND>
SC_HD inline DualN<R, ND> operator-(const DualN<R, ND>& a) {
  DualN<R, ND> r; r.v = -a.v;
  for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class R, int ND>
SC_HD inline DualN<R, ND> operator*(const DualN<R, ND>& a, const DualN<R, ND>& b) {
  DualN<R, ND> r; r.v = a.v * b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class R, int ND>
SC_HD inline DualN<R, ND> operator*(const DualN<R, ND>& a, double b) {
  const R c = R(b);
  DualN<R, ND> r; r.v = a.v * c;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * c;
  return r;
}
template <class R, int ND>
SC_HD inline DualN<R, ND> operator*(double b, const DualN<R, ND>& a) { return a * b; }
template <class R, int ND>
SC_HD inline DualN<R, ND> operator+(const DualN<R, ND>& a, double b) { DualN<R, ND> r = a; r.v += R(b); return r; }
template <class R, int ND>
SC_HD inline DualN<R, ND> operator+(double b, const DualN<R, ND>& a) { return a + b; }
template <class R, int ND>
SC_HD inline DualN<R, ND> operator-(const DualN<R, ND>& a, double b) { DualN<R, ND> r = a; r.v -= R(b); return r; }
template <class R, int ND>
SC_HD inline DualN<R, ND> operator-(double b, const DualN<R, ND>& a) { DualN<R, ND> r = -a; r.v += R(b); return r; }
template <class R, int ND>
SC_HD inline DualN<R, ND> recip(const DualN<R, ND>& a) {
  DualN<R, ND> r; r.v = R(1) / a.v;
  const R s = -r.v * r.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * s;
  return r;
}
template <class R, int ND>
SC_HD inline DualN<R, ND> operator/(const DualN<R, ND>& a, const DualN<R, ND>& b) { return a * recip(b); }
template <class R, int ND>
SC_HD inline DualN<R, ND> operator/(const DualN<R, ND>& a, double b) { return a * (1.0 / b); }
template <class R, int ND>
SC_HD inline DualN<R, ND> operator/(double a, const DualN<R, ND>& b) { return recip(b) * a; }
template <class R, int ND>
SC_HD inline DualN<R, ND> dsqrt(const DualN<R, ND>& a) {
  DualN<R, ND> r; r.v = sqrt(a.v);
  const R s = R(0.5) / r.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * s;
  return r;
}
template <class R, int ND>
SC_HD inline double vval(const DualN<R, ND>& a) { return (double)a.v; }

namespace {

using J1 = DualN<double, 1>;  // FP64 Jacobian-vector products
using J1f = DualN<float, 1>;  // FP32 products inside the condensed operator

// A value of type T from a state entry and its direction (the direction is dropped by
// plain doubles); the value and first-direction parts of a T.
template <class T> struct Val;
template <> struct Val<double> {
  SC_HD static double make(double v, double) { return v; }
  SC_HD static double der(double) { return 0.0; }
};
template <class R> struct Val<DualN<R, 1>> {
  SC_HD static DualN<R, 1> make(double v, double dv) { DualN<R, 1> t(v); t.d[0] = R(dv); return t; }
  SC_HD static double der(const DualN<R, 1>& t) { return (double)t.d[0]; }
};

// Basis and mortar tables of the orders 1..7 (index = order).
struct MxTab {
  double w[8][8];        // w[N][i]: Gauss-Lobatto weights
  double D[8][8][8];     // D[N][a][b] = l_b'(xi_a)
  double I[8][8][8][8];  // I[a][b][g][i]: order-a nodal values -> order-b node g (interpolation)
  double P[8][8][8][8];  // P[M][N][i][g]: order-M nodal values -> order-N node i (L2 projection)
  int perm[8][512];      // perm[N][m]: position of node m, interior nodes first, then the boundary ones
};

struct MxMesh {
  int K, n, force_mortar;
  double h, dx, J, Jf, dt, c0;
  const int* ord;   // [K] element orders
  const int* off;   // [K + 1] first node of each element (natural ragged order)
  const int* foff;  // [K + 1] first face node of each element's six faces (6 p_e^2 each)
  const int* nbr;   // [K][6] face neighbours, slot 2 d + (s > 0)
  const MxTab* tab;
};

SC_HD inline int mx_node(const int c[3], int p) { return c[0] + p * (c[1] + p * c[2]); }

// One face f of element e, evaluated by all threads of the CTA: the values of both sides
// at their face nodes (ld(side, x, comp), x = fc * p + fb along ((d+1)%3, (d+2)%3)) are
// interpolated to the mortar points (or used as they are on a conforming face), the point
// function pf(point, own, other, d, s, out[5]) runs there, and the result is projected back onto e's
// face nodes: out[x * 5 + k], x < p_e^2.  sbuf and stmp hold 64 * NC values each.
template <class T, int NC, class LD, class PF>
__device__ void face_eval(const MxMesh& M, int e, int f, const LD& ld, const PF& pf, T* sbuf, T* stmp, T* out) {
  const int d = f >> 1, s = (f & 1) ? 1 : -1;
  const int nb = M.nbr[e * 6 + f];
  const int Ne = M.ord[e], Nn = M.ord[nb], pe = Ne + 1;
  const bool mortar = Ne != Nn || M.force_mortar;
  const int Mo = Ne > Nn ? Ne : Nn, pm = Mo + 1;
  const int pt = mortar ? pm : pe;
  const int t = threadIdx.x;
  T va[NC], vb[NC];
  for (int side = 0; side < 2; ++side) {
    const int Nl = side ? Nn : Ne, pl = Nl + 1;
    for (int x = t; x < pl * pl; x += blockDim.x)
      for (int k = 0; k < NC; ++k) sbuf[x * NC + k] = ld(side, x, k);
    __syncthreads();
    if (!mortar) {
      if (t < pt * pt) {
        if (side == 0) for (int k = 0; k < NC; ++k) va[k] = sbuf[t * NC + k];
        else for (int k = 0; k < NC; ++k) vb[k] = sbuf[t * NC + k];
      }
    } else {
      const double* Im = &M.tab->I[Nl][Mo][0][0];  // [g][i], row stride 8
      for (int x = t; x < pm * pl; x += blockDim.x) {  // stage 1 along fc
        const int a = x / pl, j = x % pl;
        T acc[NC];
        for (int k = 0; k < NC; ++k) acc[k] = T(0.0);
        for (int i = 0; i < pl; ++i) {
          const double c = Im[a * 8 + i];
          for (int k = 0; k < NC; ++k) acc[k] = acc[k] + c * sbuf[(i * pl + j) * NC + k];
        }
        for (int k = 0; k < NC; ++k) stmp[x * NC + k] = acc[k];
      }
      __syncthreads();
      if (t < pm * pm) {  // stage 2 along fb, at the thread's point (a, b)
        const int a = t / pm, b = t % pm;
        T acc[NC];
        for (int k = 0; k < NC; ++k) acc[k] = T(0.0);
        for (int j = 0; j < pl; ++j) {
          const double c = Im[b * 8 + j];
          for (int k = 0; k < NC; ++k) acc[k] = acc[k] + c * stmp[(a * pl + j) * NC + k];
        }
        if (side == 0) for (int k = 0; k < NC; ++k) va[k] = acc[k];
        else for (int k = 0; k < NC; ++k) vb[k] = acc[k];
      }
    }
    __syncthreads();
  }
  T fp[5];
  if (t < pt * pt) pf(t, va, vb, d, s, fp);
  if (!mortar) {
    if (t < pe * pe)
      for (int k = 0; k < 5; ++k) out[t * 5 + k] = fp[k];
    __syncthreads();
    return;
  }
  if (t < pm * pm)
    for (int k = 0; k < 5; ++k) sbuf[t * 5 + k] = fp[k];
  __syncthreads();
  const double* Pm = &M.tab->P[Mo][Ne][0][0];  // [i][g], row stride 8
  for (int x = t; x < pe * pm; x += blockDim.x) {
    const int i = x / pm, b = x % pm;
    T acc[5];
    for (int k = 0; k < 5; ++k) acc[k] = T(0.0);
    for (int a = 0; a < pm; ++a) {
      const double c = Pm[i * 8 + a];
      for (int k = 0; k < 5; ++k) acc[k] = acc[k] + c * sbuf[(a * pm + b) * 5 + k];
    }
    for (int k = 0; k < 5; ++k) stmp[x * 5 + k] = acc[k];
  }
  __syncthreads();
  for (int x = t; x < pe * pe; x += blockDim.x) {
    const int i = x / pe, j = x % pe;
    T acc[5];
    for (int k = 0; k < 5; ++k) acc[k] = T(0.0);
    for (int b = 0; b < pm; ++b) {
      const double c = Pm[j * 8 + b];
      for (int k = 0; k < 5; ++k) acc[k] = acc[k] + c * stmp[(i * pm + b) * 5 + k];
    }
    for (int k = 0; k < 5; ++k) out[x * 5 + k] = acc[k];
  }
  __syncthreads();
}

// Natural node index of face node x (= fc * p + fb) of face (d, s) of an order-N element.
SC_HD inline int face_node(int N, int d, int s, int x) {
  const int p = N + 1;
  int c[3];
  c[d] = s > 0 ? N : 0; c[(d + 1) % 3] = x % p; c[(d + 2) % 3] = x / p;
  return mx_node(c, p);
}

// Point functions of the two face passes: qhat = (q+ + q-)/2 (BR1), and
// fhat = Roe / Lax-Friedrichs(q+, q-) - (1/2) s (f^nu(q+, g+) + f^nu(q-, g-)).
struct PfQhat {
  template <class T>
  __device__ void operator()(int, const T* a, const T* b, int, int, T* out) const {
    for (int k = 0; k < 5; ++k) out[k] = 0.5 * (a[k] + b[k]);
  }
};
struct PfFhat {
  Geo Gp;
  // The viscous fluxes take the face direction as a compile-time constant: the variant with
  // a run-time direction, inlined here, gave wrong dual parts.
  template <int D, class T>
  __device__ void visc(const T* qa, const T* qb, const T (*ga)[5], const T (*gb)[5], T* v) const {
    T fva[5], fvb[5];
    flux_viscous(Gp, qa, ga, D, fva);
    flux_viscous(Gp, qb, gb, D, fvb);
    for (int k = 0; k < 5; ++k) v[k] = fva[k] + fvb[k];
  }
  template <class T>
  __device__ void operator()(int, const T* a, const T* b, int d, int s, T* out) const {
    T fa[5], qa[5], qb[5], ga[3][5], gb[3][5], v[5];
    for (int k = 0; k < 5; ++k) { qa[k] = a[k]; qb[k] = b[k]; }
    for (int x = 0; x < 3; ++x)
      for (int k = 0; k < 5; ++k) { ga[x][k] = a[5 + 5 * x + k]; gb[x][k] = b[5 + 5 * x + k]; }
    flux_adv(Gp, qa, qb, d, s, fa);
    if (d == 0) visc<0>(qa, qb, ga, gb, v);
    else if (d == 1) visc<1>(qa, qb, ga, gb, v);
    else visc<2>(qa, qb, ga, gb, v);
    for (int k = 0; k < 5; ++k) out[k] = fa[k] - 0.5 * (double)s * v[k];
  }
};

// ---- the evaluation pipeline over the whole mesh (T = double, J1 or J1f) ----------------
template <class T>
struct LdGlobal {  // face node values from the global arrays; comps 5.. are the gradients
  const MxMesh* M; int e, f; const double* Q; const double* dir; const T* grad;
  __device__ T operator()(int side, int x, int k) const {
    const int s0 = (f & 1) ? 1 : -1, d = f >> 1;
    const int el = side ? M->nbr[e * 6 + f] : e, s = side ? -s0 : s0;
    const size_t node = (size_t)M->off[el] + face_node(M->ord[el], d, s, x);
    if (k < 5) return Val<T>::make(Q[node * 5 + k], dir ? dir[node * 5 + k] : 0.0);
    return grad[node * 15 + (k - 5)];
  }
};

template <class T, bool WF>
__global__ void __launch_bounds__(64) k_mx_face(MxMesh M, Geo Gp, const double* __restrict__ Q,
                                                const double* __restrict__ dir, const T* __restrict__ grad,
                                                T* __restrict__ out) {
  constexpr int NC = WF ? 20 : 5;
  __shared__ __align__(16) unsigned char raw[2 * 64 * NC * sizeof(T)];  // no constructors in shared memory
  T* sbuf = reinterpret_cast<T*>(raw);
  T* stmp = sbuf + 64 * NC;
  const int e = blockIdx.x / 6, f = blockIdx.x % 6, pe = M.ord[e] + 1;
  LdGlobal<T> ld{&M, e, f, Q, dir, grad};
  T* o = out + ((size_t)M.foff[e] + (size_t)f * pe * pe) * 5;
  if (WF) face_eval<T, NC>(M, e, f, ld, PfFhat{Gp}, sbuf, stmp, o);
  else face_eval<T, NC>(M, e, f, ld, PfQhat{}, sbuf, stmp, o);
}

// Lifted gradient g_a(m) = (2/h) [ sum_b D[m_a][b] q_b + s (qhat - q_m) / w_{m_a} on a face ]
// (the weak form of eq. DGSEMsystem:2 after summation by parts on Gauss-Lobatto nodes).
template <class T>
__global__ void __launch_bounds__(128) k_mx_lift(MxMesh M, const double* __restrict__ Q,
                                                 const double* __restrict__ dir, const T* __restrict__ qhat,
                                                 T* __restrict__ grad) {
  const int e = blockIdx.x, N = M.ord[e], p = N + 1, nn = p * p * p;
  const size_t o = M.off[e];
  const double* D = &M.tab->D[N][0][0];
  const double* w = M.tab->w[N];
  for (int m = threadIdx.x; m < nn; m += blockDim.x) {
    const int c[3] = {m % p, (m / p) % p, m / (p * p)};
    T qm[5];
    for (int k = 0; k < 5; ++k) qm[k] = Val<T>::make(Q[(o + m) * 5 + k], dir ? dir[(o + m) * 5 + k] : 0.0);
    for (int a = 0; a < 3; ++a) {
      T acc[5];
      for (int k = 0; k < 5; ++k) acc[k] = T(0.0);
      int cc[3] = {c[0], c[1], c[2]};
      for (int b = 0; b < p; ++b) {
        cc[a] = b;
        const size_t nd = o + mx_node(cc, p);
        const double Dab = D[c[a] * 8 + b];
        for (int k = 0; k < 5; ++k) acc[k] = acc[k] + Dab * Val<T>::make(Q[nd * 5 + k], dir ? dir[nd * 5 + k] : 0.0);
      }
      if (c[a] == 0 || c[a] == N) {
        const int s = c[a] == N ? 1 : -1, f = 2 * a + (s > 0);
        const int x = c[(a + 2) % 3] * p + c[(a + 1) % 3];
        const T* qh = qhat + ((size_t)M.foff[e] + (size_t)f * p * p + x) * 5;
        const double coef = s / w[c[a]];
        for (int k = 0; k < 5; ++k) acc[k] = acc[k] + coef * (qh[k] - qm[k]);
      }
      for (int k = 0; k < 5; ++k) grad[(o + m) * 15 + a * 5 + k] = M.dx * acc[k];
    }
  }
}

// Point fluxes F_d = f^a_d - f^nu_d(q, g) of every node.
template <class T>
__global__ void __launch_bounds__(128) k_mx_flux(MxMesh M, Geo Gp, const double* __restrict__ Q,
                                                 const double* __restrict__ dir, const T* __restrict__ grad,
                                                 T* __restrict__ F, int nodes) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nodes) return;
  T q[5], g[3][5];
  for (int k = 0; k < 5; ++k) q[k] = Val<T>::make(Q[(size_t)t * 5 + k], dir ? dir[(size_t)t * 5 + k] : 0.0);
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 5; ++k) g[a][k] = grad[(size_t)t * 15 + a * 5 + k];
  T fv[3][5];
  flux_viscous_all(Gp, q, g, fv);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T fa[5];
    flux_inviscid(Gp, q, d, fa);
    for (int k = 0; k < 5; ++k) F[(size_t)t * 15 + d * 5 + k] = fa[k] - fv[d][k];
  }
}

// Residual rows in the strong form that summation by parts gives:
//   R_j = c0 J W_j (q_j - qh_j) / dt + Jf W_j sum_d sum_b D[j_d][b] F_d(b)
//         + sum_{faces of j} Jf W_j / w_{j_d} (fhat_j - s F_d(j)).
// out: the value (T = double) or the derivative part (dual T).
template <class T>
__global__ void __launch_bounds__(128) k_mx_resid(MxMesh M, const double* __restrict__ Q,
                                                  const double* __restrict__ dir, const double* __restrict__ Qh,
                                                  const T* __restrict__ F, const T* __restrict__ fhat,
                                                  double* __restrict__ out) {
  const int e = blockIdx.x, N = M.ord[e], p = N + 1, nn = p * p * p;
  const size_t o = M.off[e];
  const double* D = &M.tab->D[N][0][0];
  const double* w = M.tab->w[N];
  for (int j = threadIdx.x; j < nn; j += blockDim.x) {
    const int c[3] = {j % p, (j / p) % p, j / (p * p)};
    const double Wj = w[c[0]] * w[c[1]] * w[c[2]];
    const double tc = M.c0 * M.J * Wj / M.dt;
    T r[5];
    for (int k = 0; k < 5; ++k) {
      const size_t i = (o + j) * 5 + k;
      r[k] = tc * (Val<T>::make(Q[i], dir ? dir[i] : 0.0) - Qh[i]);
    }
    for (int d = 0; d < 3; ++d) {
      int cc[3] = {c[0], c[1], c[2]};
      for (int b = 0; b < p; ++b) {
        cc[d] = b;
        const double coef = M.Jf * Wj * D[c[d] * 8 + b];
        const T* Fm = F + (o + mx_node(cc, p)) * 15 + d * 5;
        for (int k = 0; k < 5; ++k) r[k] = r[k] + coef * Fm[k];
      }
    }
    for (int d = 0; d < 3; ++d) {
      if (c[d] != 0 && c[d] != N) continue;
      const int s = c[d] == N ? 1 : -1, f = 2 * d + (s > 0);
      const int x = c[(d + 2) % 3] * p + c[(d + 1) % 3];
      const T* fh = fhat + ((size_t)M.foff[e] + (size_t)f * p * p + x) * 5;
      const T* Fj = F + (o + j) * 15 + d * 5;
      const double Sf = M.Jf * Wj / w[c[d]];
      for (int k = 0; k < 5; ++k) r[k] = r[k] + Sf * (fh[k] - (double)s * Fj[k]);
    }
    for (int k = 0; k < 5; ++k) {
      const size_t i = (o + j) * 5 + k;
      out[i] = dir ? Val<T>::der(r[k]) : vval(r[k]);
    }
  }
}

// ---- own element blocks dR_e/dQ_e by five-direction duals, one CTA per element ---------
// Per-element scratch (in T5 units): the qhat of the six faces unseeded (QH0) and seeded
// (QH), the neighbour's qhat on each shared face (QHN, <= 49 nodes), the lifted gradient
// (GE) and point fluxes (FE) of the element, the neighbour's gradients on each shared face
// (GN) and the face fluxes (FH).
// JF: per face and point, the derivatives of fhat with respect to the own side's 20 inputs
// (q, lifted gradient) and the neighbour's 15 gradient inputs, 175 reals (in T5 units: 6 reals each).
constexpr int kFaceJac = 175;
struct OwnScratch {
  int qh0, qh, qhn, ge, fe, gn, fh, jf, total;
  SC_HD OwnScratch(int N) {
    const int p = N + 1, nn = p * p * p, pf = 6 * p * p * 5;
    qh0 = 0; qh = qh0 + pf; qhn = qh + pf; ge = qhn + 6 * 49 * 5; fe = ge + nn * 15; gn = fe + nn * 15;
    fh = gn + 6 * 49 * 15; jf = fh + pf; total = jf + (6 * 49 * kFaceJac + 5) / 6;
  }
};

// Point function of the unseeded pass: the face-flux Jacobians at every point (seven passes of
// five directions: the own 20 inputs, then the neighbour's 15 gradient inputs); no output.
template <class R>
struct PfJac {
  Geo Gp; R* J;  // J[point][175] of one face
  template <class T>
  __device__ void operator()(int t, const T* a, const T* b, int d, int s, T* out) const {
    R* Jt = J + t * kFaceJac;
    for (int pass = 0; pass < 7; ++pass) {
      T qa[20], qb[20], o[5];
      for (int c = 0; c < 20; ++c) { qa[c] = T((double)a[c].v); qb[c] = T((double)b[c].v); }
      for (int i = 0; i < 5; ++i) {
        const int dir = pass * 5 + i;
        if (dir < 20) qa[dir].d[i] = R(1);
        else qb[5 + dir - 20].d[i] = R(1);
      }
      PfFhat{Gp}(t, qa, qb, d, s, o);
      for (int k = 0; k < 5; ++k)
        for (int i = 0; i < 5; ++i) {
          const int dir = pass * 5 + i;
          if (dir < 20) Jt[k * 20 + dir] = o[k].d[i];
          else Jt[100 + k * 15 + dir - 20] = o[k].d[i];
        }
    }
    for (int k = 0; k < 5; ++k) out[k] = T(0.0);
  }
};

// Point function of a seed: the dual parts of fhat from those of the inputs through the
// Jacobians of the unseeded pass (values are not needed: the rows take dual parts only).
template <class R>
struct PfLin {
  const R* J;
  template <class T>
  __device__ void operator()(int t, const T* a, const T* b, int, int, T* out) const {
    const R* Jt = J + t * kFaceJac;
    for (int k = 0; k < 5; ++k) {
      T o;
      for (int i = 0; i < 5; ++i) {
        R acc = R(0);
        for (int c = 0; c < 20; ++c) acc += Jt[k * 20 + c] * a[c].d[i];
        for (int c = 0; c < 15; ++c) acc += Jt[100 + k * 15 + c] * b[5 + c].d[i];
        o.d[i] = acc;
      }
      out[k] = o;
    }
  }
};

// Destination of the blocks: natural order (row 5 j + k, column 5 r + l, leading dimension
// 5 nn) or the condensation layout (rows 5 perm[j] + k; interior columns 5 perm[r] + l,
// boundary columns cb0 + 5 (perm[r] - nin) + l, leading dimension lda).
template <class R>
struct OwnOut {
  R* const* base;  // per list entry
  int natural;
};

template <class R>
__global__ void __launch_bounds__(128) k_mx_own(MxMesh M, Geo Gp, const double* __restrict__ Q,
                                                const double* __restrict__ grad0, const int* __restrict__ elist,
                                                DualN<R, 5>* __restrict__ scratch, long long scratch_slot,
                                                OwnOut<R> outd) {
  using T5 = DualN<R, 5>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T5* sbuf = reinterpret_cast<T5*>(smem_raw);
  T5* stmp = sbuf + 64 * 20;
  const int e = elist[blockIdx.x], N = M.ord[e], p = N + 1, pp = p * p, nn = pp * p;
  const int nin = (N - 1) * (N - 1) * (N - 1), ni = 5 * nin, cb0 = (ni + 3) & ~3;
  const int lda = outd.natural ? 5 * nn : ((cb0 + 5 * (nn - nin) + 3) & ~3);
  R* out = outd.base[blockIdx.x];
  const size_t o = M.off[e];
  const double* D = &M.tab->D[N][0][0];
  const double* w = M.tab->w[N];
  const int* perm = M.tab->perm[N];
  const OwnScratch L(N);
  T5* S = scratch + (long long)blockIdx.x * scratch_slot;
  int seed = -1;  // the node whose five variables are the dual directions
  auto qown = [&](int m, int k) {
    T5 t(Q[(o + m) * 5 + k]);
    if (m == seed) t.d[k] = R(1);
    return t;
  };
  // neighbour across face f of e and the face of the neighbour that faces e
  auto nbr_of = [&](int f) { return M.nbr[e * 6 + f]; };
  for (int r = -1; r < nn; ++r) {
    seed = r;
    int cr[3] = {0, 0, 0};
    if (r >= 0) { cr[0] = r % p; cr[1] = (r / p) % p; cr[2] = r / pp; }
    auto on_face = [&](int f) { const int d = f >> 1; return r >= 0 && cr[d] == ((f & 1) ? N : 0); };
    // qhat of e's faces (r = -1: the unseeded values)
    for (int f = 0; f < 6; ++f) {
      T5* dst = S + (r < 0 ? L.qh0 : L.qh) + f * pp * 5;
      if (r >= 0 && !on_face(f)) continue;  // the lifting reads the unseeded qhat of this face
      const int d = f >> 1, s = (f & 1) ? 1 : -1, nb = nbr_of(f);
      auto ld = [&](int side, int x, int k) -> T5 {
        if (side == 0) return qown(face_node(N, d, s, x), k);
        const size_t node = (size_t)M.off[nb] + face_node(M.ord[nb], d, -s, x);
        return T5(Q[node * 5 + k]);
      };
      face_eval<T5, 5>(M, e, f, ld, PfQhat{}, sbuf, stmp, dst);
    }
    // the neighbours' qhat on the faces through the seed (their lifted gradients move too)
    for (int f = 0; f < 6 && r >= 0; ++f) {
      if (!on_face(f)) continue;
      const int d = f >> 1, s = (f & 1) ? 1 : -1, nb = nbr_of(f), fo = 2 * d + (s < 0);
      auto ld = [&](int side, int x, int k) -> T5 {
        if (side == 1) return qown(face_node(N, d, s, x), k);
        const size_t node = (size_t)M.off[nb] + face_node(M.ord[nb], d, -s, x);
        return T5(Q[node * 5 + k]);
      };
      face_eval<T5, 5>(M, nb, fo, ld, PfQhat{}, sbuf, stmp, S + L.qhn + f * 49 * 5);
    }
    // lifted gradient and point fluxes of e; only nodes on a grid line through the seed or
    // on a face through it move (their derivative parts are cleared again after the seed)
    auto moves = [&](const int c[3]) {
      if (r < 0) return true;
      const int same = (c[0] == cr[0]) + (c[1] == cr[1]) + (c[2] == cr[2]);
      if (same >= 2) return true;
      for (int d = 0; d < 3; ++d)
        if ((c[d] == 0 || c[d] == N) && c[d] == cr[d]) return true;
      return false;
    };
    for (int m = threadIdx.x; m < nn; m += blockDim.x) {
      const int c[3] = {m % p, (m / p) % p, m / pp};
      if (!moves(c)) continue;
      T5 qm[5];
      for (int k = 0; k < 5; ++k) qm[k] = qown(m, k);
      T5 g[3][5];
      for (int a = 0; a < 3; ++a) {
        T5 acc[5];
        int cc[3] = {c[0], c[1], c[2]};
        for (int b = 0; b < p; ++b) {
          cc[a] = b;
          const int mb = mx_node(cc, p);
          const double Dab = D[c[a] * 8 + b];
          for (int k = 0; k < 5; ++k) acc[k] = acc[k] + Dab * qown(mb, k);
        }
        if (c[a] == 0 || c[a] == N) {
          const int s = c[a] == N ? 1 : -1, f = 2 * a + (s > 0);
          const int x = c[(a + 2) % 3] * p + c[(a + 1) % 3];
          const T5* qh = S + (on_face(f) ? L.qh : L.qh0) + (f * pp + x) * 5;
          const double coef = s / w[c[a]];
          for (int k = 0; k < 5; ++k) acc[k] = acc[k] + coef * (qh[k] - qm[k]);
        }
        for (int k = 0; k < 5; ++k) { g[a][k] = M.dx * acc[k]; S[L.ge + m * 15 + a * 5 + k] = g[a][k]; }
      }
      T5 fv[3][5];
      flux_viscous_all(Gp, qm, g, fv);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T5 fa[5];
        flux_inviscid(Gp, qm, d, fa);
        for (int k = 0; k < 5; ++k) S[L.fe + m * 15 + d * 5 + k] = fa[k] - fv[d][k];
      }
    }
    // the neighbours' gradients at their face nodes on the shared faces: the FP64 values
    // plus, on the faces through the seed, the move of their lifting term
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, s = (f & 1) ? 1 : -1, nb = nbr_of(f), Nn = M.ord[nb], pn = Nn + 1;
      const bool moved = on_face(f);
      if (r >= 0 && !moved) continue;  // only the general face path (faces through the seed) reads these
      const double coef = M.dx * (double)(-s) / M.tab->w[Nn][0];
      for (int x = threadIdx.x; x < pn * pn; x += blockDim.x) {
        const size_t node = (size_t)M.off[nb] + face_node(Nn, d, -s, x);
        for (int c = 0; c < 15; ++c) {
          T5 v(grad0[node * 15 + c]);
          if (moved && c / 5 == d) {
            const T5& qh = S[L.qhn + (f * 49 + x) * 5 + c % 5];
            for (int i = 0; i < 5; ++i) v.d[i] = R(coef) * qh.d[i];
          }
          S[L.gn + (f * 49 + x) * 15 + c] = v;
        }
      }
    }
    __syncthreads();
    R* Jf = reinterpret_cast<R*>(S + L.jf);
    // face fluxes of e: at r = -1 the Jacobians of every face point, then per seed their
    // products with the moved inputs
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1, s = (f & 1) ? 1 : -1, nb = nbr_of(f);
      if (r >= 0 && !on_face(f)) {
        // a face away from the seed: the state on it does not move, nor does the neighbour's
        // gradient; the lifted gradient moves at the face nodes the seed moves (the one on
        // its grid line along d, and the rows on faces through the seed), so fhat moves by
        // J_g times their interpolated moves
        const int Nn = M.ord[nb], pe = p;
        const bool mortar = N != Nn || M.force_mortar;
        const int Mo = N > Nn ? N : Nn, pm = Mo + 1, npt = mortar ? pm * pm : pe * pe;
        const R* J = Jf + f * 49 * kFaceJac;
        T5* out5 = S + L.fh + f * pp * 5;
        const double* Im = &M.tab->I[N][Mo][0][0];
        for (int t = threadIdx.x; t < npt; t += blockDim.x) {
          R dg[15][5];
          for (int c = 0; c < 15; ++c)
            for (int i = 0; i < 5; ++i) dg[c][i] = R(0);
          bool any = false;
          for (int x = 0; x < pe * pe; ++x) {
            const int m = face_node(N, d, s, x);
            const int cm[3] = {m % p, (m / p) % p, m / pp};
            if (!moves(cm)) continue;
            const double wgt = mortar ? Im[(t / pm) * 8 + x / pe] * Im[(t % pm) * 8 + x % pe] : (t == x ? 1.0 : 0.0);
            if (wgt == 0.0) continue;
            any = true;
            const T5* g = S + L.ge + m * 15;
            for (int c = 0; c < 15; ++c)
              for (int i = 0; i < 5; ++i) dg[c][i] += R(wgt) * g[c].d[i];
          }
          const R* Jt = J + t * kFaceJac;
          for (int k = 0; k < 5; ++k) {
            T5 o;
            if (any)
              for (int i = 0; i < 5; ++i) {
                R acc = R(0);
                for (int c = 0; c < 15; ++c) acc += Jt[k * 20 + 5 + c] * dg[c][i];
                o.d[i] = acc;
              }
            if (mortar) sbuf[t * 5 + k] = o;
            else out5[t * 5 + k] = o;
          }
        }
        __syncthreads();
        if (mortar) {  // projection onto e's face nodes, as in face_eval
          const double* Pm = &M.tab->P[Mo][N][0][0];
          for (int x = threadIdx.x; x < pe * pm; x += blockDim.x) {
            const int i = x / pm, b = x % pm;
            for (int k = 0; k < 5; ++k) {
              T5 acc;
              for (int a = 0; a < pm; ++a) acc = acc + Pm[i * 8 + a] * sbuf[(a * pm + b) * 5 + k];
              stmp[x * 5 + k] = acc;
            }
          }
          __syncthreads();
          for (int x = threadIdx.x; x < pe * pe; x += blockDim.x) {
            const int i = x / pe, j = x % pe;
            for (int k = 0; k < 5; ++k) {
              T5 acc;
              for (int b = 0; b < pm; ++b) acc = acc + Pm[j * 8 + b] * stmp[(i * pm + b) * 5 + k];
              out5[x * 5 + k] = acc;
            }
          }
          __syncthreads();
        }
        continue;
      }
      auto ld = [&](int side, int x, int k) -> T5 {
        if (side == 0) {
          const int m = face_node(N, d, s, x);
          return k < 5 ? qown(m, k) : S[L.ge + m * 15 + (k - 5)];
        }
        if (k < 5) {
          const size_t node = (size_t)M.off[nb] + face_node(M.ord[nb], d, -s, x);
          return T5(Q[node * 5 + k]);
        }
        return S[L.gn + (f * 49 + x) * 15 + (k - 5)];
      };
      if (r < 0) face_eval<T5, 20>(M, e, f, ld, PfJac<R>{Gp, Jf + f * 49 * kFaceJac}, sbuf, stmp, S + L.fh + f * pp * 5);
      else face_eval<T5, 20>(M, e, f, ld, PfLin<R>{Jf + f * 49 * kFaceJac}, sbuf, stmp, S + L.fh + f * pp * 5);
    }
    if (r < 0) continue;  // unseeded gradients, fluxes and face Jacobians are in place
    // rows of e: the column block of the seed.  Only moved nodes carry a flux derivative, so
    // a row reads the fluxes of the moved nodes on its grid lines; rows with no moved node
    // on them and no face keep the zeros already in the block
    for (int j = threadIdx.x; j < nn; j += blockDim.x) {
      const int c[3] = {j % p, (j / p) % p, j / pp};
      const double Wj = w[c[0]] * w[c[1]] * w[c[2]];
      T5 rr[5];
      bool any = false;
      if (j == r) {
        for (int k = 0; k < 5; ++k) rr[k].d[k] = R(M.c0 * M.J * Wj / M.dt);
        any = true;
      }
      for (int d = 0; d < 3; ++d) {
        int cc[3] = {c[0], c[1], c[2]};
        for (int b = 0; b < p; ++b) {
          cc[d] = b;
          if (!moves(cc)) continue;
          any = true;
          const double coef = M.Jf * Wj * D[c[d] * 8 + b];
          const T5* Fm = S + L.fe + mx_node(cc, p) * 15 + d * 5;
          for (int k = 0; k < 5; ++k) rr[k] = rr[k] + coef * Fm[k];
        }
      }
      const bool jm = moves(c);
      for (int d = 0; d < 3; ++d) {
        if (c[d] != 0 && c[d] != N) continue;
        any = true;
        const int s = c[d] == N ? 1 : -1, f = 2 * d + (s > 0);
        const int x = c[(d + 2) % 3] * p + c[(d + 1) % 3];
        const T5* fh = S + L.fh + (f * pp + x) * 5;
        const double Sf = M.Jf * Wj / w[c[d]];
        for (int k = 0; k < 5; ++k) rr[k] = rr[k] + Sf * fh[k];
        if (jm) {
          const T5* Fj = S + L.fe + j * 15 + d * 5;
          for (int k = 0; k < 5; ++k) rr[k] = rr[k] - (Sf * (double)s) * Fj[k];
        }
      }
      if (!any) continue;
      const int pj = perm[j], pr = perm[r];
      for (int k = 0; k < 5; ++k)
        for (int l = 0; l < 5; ++l) {
          size_t row, col;
          if (outd.natural) { row = 5 * j + k; col = 5 * r + l; }
          else { row = 5 * pj + k; col = pr < nin ? 5 * pr + l : cb0 + 5 * (pr - nin) + l; }
          out[row * lda + col] = rr[k].d[l];
        }
    }
    __syncthreads();
    // back to the unseeded gradients and fluxes (their values do not depend on the seed)
    for (int m = threadIdx.x; m < nn; m += blockDim.x) {
      const int c[3] = {m % p, (m / p) % p, m / pp};
      if (!moves(c)) continue;
      for (int x = 0; x < 15; ++x)
        for (int i = 0; i < 5; ++i) { S[L.ge + m * 15 + x].d[i] = R(0); S[L.fe + m * 15 + x].d[i] = R(0); }
    }
    __syncthreads();
  }
}

// ---- condensed vectors: boundary and interior dofs of every element, elements ordered by
// order class (decreasing N), so that each class is one uniform block of the vectors -----
template <class TI>
__global__ void k_mx_scatter(int nodes, const int* __restrict__ bmap, const int* __restrict__ imap,
                             const TI* __restrict__ xb, const TI* __restrict__ xi, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nodes) return;
  const int b = bmap[t], i = imap[t];
  for (int k = 0; k < 5; ++k) {
    double v = 0.0;
    if (b >= 0 && xb) v = (double)xb[b + k];
    if (i >= 0 && xi) v = (double)xi[i + k];
    out[(size_t)t * 5 + k] = v;
  }
}

// yb = in_b (sub = 0) or yb -= in_b (sub = 1); yi = in_i.
__global__ void k_mx_gather(int nodes, const int* __restrict__ bmap, const int* __restrict__ imap,
                            const double* __restrict__ in, double* __restrict__ yb, double* __restrict__ yi, int sub) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nodes) return;
  const int b = bmap[t], i = imap[t];
  for (int k = 0; k < 5; ++k) {
    const double v = in[(size_t)t * 5 + k];
    if (b >= 0 && yb) yb[b + k] = sub ? yb[b + k] - v : v;
    if (i >= 0 && yi) yi[i + k] = v;
  }
}

// u = A_ii^-1 x for the elements of one order class (FP32 inverses n_i x ldi, one CTA per
// element, a warp per row); x and u in FP64, class-contiguous with stride n_i.
__global__ void __launch_bounds__(256) k_mx_ainv(int ni, int ldi, const float* __restrict__ Ainv,
                                                 const double* __restrict__ x, const double* __restrict__ xsub,
                                                 double* __restrict__ u) {
  __shared__ float xs[640];
  const size_t el = blockIdx.x;
  const double* xe = x + el * ni;
  for (int j = threadIdx.x; j < ni; j += blockDim.x) xs[j] = (float)(xsub ? xe[j] - xsub[el * ni + j] : xe[j]);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* A = Ainv + el * (size_t)ni * ldi;
  for (int i = warp; i < ni; i += blockDim.x / 32) {
    float acc = 0.f;
    for (int j = lane; j < ni; j += 32) acc = fmaf(A[(size_t)i * ldi + j], xs[j], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) u[el * ni + i] = (double)acc;
  }
}

__global__ void k_mx_history(const double* __restrict__ Qs, const double* __restrict__ Qsm1, double* __restrict__ Qh,
                             size_t n, int bdf) {
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t < n) Qh[t] = bdf == 2 ? (4.0 * Qs[t] - Qsm1[t]) / 3.0 : Qs[t];
}

inline unsigned mx_blocks(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---- host tables ---------------------------------------------------------------------
double lagrange_at(const std::vector<double>& x, int i, double t) {
  double v = 1.0;
  for (int j = 0; j < (int)x.size(); ++j)
    if (j != i) v *= (t - x[j]) / (x[i] - x[j]);
  return v;
}

// Gauss-Legendre points and weights of m points: Newton on P_m from cos(pi (i + 3/4) / (m + 1/2)).
void gauss_legendre_rule(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0); w.assign(m, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < m; ++i) {
    double z = std::cos(pi * (i + 0.75) / (m + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= m; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= m; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    dp = m * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z; w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void build_tables(MxTab& T) {
  std::memset(&T, 0, sizeof(T));
  std::vector<double> X[8];
  for (int N = 1; N <= 7; ++N) {
    std::vector<double> w;
    double Dm[SC_MAXP][SC_MAXP];
    sc::gl_basis(N, X[N], w, Dm);
    for (int i = 0; i <= N; ++i) {
      T.w[N][i] = w[i];
      for (int j = 0; j <= N; ++j) T.D[N][i][j] = Dm[i][j];
    }
    const int p = N + 1, nin = (N - 1) * (N - 1) * (N - 1);
    int ii = 0, bb = nin;
    for (int m = 0; m < p * p * p; ++m) {
      const int i = m % p, j = (m / p) % p, k = m / (p * p);
      const bool inner = i > 0 && i < N && j > 0 && j < N && k > 0 && k < N;
      T.perm[N][m] = inner ? ii++ : bb++;
    }
  }
  for (int a = 1; a <= 7; ++a)
    for (int b = 1; b <= 7; ++b)
      for (int g = 0; g <= b; ++g)
        for (int i = 0; i <= a; ++i) T.I[a][b][g][i] = lagrange_at(X[a], i, X[b][g]);
  // projection onto order N of the order-M interpolant: mass matrix and mixed moments with
  // the Gauss rule of M + 1 points (exact for the degree 2M products), then M^-1 B
  for (int M = 1; M <= 7; ++M) {
    std::vector<double> gx, gw;
    gauss_legendre_rule(M + 1, gx, gw);
    for (int N = 1; N <= M; ++N) {
      const int pe = N + 1, pm = M + 1;
      std::vector<double> A((size_t)pe * pe, 0.0), Bm((size_t)pe * pm, 0.0);
      for (size_t q = 0; q < gx.size(); ++q)
        for (int i = 0; i < pe; ++i) {
          const double li = lagrange_at(X[N], i, gx[q]);
          for (int j = 0; j < pe; ++j) A[(size_t)i * pe + j] += gw[q] * li * lagrange_at(X[N], j, gx[q]);
          for (int g = 0; g < pm; ++g) Bm[(size_t)i * pm + g] += gw[q] * li * lagrange_at(X[M], g, gx[q]);
        }
      // Cholesky of the symmetric positive definite mass matrix, then the pm right-hand sides
      std::vector<double> Lc((size_t)pe * pe, 0.0);
      for (int i = 0; i < pe; ++i)
        for (int j = 0; j <= i; ++j) {
          double s = A[(size_t)i * pe + j];
          for (int k = 0; k < j; ++k) s -= Lc[(size_t)i * pe + k] * Lc[(size_t)j * pe + k];
          Lc[(size_t)i * pe + j] = (i == j) ? std::sqrt(s) : s / Lc[(size_t)j * pe + j];
        }
      for (int g = 0; g < pm; ++g) {
        std::vector<double> y(pe);
        for (int i = 0; i < pe; ++i) {
          double s = Bm[(size_t)i * pm + g];
          for (int k = 0; k < i; ++k) s -= Lc[(size_t)i * pe + k] * y[k];
          y[i] = s / Lc[(size_t)i * pe + i];
        }
        for (int i = pe - 1; i >= 0; --i) {
          double s = y[i];
          for (int k = i + 1; k < pe; ++k) s -= Lc[(size_t)k * pe + i] * y[k];
          y[i] = s / Lc[(size_t)i * pe + i];
        }
        for (int i = 0; i < pe; ++i) T.P[M][N][i][g] = y[i];
      }
    }
  }
}

struct MxClass {  // the elements of one order
  int N = 0, nin = 0, ni = 0, nb = 0, ne = 0, cb0 = 0, lda = 0, ldi = 0, lds = 0, count = 0, slot0 = 0;
  long long ls = 0;  // solve-layout stride
  float *Aown32 = nullptr, *Ainv32 = nullptr, *Y32 = nullptr, *See32 = nullptr, *Sls32 = nullptr, *dsc = nullptr;
  int *piv = nullptr, *rowperm = nullptr;
  sc_ctx* view = nullptr;  // sizes and stream for the shared block-solve kernels
  cudaStream_t st = nullptr;       // the class's own stream (the class passes run concurrently)
  cudaEvent_t done = nullptr;
  int bn_y = 144, bn_s = 144, bn_t = 144;
  size_t off_y = 0, off_s = 0;
  std::vector<size_t> off_t;
};

}  // namespace

struct sc_mixed {
  sc_config cfg{};
  cudaStream_t stream = nullptr;
  std::string err;
  int n = 0, K = 0, force_mortar = 0, bdf = 1;
  double L = 0.0, dt = 1.0;
  bool has_state = false, condensed = false;
  std::vector<int> ord, off, foff, nbr, slot_elem;  // slot_elem: element of each slot
  std::vector<long long> boff, ioff;                // per slot
  long long nodes = 0, nbt = 0, nit = 0;
  Geo Gp{};
  MxMesh M{};
  MxTab* d_tab = nullptr;
  int *d_ord = nullptr, *d_off = nullptr, *d_foff = nullptr, *d_nbr = nullptr, *d_bmap = nullptr, *d_imap = nullptr;
  double *Q = nullptr, *Qh = nullptr, *grad0 = nullptr, *F0 = nullptr, *qh0 = nullptr, *fh0 = nullptr;
  double *gJ = nullptr, *FJ = nullptr, *qhJ = nullptr, *fhJ = nullptr;  // dual pipeline (sized for J1)
  double *vA = nullptr, *vB = nullptr, *B = nullptr, *Rr = nullptr, *dQ = nullptr;  // full vectors
  double *ri = nullptr, *ui = nullptr, *xi = nullptr;               // interior vectors
  double *gb = nullptr, *xb = nullptr, *V = nullptr, *Wv = nullptr, *Tb = nullptr, *Zb = nullptr;  // boundary
  std::vector<MxClass> cls;
  std::vector<CondItem> items;
  CondItem* d_items = nullptr;
  void** d_ptrs = nullptr;
  std::vector<void*> h_ptrs;
  int max_ni = 0, max_nb = 0, nbig_gj = 0, nbig_lu = 0, restart = 30;
  int* d_status = nullptr;
  DualN<float, 5>* own_scratch = nullptr;
  long long own_slot = 0, own_chunk = 0;
  float** d_own_out = nullptr;
  int* d_elist = nullptr;
  sc_ctx* aux = nullptr;  // Krylov workspace of the shared vector kernels
  cudaEvent_t fork = nullptr;
  // measurement hook: events around every block-Jacobi application
  bool prof = false;
  int prof_used = 0;
  std::vector<cudaEvent_t> prof_ev;
  long long launches = 0;
};

namespace {

sc_status mfail(sc_mixed* m, sc_status s, const std::string& msg) {
  if (m) m->err = msg;
  return s;
}

#define MX_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t _e = (call);                                                                     \
    if (_e != cudaSuccess) return mfail(m, SC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

template <class P>
cudaError_t mx_alloc(P** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(P));
}

// One evaluation of the pipeline in type T: out = R(Q) (dir null) or (dR/dQ) dir.
template <class T>
cudaError_t mx_eval(sc_mixed* m, const double* dir, double* out) {
  const MxMesh& M = m->M;
  T* qh = std::is_same<T, double>::value ? reinterpret_cast<T*>(m->qh0) : reinterpret_cast<T*>(m->qhJ);
  T* g = std::is_same<T, double>::value ? reinterpret_cast<T*>(m->grad0) : reinterpret_cast<T*>(m->gJ);
  T* fh = std::is_same<T, double>::value ? reinterpret_cast<T*>(m->fh0) : reinterpret_cast<T*>(m->fhJ);
  T* F = std::is_same<T, double>::value ? reinterpret_cast<T*>(m->F0) : reinterpret_cast<T*>(m->FJ);
  const cudaStream_t st = m->stream;
  k_mx_face<T, false><<<M.K * 6, 64, 0, st>>>(M, m->Gp, m->Q, dir, nullptr, qh);
  k_mx_lift<T><<<M.K, 128, 0, st>>>(M, m->Q, dir, qh, g);
  k_mx_face<T, true><<<M.K * 6, 64, 0, st>>>(M, m->Gp, m->Q, dir, g, fh);
  k_mx_flux<T><<<mx_blocks(m->nodes, 128), 128, 0, st>>>(M, m->Gp, m->Q, dir, g, F, (int)m->nodes);
  k_mx_resid<T><<<M.K, 128, 0, st>>>(M, m->Q, dir, m->Qh, F, fh, out);
  m->launches += 5;
  return cudaGetLastError();
}

}  // namespace

namespace {

// Scratch of the own-block kernel: elements processed per launch, and the per-element slot.
constexpr int kOwnChunk = 512;

template <class R>
cudaError_t mx_own_launch(sc_mixed* m, const int* d_elist, int count, DualN<R, 5>* scratch, long long slot,
                          R* const* d_out, int natural) {
  const size_t smem = (size_t)2 * 64 * 20 * sizeof(DualN<R, 5>);
  cudaError_t e = cudaFuncSetAttribute(k_mx_own<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  OwnOut<R> od{d_out, natural};
  k_mx_own<R><<<count, 128, smem, m->stream>>>(m->M, m->Gp, m->Q, m->grad0, d_elist, scratch, slot, od);
  m->launches += 1;
  return cudaGetLastError();
}

}  // namespace

extern "C" {

sc_status sc_mixed_create(const sc_config* cfg, void* cuda_stream, int n, double L, const int* orders,
                          int force_mortar, sc_mixed** out) {
  if (!cfg || !orders || !out) return SC_ERR_ARG;
  *out = nullptr;
  if (n < 2 || n > 32 || !(L > 0)) return SC_ERR_ARG;
  if (cfg->precision != SC_PREC_MIXED || (cfg->precond != SC_PC_BLOCK_JACOBI && cfg->precond != SC_PC_NONE) ||
      cfg->visc_flux != SC_VISC_BR1 || (cfg->adv_flux != SC_FLUX_ROE && cfg->adv_flux != SC_FLUX_LF) ||
      cfg->gmres_restart < 1 || cfg->gmres_restart > 400 || cfg->gmres_max_iters < 1 || !(cfg->rel_tol > 0) ||
      !(cfg->inner_tol > 0) || !(cfg->Re > 0) || !(cfg->Ma > 0) || !(cfg->gamma > 1) || !(cfg->Pr > 0))
    return SC_ERR_ARG;
  const int K = n * n * n;
  for (int e = 0; e < K; ++e)
    if (orders[e] < 2 || orders[e] > 6) return SC_ERR_ARG;
  sc_mixed* m = new sc_mixed();
  m->cfg = *cfg;
  m->stream = (cudaStream_t)cuda_stream;
  m->n = n; m->K = K; m->L = L; m->force_mortar = force_mortar ? 1 : 0;
  m->restart = cfg->gmres_restart;
  m->ord.assign(orders, orders + K);
  m->off.assign(K + 1, 0); m->foff.assign(K + 1, 0);
  for (int e = 0; e < K; ++e) {
    const int p = m->ord[e] + 1;
    m->off[e + 1] = m->off[e] + p * p * p;
    m->foff[e + 1] = m->foff[e] + 6 * p * p;
  }
  m->nodes = m->off[K];
  m->nbr.assign((size_t)K * 6, 0);
  for (int e = 0; e < K; ++e) {
    const int c[3] = {e % n, (e / n) % n, e / (n * n)};
    for (int d = 0; d < 3; ++d)
      for (int s = -1; s <= 1; s += 2) {
        int cc[3] = {c[0], c[1], c[2]};
        cc[d] = (cc[d] + s + n) % n;
        m->nbr[(size_t)e * 6 + 2 * d + (s > 0)] = cc[0] + n * (cc[1] + n * cc[2]);
      }
  }
  // order classes, largest first; slots of the condensed vectors follow them
  MxTab* tab = new MxTab();
  build_tables(*tab);
  for (int N = 6; N >= 2; --N) {
    MxClass c;
    c.N = N; c.nin = (N - 1) * (N - 1) * (N - 1);
    c.ni = 5 * c.nin; c.ne = 5 * (N + 1) * (N + 1) * (N + 1); c.nb = c.ne - c.ni;
    c.cb0 = (c.ni + 3) & ~3; c.lda = (c.cb0 + c.nb + 3) & ~3; c.ldi = (c.ni + 3) & ~3; c.lds = (c.nb + 3) & ~3;
    c.slot0 = (int)m->slot_elem.size();
    for (int e = 0; e < K; ++e)
      if (m->ord[e] == N) m->slot_elem.push_back(e);
    c.count = (int)m->slot_elem.size() - c.slot0;
    if (c.count > 0) m->cls.push_back(c);
  }
  std::vector<int> slot_of(K), bmap(m->nodes, -1), imap(m->nodes, -1);
  m->boff.assign(K + 1, 0); m->ioff.assign(K + 1, 0);
  for (int s = 0; s < K; ++s) {
    const int e = m->slot_elem[s], N = m->ord[e], p = N + 1, nin = (N - 1) * (N - 1) * (N - 1);
    slot_of[e] = s;
    m->boff[s + 1] = m->boff[s] + 5LL * (p * p * p - nin);
    m->ioff[s + 1] = m->ioff[s] + 5LL * nin;
    for (int mm = 0; mm < p * p * p; ++mm) {
      const int pos = tab->perm[N][mm];
      if (pos < nin) imap[m->off[e] + mm] = (int)(m->ioff[s] + 5 * pos);
      else bmap[m->off[e] + mm] = (int)(m->boff[s] + 5 * (pos - nin));
    }
  }
  m->nbt = m->boff[K]; m->nit = m->ioff[K];
  Geo& G = m->Gp;
  G.gamma = cfg->gamma; G.Pr = cfg->Pr; G.Re = cfg->Re; G.Ma = cfg->Ma; G.Ts = cfg->Ts;
  G.roe_delta = cfg->roe_delta; G.sutherland = cfg->sutherland; G.adv_flux = cfg->adv_flux; G.visc_flux = 0;
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  const size_t dofs = (size_t)m->nodes * 5, fpts = (size_t)m->foff[K] * 5;
  A(mx_alloc(&m->d_tab, 1)); A(mx_alloc(&m->d_ord, K)); A(mx_alloc(&m->d_off, K + 1));
  A(mx_alloc(&m->d_foff, K + 1)); A(mx_alloc(&m->d_nbr, (size_t)K * 6));
  A(mx_alloc(&m->d_bmap, m->nodes)); A(mx_alloc(&m->d_imap, m->nodes));
  A(mx_alloc(&m->Q, dofs)); A(mx_alloc(&m->Qh, dofs)); A(mx_alloc(&m->grad0, dofs * 3)); A(mx_alloc(&m->F0, dofs * 3));
  A(mx_alloc(&m->qh0, fpts)); A(mx_alloc(&m->fh0, fpts));
  A(mx_alloc(&m->gJ, dofs * 6)); A(mx_alloc(&m->FJ, dofs * 6)); A(mx_alloc(&m->qhJ, fpts * 2)); A(mx_alloc(&m->fhJ, fpts * 2));
  A(mx_alloc(&m->vA, dofs)); A(mx_alloc(&m->vB, dofs)); A(mx_alloc(&m->B, dofs)); A(mx_alloc(&m->Rr, dofs));
  A(mx_alloc(&m->dQ, dofs));
  A(mx_alloc(&m->ri, m->nit)); A(mx_alloc(&m->ui, m->nit)); A(mx_alloc(&m->xi, m->nit));
  A(mx_alloc(&m->gb, m->nbt)); A(mx_alloc(&m->xb, m->nbt)); A(mx_alloc(&m->Wv, m->nbt)); A(mx_alloc(&m->Tb, m->nbt));
  A(mx_alloc(&m->Zb, m->nbt)); A(mx_alloc(&m->V, (size_t)m->nbt * (m->restart + 1)));
  if (e == cudaSuccess) {
    A(cudaMemcpy(m->d_tab, tab, sizeof(MxTab), cudaMemcpyHostToDevice));
    A(cudaMemcpy(m->d_ord, m->ord.data(), K * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemcpy(m->d_off, m->off.data(), (K + 1) * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemcpy(m->d_foff, m->foff.data(), (K + 1) * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemcpy(m->d_nbr, m->nbr.data(), (size_t)K * 6 * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemcpy(m->d_bmap, bmap.data(), m->nodes * sizeof(int), cudaMemcpyHostToDevice));
    A(cudaMemcpy(m->d_imap, imap.data(), m->nodes * sizeof(int), cudaMemcpyHostToDevice));
  }
  delete tab;
  MxMesh& M = m->M;
  M.K = K; M.n = n; M.force_mortar = m->force_mortar;
  M.h = L / n; M.dx = 2.0 / M.h; M.J = std::pow(0.5 * M.h, 3); M.Jf = std::pow(0.5 * M.h, 2);
  M.dt = 1.0; M.c0 = 1.0;
  M.ord = m->d_ord; M.off = m->d_off; M.foff = m->d_foff; M.nbr = m->d_nbr; M.tab = m->d_tab;
  // condensation buffers per class, and the grouped items (largest blocks first)
  for (MxClass& c : m->cls) {
    Geo Gc{};
    Gc.nb = c.nb; Gc.ni = c.ni; Gc.ne = c.ne; Gc.K = c.count; Gc.N = c.N;
    c.ls = sc::solve_layout_stride(Gc);
    const size_t k = c.count;
    A(mx_alloc(&c.Aown32, k * c.ne * c.lda)); A(mx_alloc(&c.Ainv32, k * c.ni * c.ldi));
    A(mx_alloc(&c.Y32, k * c.nb * c.ldi)); A(mx_alloc(&c.See32, k * c.nb * c.lds));
    A(mx_alloc(&c.Sls32, k * c.ls)); A(mx_alloc(&c.dsc, k * c.ni));
    A(mx_alloc(&c.piv, k * c.nb)); A(mx_alloc(&c.rowperm, k * c.nb));
    A(cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking));
    A(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
    c.view = new sc_ctx();
    c.view->G = Gc; c.view->stream = c.st; c.view->cfg = *cfg;
    c.view->rowperm = c.rowperm;
    m->max_ni = std::max(m->max_ni, c.ni);
    m->max_nb = std::max(m->max_nb, c.nb);
  }
  A(mx_alloc(&m->d_status, 1));
  A(cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming));
  if (e == cudaSuccess) {
    for (MxClass& c : m->cls)
      for (int i = 0; i < c.count; ++i) {
        CondItem it;
        it.ni = c.ni; it.nb = c.nb; it.lda = c.lda; it.ldi = c.ldi; it.lds = c.lds; it.cb0 = c.cb0;
        it.e = m->slot_elem[c.slot0 + i];
        it.Aown = c.Aown32 + (size_t)i * c.ne * c.lda;
        it.Ainv = c.Ainv32 + (size_t)i * c.ni * c.ldi;
        it.Yt = c.Y32 + (size_t)i * c.nb * c.ldi;
        it.See = c.See32 + (size_t)i * c.nb * c.lds;
        it.Sls = c.Sls32 + (size_t)i * c.ls;
        it.piv = c.piv + (size_t)i * c.nb;
        it.rowperm = c.rowperm + (size_t)i * c.nb;
        it.status = m->d_status;
        it.dsc = c.dsc + (size_t)i * c.ni;
        m->items.push_back(it);
      }
    for (const CondItem& it : m->items) {
      if (sc::gj_blocked_item(it.ni)) ++m->nbig_gj;
      if (sc::lu_panel_smem_item(it.nb)) ++m->nbig_lu;
    }
    // address tables of the tensor-core products, per class (items of a class are contiguous)
    size_t first = 0;
    for (MxClass& c : m->cls) {
      const CondItem* its = m->items.data() + first;
      auto push3 = [&](auto fa, auto fb, auto fc) {
        const size_t o = m->h_ptrs.size();
        for (int i = 0; i < c.count; ++i) m->h_ptrs.push_back((void*)fa(its[i]));
        for (int i = 0; i < c.count; ++i) m->h_ptrs.push_back((void*)fb(its[i]));
        for (int i = 0; i < c.count; ++i) m->h_ptrs.push_back((void*)fc(its[i]));
        return o;
      };
      c.off_y = push3([](const CondItem& it) { return it.Aown + it.cb0; }, [](const CondItem& it) { return it.Ainv; },
                      [](const CondItem& it) { return it.Yt; });
      c.off_s = push3([](const CondItem& it) { return it.Aown + (size_t)it.ni * it.lda; },
                      [](const CondItem& it) { return it.Yt; }, [](const CondItem& it) { return it.See; });
      for (int k0 = 0; c.nb - k0 - 32 > 0; k0 += 32)
        c.off_t.push_back(push3([k0](const CondItem& it) { return it.See + (size_t)(k0 + 32) * it.lds + k0; },
                                [k0](const CondItem& it) { return it.See + (size_t)k0 * it.lds + k0 + 32; },
                                [k0](const CondItem& it) { return it.See + (size_t)(k0 + 32) * it.lds + k0 + 32; }));
      first += c.count;
    }
    A(mx_alloc(&m->d_items, m->items.size()));
    A(mx_alloc(&m->d_ptrs, m->h_ptrs.size()));
    if (e == cudaSuccess) {
      A(cudaMemcpy(m->d_items, m->items.data(), m->items.size() * sizeof(CondItem), cudaMemcpyHostToDevice));
      A(cudaMemcpy(m->d_ptrs, m->h_ptrs.data(), m->h_ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice));
    }
  }
  // own-block scratch: a chunk of elements per launch, slots sized for the largest order
  m->own_chunk = std::min<long long>(K, kOwnChunk);
  m->own_slot = OwnScratch(m->cls.empty() ? 2 : m->cls[0].N).total;
  A(mx_alloc(&m->own_scratch, (size_t)m->own_chunk * m->own_slot));
  A(mx_alloc(&m->d_own_out, (size_t)K));
  A(mx_alloc(&m->d_elist, (size_t)K));
  // Krylov workspace
  m->aux = new sc_ctx();
  m->aux->stream = m->stream; m->aux->cfg = *cfg; m->aux->restart_alloc = m->restart;
  A(mx_alloc(&m->aux->partial, 152 * (size_t)(m->restart + 2)));
  A(mx_alloc(&m->aux->Hd, 3 * (size_t)(m->restart + 2) + 16));
  if (e != cudaSuccess) {
    sc_mixed_destroy(m);
    return SC_ERR_OOM;
  }
  *out = m;
  return SC_OK;
}

void sc_mixed_destroy(sc_mixed* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  void* ps[] = {m->d_tab, m->d_ord, m->d_off, m->d_foff, m->d_nbr, m->d_bmap, m->d_imap, m->Q, m->Qh, m->grad0,
                m->F0, m->qh0, m->fh0, m->gJ, m->FJ, m->qhJ, m->fhJ, m->vA, m->vB, m->B, m->Rr, m->dQ, m->ri,
                m->ui, m->xi, m->gb, m->xb, m->V, m->Wv, m->Tb, m->Zb, m->d_items, m->d_ptrs, m->d_status,
                m->own_scratch, m->d_own_out, m->d_elist};
  for (void* p : ps) if (p) cudaFree(p);
  for (MxClass& c : m->cls) {
    void* cs[] = {c.Aown32, c.Ainv32, c.Y32, c.See32, c.Sls32, c.dsc, c.piv, c.rowperm};
    for (void* p : cs) if (p) cudaFree(p);
    if (c.st) cudaStreamDestroy(c.st);
    if (c.done) cudaEventDestroy(c.done);
    delete c.view;
  }
  if (m->fork) cudaEventDestroy(m->fork);
  for (cudaEvent_t ev : m->prof_ev) cudaEventDestroy(ev);
  if (m->aux) {
    if (m->aux->partial) cudaFree(m->aux->partial);
    if (m->aux->Hd) cudaFree(m->aux->Hd);
    delete m->aux;
  }
  delete m;
}

const char* sc_mixed_last_error(const sc_mixed* m) { return m ? m->err.c_str() : "null context"; }

sc_status sc_mixed_sizes(const sc_mixed* m, long long* nodes, long long* nb_total, long long* ni_total) {
  if (!m) return SC_ERR_ARG;
  if (nodes) *nodes = m->nodes;
  if (nb_total) *nb_total = m->nbt;
  if (ni_total) *ni_total = m->nit;
  return SC_OK;
}

sc_status sc_mixed_set_state(sc_mixed* m, const double* Q, const double* Qs, const double* Qsm1, double dt, int bdf,
                             int on_device) {
  if (!m || !Q || !Qs || !(dt > 0) || (bdf != 1 && bdf != 2) || (bdf == 2 && !Qsm1)) return SC_ERR_ARG;
  const size_t n = (size_t)m->nodes * 5, bytes = n * sizeof(double);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  MX_CUDA(cudaMemcpyAsync(m->Q, Q, bytes, kind, m->stream));
  MX_CUDA(cudaMemcpyAsync(m->vA, Qs, bytes, kind, m->stream));
  if (bdf == 2) MX_CUDA(cudaMemcpyAsync(m->vB, Qsm1, bytes, kind, m->stream));
  k_mx_history<<<mx_blocks((long long)n, 256), 256, 0, m->stream>>>(m->vA, bdf == 2 ? m->vB : m->vA, m->Qh, n, bdf);
  m->launches += 1;
  MX_CUDA(cudaGetLastError());
  m->dt = dt; m->bdf = bdf;
  m->M.dt = dt; m->M.c0 = bdf == 2 ? 1.5 : 1.0;
  m->has_state = true; m->condensed = false;
  MX_CUDA(cudaStreamSynchronize(m->stream));
  return SC_OK;
}

sc_status sc_mixed_residual(sc_mixed* m, double* R, int on_device) {
  if (!m || !R) return SC_ERR_ARG;
  if (!m->has_state) return mfail(m, SC_ERR_STATE, "residual before set_state");
  MX_CUDA(mx_eval<double>(m, nullptr, m->Rr));
  MX_CUDA(cudaMemcpyAsync(R, m->Rr, (size_t)m->nodes * 5 * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  MX_CUDA(cudaStreamSynchronize(m->stream));
  return SC_OK;
}

sc_status sc_mixed_jvp(sc_mixed* m, const double* x, double* y, int on_device) {
  if (!m || !x || !y) return SC_ERR_ARG;
  if (!m->has_state) return mfail(m, SC_ERR_STATE, "jvp before set_state");
  const size_t bytes = (size_t)m->nodes * 5 * sizeof(double);
  const double* dir = x;
  if (!on_device) {
    MX_CUDA(cudaMemcpyAsync(m->vB, x, bytes, cudaMemcpyHostToDevice, m->stream));
    dir = m->vB;
  }
  MX_CUDA(mx_eval<J1>(m, dir, m->Rr));
  MX_CUDA(cudaMemcpyAsync(y, m->Rr, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  MX_CUDA(cudaStreamSynchronize(m->stream));
  return SC_OK;
}

// FP64 dR_e/dQ_e of element e in natural node order (5 nn_e x 5 nn_e, row-major), to host.
sc_status sc_mixed_own_block(sc_mixed* m, int e, double* block) {
  if (!m || !block || e < 0 || e >= m->K) return SC_ERR_ARG;
  if (!m->has_state) return mfail(m, SC_ERR_STATE, "own_block before set_state");
  const int p = m->ord[e] + 1, ne = 5 * p * p * p;
  MX_CUDA(mx_eval<double>(m, nullptr, m->Rr));  // the lifted gradients of the state
  DualN<double, 5>* scr = nullptr;
  double* blk = nullptr;
  double** outp = nullptr;
  int* el = nullptr;
  cudaError_t ce = mx_alloc(&scr, (size_t)OwnScratch(m->ord[e]).total);
  if (ce == cudaSuccess) ce = mx_alloc(&blk, (size_t)ne * ne);
  if (ce == cudaSuccess) ce = mx_alloc(&outp, 1);
  if (ce == cudaSuccess) ce = mx_alloc(&el, 1);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(outp, &blk, sizeof(double*), cudaMemcpyHostToDevice, m->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(el, &e, sizeof(int), cudaMemcpyHostToDevice, m->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(blk, 0, (size_t)ne * ne * sizeof(double), m->stream);
  if (ce == cudaSuccess) ce = mx_own_launch<double>(m, el, 1, scr, 0, outp, 1);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(block, blk, (size_t)ne * ne * sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(m->stream);
  cudaFree(scr); cudaFree(blk); cudaFree(outp); cudaFree(el);
  if (ce != cudaSuccess) return mfail(m, SC_ERR_CUDA, std::string("own block: ") + cudaGetErrorString(ce));
  return SC_OK;
}

}  // extern "C"

namespace {

cudaError_t mx_products(sc_mixed* m, const MxClass& c, size_t off, int M, int N, int K, float alpha, int lda,
                        bool ta, int ldb, bool tb, float beta, int ldc) {
  const float* const* A = reinterpret_cast<const float* const*>(m->d_ptrs + off);
  m->launches += 1;
  return sc::gemm_tf32_ptrs(m->stream, M, N, K, alpha, A, lda, ta, A + c.count, ldb, tb, beta,
                            reinterpret_cast<float* const*>(m->d_ptrs + off + 2 * c.count), ldc, c.count, c.bn_y,
                            m->d_status);
}

// The grouped condensation of all elements (the sequence of the batched condensation).
cudaError_t mx_condense_blocks(sc_mixed* m) {
  const cudaStream_t st = m->stream;
  const int n = (int)m->items.size();
  cudaError_t e = sc::grouped_gj(st, m->d_items, n, m->nbig_gj, m->max_ni);
  m->launches += sc::grouped_gj_launches(m->nbig_gj, n, m->max_ni);
  for (const MxClass& c : m->cls)  // Y^T = A_ib^T A_ii^-T
    if (e == cudaSuccess) e = mx_products(m, c, c.off_y, c.nb, c.ni, c.ni, 1.0f, c.lda, true, c.ldi, true, 0.0f, c.ldi);
  if (e == cudaSuccess) { e = sc::grouped_copy_bb(st, m->d_items, n); m->launches += 1; }
  for (const MxClass& c : m->cls)  // S_ee = A_bb - A_bi Y
    if (e == cudaSuccess) e = mx_products(m, c, c.off_s, c.nb, c.nb, c.ni, -1.0f, c.lda, false, c.ldi, true, 1.0f, c.lds);
  for (int step = 0; 32 * step < m->max_nb && e == cudaSuccess; ++step) {
    e = sc::grouped_lu_panel(st, m->d_items, n, m->nbig_lu, 32 * step, m->max_nb);
    m->launches += 2;
    for (const MxClass& c : m->cls) {
      if (e != cudaSuccess || step >= (int)c.off_t.size()) continue;
      const int rest = c.nb - 32 * step - 32;
      e = mx_products(m, c, c.off_t[step], rest, rest, 32, -1.0f, c.lds, false, c.lds, false, 1.0f, c.lds);
    }
  }
  if (e == cudaSuccess) { e = sc::grouped_finish(st, m->d_items, n, m->max_nb); m->launches += 3; }
  return e;
}

// u = A_ii^-1 (x - xsub) over all classes (interior vectors, slot order).
// The classes' passes run on the classes' streams, forked from and joined back into the
// context's stream.
template <class F>
cudaError_t mx_per_class(sc_mixed* m, F&& launch) {
  cudaError_t e = cudaEventRecord(m->fork, m->stream);
  for (MxClass& c : m->cls) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.st, m->fork, 0);
    if (e == cudaSuccess) e = launch(c);
    if (e == cudaSuccess) e = cudaEventRecord(c.done, c.st);
  }
  for (MxClass& c : m->cls)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->stream, c.done, 0);
  return e;
}

cudaError_t mx_ainv(sc_mixed* m, const double* x, const double* xsub, double* u) {
  return mx_per_class(m, [&](MxClass& c) {
    const long long o = m->ioff[c.slot0];
    k_mx_ainv<<<c.count, 256, 0, c.st>>>(c.ni, c.ldi, c.Ainv32, x + o, xsub ? xsub + o : nullptr, u + o);
    m->launches += 1;
    return cudaGetLastError();
  });
}

// y = S x with two FP32 Jacobian-vector products (x, y boundary vectors).
cudaError_t mx_apply_S(sc_mixed* m, const double* x, double* y) {
  const int nodes = (int)m->nodes;
  const unsigned nbk = mx_blocks(nodes, 256);
  cudaError_t e;
  k_mx_scatter<double><<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, x, nullptr, m->vA);
  if ((e = mx_eval<J1f>(m, m->vA, m->vB)) != cudaSuccess) return e;
  k_mx_gather<<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, m->vB, y, m->ui, 0);
  if ((e = mx_ainv(m, m->ui, nullptr, m->xi)) != cudaSuccess) return e;
  k_mx_scatter<double><<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, nullptr, m->xi, m->vA);
  if ((e = mx_eval<J1f>(m, m->vA, m->vB)) != cudaSuccess) return e;
  k_mx_gather<<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, m->vB, y, nullptr, 1);
  m->launches += 4;
  return cudaGetLastError();
}

// z = blockdiag(S_ee)^-1 v from the FP32 LU factors (or z = v without a preconditioner).
cudaError_t mx_precond(sc_mixed* m, const double* v, double* z) {
  if (m->cfg.precond == SC_PC_NONE)
    return cudaMemcpyAsync(z, v, (size_t)m->nbt * sizeof(double), cudaMemcpyDeviceToDevice, m->stream);
  if (m->prof) {
    while ((int)m->prof_ev.size() < 2 * (m->prof_used + 1)) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return cudaErrorMemoryAllocation;
      m->prof_ev.push_back(ev);
    }
    cudaEventRecord(m->prof_ev[2 * m->prof_used], m->stream);
  }
  cudaError_t e = mx_per_class(m, [&](MxClass& c) {
    const long long o = m->boff[c.slot0];
    m->launches += 1;
    return sc::lu_solve_list32(c.view, c.Sls32, c.rowperm, 0, nullptr, c.count, v + o, nullptr, z + o, nullptr);
  });
  if (m->prof) cudaEventRecord(m->prof_ev[2 * m->prof_used++ + 1], m->stream);
  return e;
}

double mx_norm(sc_mixed* m, const double* v, size_t n) {
  double* slot = m->aux->Hd + 3 * (m->restart + 2);
  sc::multidot(m->aux, v, 1, n, v, slot);
  double h = 0.0;
  cudaMemcpyAsync(&h, slot, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
  cudaStreamSynchronize(m->stream);
  return std::sqrt(h);
}

// Right-preconditioned restarted GMRES (classical Gram-Schmidt twice, Givens rotations) on
// S x = g (m->gb), x0 = 0, into m->xb; stops at ||g - S x|| <= tol or after max_iters.
sc_status mx_gmres(sc_mixed* m, double tol, int max_iters, int* iters_out) {
  sc_ctx* c = m->aux;
  const size_t n1 = m->nbt;
  const int mr = m->restart;
  double* h1 = c->Hd;
  double* h2 = c->Hd + (mr + 1);
  double* hn2 = c->Hd + 2 * (mr + 1);
  MX_CUDA(cudaMemsetAsync(m->xb, 0, n1 * sizeof(double), m->stream));
  MX_CUDA(cudaMemcpyAsync(m->Tb, m->gb, n1 * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  double beta = mx_norm(m, m->Tb, n1);
  std::vector<double> H((size_t)(mr + 1) * mr), cs(mr), sn(mr), gv(mr + 1), hbuf(2 * (mr + 1) + 1), y(mr);
  int iters = 0;
  bool ok = beta <= tol;
  while (!ok && iters < max_iters) {
    MX_CUDA(sc::vec_axpby(c, m->V, 1.0 / beta, m->Tb, 0.0, n1));
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    for (int j = 0; j < mr && iters < max_iters; ++j) {
      MX_CUDA(mx_precond(m, m->V + (size_t)j * n1, m->Zb));
      MX_CUDA(mx_apply_S(m, m->Zb, m->Wv));
      MX_CUDA(sc::multidot(c, m->V, j + 1, n1, m->Wv, h1));
      MX_CUDA(sc::vec_update(c, m->Wv, m->V, j + 1, n1, h1, -1.0));
      MX_CUDA(sc::multidot(c, m->V, j + 1, n1, m->Wv, h2));
      MX_CUDA(sc::vec_update(c, m->Wv, m->V, j + 1, n1, h2, -1.0));
      MX_CUDA(sc::multidot(c, m->Wv, 1, n1, m->Wv, hn2));
      MX_CUDA(cudaMemcpyAsync(hbuf.data(), c->Hd, (2 * (mr + 1) + 1) * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
      MX_CUDA(cudaStreamSynchronize(m->stream));
      for (int i = 0; i <= j; ++i) H[(size_t)i * mr + j] = hbuf[i] + hbuf[(mr + 1) + i];
      const double hn = std::sqrt(std::max(hbuf[2 * (mr + 1)], 0.0));
      H[(size_t)(j + 1) * mr + j] = hn;
      if (!std::isfinite(hn)) return mfail(m, SC_ERR_NONFINITE, "non-finite value in GMRES");
      if (hn > 0) MX_CUDA(sc::vec_axpby(c, m->V + (size_t)(j + 1) * n1, 1.0 / hn, m->Wv, 0.0, n1));
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * mr + j], b = H[(size_t)(i + 1) * mr + j];
        H[(size_t)i * mr + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * mr + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[(size_t)j * mr + j], b = H[(size_t)(j + 1) * mr + j];
      const double den = std::hypot(a, b);
      cs[j] = a / den; sn[j] = b / den;
      H[(size_t)j * mr + j] = den; H[(size_t)(j + 1) * mr + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++iters; k = j + 1;
      if (std::fabs(gv[j + 1]) <= tol || hn == 0.0) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = gv[i];
      for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * mr + l] * y[l];
      y[i] = s / H[(size_t)i * mr + i];
    }
    MX_CUDA(cudaMemcpyAsync(c->Hd, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    MX_CUDA(cudaMemsetAsync(m->Tb, 0, n1 * sizeof(double), m->stream));
    MX_CUDA(sc::vec_update(c, m->Tb, m->V, k, n1, c->Hd, 1.0));
    MX_CUDA(mx_precond(m, m->Tb, m->Zb));
    MX_CUDA(sc::vec_axpby(c, m->xb, 1.0, m->Zb, 1.0, n1));
    // true residual g - S x
    MX_CUDA(mx_apply_S(m, m->xb, m->Wv));
    MX_CUDA(cudaMemcpyAsync(m->Tb, m->gb, n1 * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    MX_CUDA(sc::vec_axpby(c, m->Tb, -1.0, m->Wv, 1.0, n1));
    beta = mx_norm(m, m->Tb, n1);
    if (!std::isfinite(beta)) return mfail(m, SC_ERR_NONFINITE, "non-finite condensed residual");
    ok = beta <= tol;
  }
  *iters_out = iters;
  return SC_OK;
}

}  // namespace

extern "C" {

sc_status sc_mixed_condense(sc_mixed* m) {
  if (!m) return SC_ERR_ARG;
  if (!m->has_state) return mfail(m, SC_ERR_STATE, "condense before set_state");
  const size_t n = (size_t)m->nodes * 5;
  // residual and lifted gradients of the state; B = -R
  MX_CUDA(mx_eval<double>(m, nullptr, m->Rr));
  MX_CUDA(sc::vec_axpby(m->aux, m->B, -1.0, m->Rr, 0.0, n));
  // the element blocks in FP32, in the layout of the condensation (padding stays zero)
  std::vector<float*> outs;
  for (const CondItem& it : m->items) outs.push_back(const_cast<float*>(it.Aown));
  MX_CUDA(cudaMemcpyAsync(m->d_own_out, outs.data(), outs.size() * sizeof(float*), cudaMemcpyHostToDevice, m->stream));
  MX_CUDA(cudaMemcpyAsync(m->d_elist, m->slot_elem.data(), m->slot_elem.size() * sizeof(int), cudaMemcpyHostToDevice,
                          m->stream));
  for (const MxClass& c : m->cls)
    MX_CUDA(cudaMemsetAsync(c.Aown32, 0, (size_t)c.count * c.ne * c.lda * sizeof(float), m->stream));
  for (long long s0 = 0; s0 < m->K; s0 += m->own_chunk) {
    const int cnt = (int)std::min<long long>(m->own_chunk, m->K - s0);
    MX_CUDA(mx_own_launch<float>(m, m->d_elist + s0, cnt, m->own_scratch, m->own_slot, m->d_own_out + s0, 0));
  }
  const int minus1 = -1;
  MX_CUDA(cudaMemcpyAsync(m->d_status, &minus1, sizeof(int), cudaMemcpyHostToDevice, m->stream));
  MX_CUDA(mx_condense_blocks(m));
  int bad = -1;
  MX_CUDA(cudaMemcpyAsync(&bad, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  MX_CUDA(cudaStreamSynchronize(m->stream));
  if (bad >= SC_TC_TIMEOUT) return mfail(m, SC_ERR_CUDA, "tensor-core wait timed out");
  if (bad >= 0) return mfail(m, SC_ERR_SINGULAR_BLOCK, "singular element block");
  m->condensed = true;
  return SC_OK;
}

// A dQ = -R(Q): FP64 iterative refinement of the global system; each sweep solves the
// condensed system of the current residual (GMRES on S to inner_tol) and back-substitutes.
sc_status sc_mixed_solve(sc_mixed* m, double* dQ, int on_device, sc_solve_stats* st) {
  if (!m || !dQ) return SC_ERR_ARG;
  if (!m->condensed) return mfail(m, SC_ERR_STATE, "solve before condense");
  sc_ctx* c = m->aux;
  const size_t n = (size_t)m->nodes * 5;
  const int nodes = (int)m->nodes;
  const unsigned nbk = mx_blocks(nodes, 256);
  sc_solve_stats S{};
  S.first_bad_element = -1;
  MX_CUDA(cudaMemsetAsync(m->dQ, 0, n * sizeof(double), m->stream));
  MX_CUDA(cudaMemcpyAsync(m->Rr, m->B, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  const double bn = mx_norm(m, m->B, n);
  double rn = bn;
  int total = 0, sweeps = 0;
  const int cap = m->cfg.inner_iters > 0 ? m->cfg.inner_iters : m->cfg.gmres_max_iters;
  while (rn > m->cfg.rel_tol * bn && sweeps < m->cfg.max_refine && total < m->cfg.gmres_max_iters) {
    // condensed right-hand side g = r_b - A_bi A_ii^-1 r_i
    k_mx_gather<<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, m->Rr, m->gb, m->ri, 0);
    MX_CUDA(mx_ainv(m, m->ri, nullptr, m->ui));
    k_mx_scatter<double><<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, nullptr, m->ui, m->vA);
    MX_CUDA(mx_eval<J1f>(m, m->vA, m->vB));
    k_mx_gather<<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, m->vB, m->gb, nullptr, 1);
    m->launches += 3;
    const double gn = mx_norm(m, m->gb, m->nbt);
    int its = 0;
    sc_status s = mx_gmres(m, m->cfg.inner_tol * gn, std::min(cap, m->cfg.gmres_max_iters - total), &its);
    if (s != SC_OK) return s;
    total += its;
    // back-substitution x_i = A_ii^-1 (r_i - A_ib x_b)
    k_mx_scatter<double><<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, m->xb, nullptr, m->vA);
    MX_CUDA(mx_eval<J1f>(m, m->vA, m->vB));
    k_mx_gather<<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, m->vB, nullptr, m->ui, 0);
    MX_CUDA(mx_ainv(m, m->ri, m->ui, m->xi));
    k_mx_scatter<double><<<nbk, 256, 0, m->stream>>>(nodes, m->d_bmap, m->d_imap, m->xb, m->xi, m->vA);
    MX_CUDA(sc::vec_axpby(c, m->dQ, 1.0, m->vA, 1.0, n));
    // FP64 residual of the global system
    MX_CUDA(mx_eval<J1>(m, m->dQ, m->vB));
    MX_CUDA(cudaMemcpyAsync(m->Rr, m->B, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    MX_CUDA(sc::vec_axpby(c, m->Rr, -1.0, m->vB, 1.0, n));
    m->launches += 3;
    rn = mx_norm(m, m->Rr, n);
    ++sweeps;
    if (!std::isfinite(rn)) return mfail(m, SC_ERR_NONFINITE, "non-finite residual");
  }
  MX_CUDA(cudaMemcpyAsync(dQ, m->dQ, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          m->stream));
  MX_CUDA(cudaStreamSynchronize(m->stream));
  S.gmres_iters = total;
  S.refinements = sweeps;
  S.rel_residual = bn > 0 ? rn / bn : 0.0;
  if (st) *st = S;
  if (rn > m->cfg.rel_tol * bn) return mfail(m, SC_ERR_NOT_CONVERGED, "refinement did not reach rel_tol");
  return SC_OK;
}

long long sc_mixed_launch_count(const sc_mixed* m) { return m ? m->launches + (m->aux ? m->aux->launches : 0) : 0; }

sc_status sc_mixed_profile(sc_mixed* m, int on) {
  if (!m) return SC_ERR_ARG;
  m->prof = on != 0;
  m->prof_used = 0;
  return SC_OK;
}

sc_status sc_mixed_profile_read(sc_mixed* m, int* count, double* ms_total, double* bytes_each) {
  if (!m || !count || !ms_total || !bytes_each) return SC_ERR_ARG;
  MX_CUDA(cudaStreamSynchronize(m->stream));
  double ms = 0.0;
  for (int i = 0; i < m->prof_used; ++i) {
    float t = 0.f;
    MX_CUDA(cudaEventElapsedTime(&t, m->prof_ev[2 * i], m->prof_ev[2 * i + 1]));
    ms += t;
  }
  double b = 0.0;  // per application: the FP32 factors, the row permutation, v in and z out
  for (const MxClass& c : m->cls) b += (double)c.count * (4.0 * c.nb * c.lds + 4.0 * c.nb + 16.0 * c.nb);
  *count = m->prof_used;
  *ms_total = ms;
  *bytes_each = b;
  return SC_OK;
}

}  // extern "C"
