// Time marching of the GL-DGSEM towards a steady state (Sec. 4, numerical example).
//
// The paper compares three ways of driving the discretisation to a steady state,
// measured by ||M^-1 H(Q)||_inf (M the diagonal GL mass matrix, H the spatial operator
// of eq. DGSEMsystem):
//   * explicit: Williamson's low-storage third-order Runge-Kutta scheme (two registers
//     per dof) on dQ/dt = -M^-1 H(Q), the time step adapted to the CFL condition at every
//     step;
//   * implicit: BDF1 with a fixed time step, each step one Newton-linearised solve
//     (M/dt + dH/dQ) dQ = -H(Q) with a Jacobian computed once and reused;
//   * implicit with static condensation (the same solve through eqs. SC_step1/SC_step2),
//     which is what sc_solve does here.
// The convergence rate eta = d log ||M^-1 H||_inf / d tau (tau the compute time) is read off
// the residual histories these calls return.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sc_internal.cuh"

namespace {

#define MC_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess) { c->err = std::string(#call) + ": " + cudaGetErrorString(_e); return SC_ERR_CUDA; } \
  } while (0)

constexpr int kThreads = 256;
constexpr int kBlocks = 4 * 152;

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block maximum of a non-negative value, folded into *out with an integer atomicMax
// (non-negative IEEE doubles order like their bit patterns; NaN is mapped to +inf).
__device__ void block_max_into(double v, unsigned long long* out) {
  __shared__ double red[kThreads / 32];
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
    w = warp_max(w);
    if (threadIdx.x == 0 && out) atomicMax(out, (unsigned long long)__double_as_longlong(w));
  }
}

// rhs = B / (J W_j), B = -H(Q): the right-hand side -M^-1 H(Q) of the semi-discrete system;
// max |rhs| (the steady-state residual ||M^-1 H||_inf) into *rmax.  rhs may be null.
__global__ void __launch_bounds__(kThreads) k_rhs(Geo G, const double* __restrict__ B, double* __restrict__ rhs,
                                                  unsigned long long* rmax) {
  const size_t n = (size_t)G.K * G.nn * 5;
  double mx = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)((t / 5) % G.nn);
    const int i0 = j % G.p, i1 = (j / G.p) % G.p, i2 = j / (G.p * G.p);
    const double MJ = G.Jf * 0.5 * G.h * G.w[i0] * G.w[i1] * G.w[i2];
    const double v = B[t] / MJ;
    if (rhs) rhs[t] = v;
    mx = (v == v) ? fmax(mx, fabs(v)) : INFINITY;
  }
  block_max_into(mx, rmax);
}

// Largest signal speed |v| + c and largest diffusivity max(4/3, gamma/Pr) mu / (rho Re) over
// all nodes (App. B nondimensionalisation: p = (gamma - 1)(rho E - rho |v|^2 / 2),
// c^2 = gamma p / rho, T = gamma Ma^2 p / rho, Sutherland mu(T)).
__global__ void __launch_bounds__(kThreads) k_speeds(Geo G, const double* __restrict__ Q,
                                                     unsigned long long* __restrict__ out) {
  const size_t nodes = (size_t)G.K * G.nn;
  double smax = 0.0, nmax = 0.0;
  const double dcoef = fmax(4.0 / 3.0, G.gamma / G.Pr) / G.Re;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nodes; t += (size_t)gridDim.x * blockDim.x) {
    const double* q = Q + t * 5;
    const double ir = 1.0 / q[0];
    const double u = q[1] * ir, v = q[2] * ir, w = q[3] * ir;
    const double vv = u * u + v * v + w * w;
    const double p = (G.gamma - 1.0) * (q[4] - 0.5 * q[0] * vv);
    const double s = sqrt(vv) + sqrt(G.gamma * p * ir);
    double mu = 1.0;
    if (G.sutherland) {
      const double T = G.gamma * G.Ma * G.Ma * p * ir;
      mu = (1.0 + G.Ts) * T * sqrt(T) / (T + G.Ts);
    }
    const double nu = dcoef * mu * ir;
    smax = (s == s) ? fmax(smax, s) : INFINITY;
    nmax = (nu == nu) ? fmax(nmax, nu) : INFINITY;
  }
  block_max_into(smax, out);
  __syncthreads();
  block_max_into(nmax, out + 1);
}

// dt = min(cfl (h/N) / smax, dfl (h/N)^2 / numax) (dfl <= 0: no diffusive limit); clears
// the speed maxima for the next step.
__global__ void k_dt(Geo G, double cfl, double dfl, unsigned long long* spd, double* dt_out) {
  const double smax = __longlong_as_double((long long)spd[0]);
  const double nmax = __longlong_as_double((long long)spd[1]);
  const double dx = G.h / G.N;
  double dt = cfl * dx / smax;
  if (dfl > 0.0 && nmax > 0.0) dt = fmin(dt, dfl * dx * dx / nmax);
  *dt_out = dt;
  spd[0] = 0ull;
  spd[1] = 0ull;
}

// One stage of the two-register scheme: dq <- a dq + dt rhs, q <- q + b dq.
__global__ void __launch_bounds__(kThreads) k_rk_stage(size_t n, double a, double b, const double* __restrict__ rhs,
                                                       const double* __restrict__ dtp, double* __restrict__ dq,
                                                       double* __restrict__ q) {
  const double dt = *dtp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double d = a * dq[t] + dt * rhs[t];
    dq[t] = d;
    q[t] += b * d;
  }
}

__global__ void k_axpy(size_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] += a * x[t];
}

// Williamson (1980), low-storage RK3: A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15).
constexpr double kRkA[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
constexpr double kRkB[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

double bits_to_double(unsigned long long b) {
  double d;
  static_assert(sizeof(d) == sizeof(b), "64-bit doubles");
  std::memcpy(&d, &b, sizeof(d));
  return d;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

sc_status state_checks(sc_ctx* c, int nsteps) {
  if (!c) return SC_ERR_ARG;
  if (nsteps < 0) { c->err = "march: nsteps >= 0"; return SC_ERR_ARG; }
  if (!c->has_mesh || !c->has_state) { c->err = "march needs mesh and state"; return SC_ERR_STATE; }
  return SC_OK;
}

}  // namespace

extern "C" {

sc_status sc_steady_residual(sc_ctx* c, double* res_inf) {
  sc_status s = state_checks(c, 0);
  if (s != SC_OK) return s;
  if (!res_inf) return SC_ERR_ARG;
  const Geo& G = c->G;
  Geo Gs = G;
  Gs.c0 = 0.0;
  DevBuf r;
  MC_CUDA(cudaMalloc(&r.p, sizeof(unsigned long long)));
  MC_CUDA(cudaMemsetAsync(r.p, 0, sizeof(unsigned long long), c->stream));
  MC_CUDA(sc::launch_residual_geo(c, Gs, c->Q, c->Q, c->Rfull));
  count_launch(c);
  k_rhs<<<kBlocks, kThreads, 0, c->stream>>>(Gs, c->Rfull, nullptr, (unsigned long long*)r.p);
  unsigned long long b = 0;
  MC_CUDA(cudaMemcpyAsync(&b, r.p, sizeof(b), cudaMemcpyDeviceToHost, c->stream));
  MC_CUDA(cudaStreamSynchronize(c->stream));
  *res_inf = bits_to_double(b);
  return SC_OK;
}

sc_status sc_explicit_march(sc_ctx* c, double cfl, double dfl, int nsteps, double* res_hist, double* dt_hist,
                            double* ms_total) {
  sc_status s = state_checks(c, nsteps);
  if (s != SC_OK) return s;
  if (!(cfl > 0.0)) { c->err = "explicit march: cfl > 0"; return SC_ERR_ARG; }
  const Geo& G = c->G;
  const size_t dofs = (size_t)G.K * G.ne;
  Geo Gs = G;
  Gs.c0 = 0.0;  // the spatial operator alone
  DevBuf dq, rhs, r, spd, dtv;
  MC_CUDA(cudaMalloc(&dq.p, dofs * sizeof(double)));
  MC_CUDA(cudaMalloc(&rhs.p, dofs * sizeof(double)));
  MC_CUDA(cudaMalloc(&r.p, (size_t)(nsteps + 2) * sizeof(unsigned long long)));
  MC_CUDA(cudaMalloc(&spd.p, 2 * sizeof(unsigned long long)));
  MC_CUDA(cudaMalloc(&dtv.p, (size_t)std::max(nsteps, 1) * sizeof(double)));
  unsigned long long* rd = (unsigned long long*)r.p;
  double* dqd = (double*)dq.p;
  double* rhsd = (double*)rhs.p;
  double* dtd = (double*)dtv.p;
  MC_CUDA(cudaMemsetAsync(r.p, 0, (size_t)(nsteps + 2) * sizeof(unsigned long long), c->stream));
  MC_CUDA(cudaMemsetAsync(spd.p, 0, 2 * sizeof(unsigned long long), c->stream));
  MC_CUDA(cudaMemsetAsync(dq.p, 0, dofs * sizeof(double), c->stream));
  cudaEvent_t e0, e1;
  MC_CUDA(cudaEventCreate(&e0));
  MC_CUDA(cudaEventCreate(&e1));
  struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{e0, e1};
  MC_CUDA(cudaEventRecord(e0, c->stream));
  for (int st = 0; st < nsteps; ++st) {
    count_launch(c, 2);
    k_speeds<<<kBlocks, kThreads, 0, c->stream>>>(Gs, c->Q, (unsigned long long*)spd.p);
    k_dt<<<1, 1, 0, c->stream>>>(Gs, cfl, dfl, (unsigned long long*)spd.p, dtd + st);
    for (int k = 0; k < 3; ++k) {
      MC_CUDA(sc::launch_residual_geo(c, Gs, c->Q, c->Q, c->Rfull));
      count_launch(c, 2);
      k_rhs<<<kBlocks, kThreads, 0, c->stream>>>(Gs, c->Rfull, rhsd, k == 0 ? rd + st : rd + nsteps + 1);
      k_rk_stage<<<kBlocks, kThreads, 0, c->stream>>>(dofs, kRkA[k], kRkB[k], rhsd, dtd + st, dqd, c->Q);
    }
  }
  MC_CUDA(sc::launch_residual_geo(c, Gs, c->Q, c->Q, c->Rfull));
  count_launch(c);
  k_rhs<<<kBlocks, kThreads, 0, c->stream>>>(Gs, c->Rfull, nullptr, rd + nsteps);
  MC_CUDA(cudaEventRecord(e1, c->stream));
  // the new state is also the BDF1 history of a following implicit step
  MC_CUDA(sc::launch_history(c, c->Q, c->Q));
  MC_CUDA(cudaGetLastError());
  std::vector<unsigned long long> rb(nsteps + 1);
  MC_CUDA(cudaMemcpyAsync(rb.data(), rd, (nsteps + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          c->stream));
  if (dt_hist && nsteps > 0)
    MC_CUDA(cudaMemcpyAsync(dt_hist, dtd, nsteps * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MC_CUDA(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  MC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  if (ms_total) *ms_total = ms;
  if (res_hist)
    for (int i = 0; i <= nsteps; ++i) res_hist[i] = bits_to_double(rb[i]);
  c->assembled = c->condensed = false;  // the state moved: any Jacobian is stale
  if (!std::isfinite(bits_to_double(rb[nsteps]))) { c->err = "explicit march: non-finite residual"; return SC_ERR_NONFINITE; }
  return SC_OK;
}

sc_status sc_implicit_march(sc_ctx* c, double dt, int nsteps, int jacobian_every, int direct, double steady_tol,
                            double* res_hist, double* ms_hist, int* gmres_iters, int* steps_taken) {
  sc_status s = state_checks(c, nsteps);
  if (s != SC_OK) return s;
  if (jacobian_every < 0) { c->err = "implicit march: jacobian_every >= 0"; return SC_ERR_ARG; }
  if (direct != -1 && direct != SC_DIRECT_GLOBAL && direct != SC_DIRECT_CONDENSED) {
    c->err = "implicit march: direct is -1, SC_DIRECT_GLOBAL or SC_DIRECT_CONDENSED";
    return SC_ERR_ARG;
  }
  s = sc_set_timestep(c, dt, 1);
  if (s != SC_OK) return s;
  const Geo& G = c->G;
  const size_t dofs = (size_t)G.K * G.ne;
  Geo Gs = G;
  Gs.c0 = 0.0;
  DevBuf r;
  MC_CUDA(cudaMalloc(&r.p, (size_t)(nsteps + 1) * sizeof(unsigned long long)));
  unsigned long long* rd = (unsigned long long*)r.p;
  MC_CUDA(cudaMemsetAsync(r.p, 0, (size_t)(nsteps + 1) * sizeof(unsigned long long), c->stream));
  std::vector<cudaEvent_t> ev(nsteps + 1);
  for (auto& e : ev) MC_CUDA(cudaEventCreate(&e));
  struct Evs { std::vector<cudaEvent_t>& v; ~Evs() { for (auto e : v) if (e) cudaEventDestroy(e); } } evg{ev};
  MC_CUDA(cudaEventRecord(ev[0], c->stream));
  int taken = 0;
  for (int st = 0; st < nsteps; ++st) {
    // BDF1: the history is the state at the start of the step, so R(Q) = H(Q) there
    MC_CUDA(sc::launch_history(c, c->Q, c->Q));
    const bool fresh = st == 0 || (direct >= 0 ? !c->direct_valid : !c->condensed) ||
                       (jacobian_every > 0 && st % jacobian_every == 0);
    if (fresh) {
      s = sc_assemble(c);
      if (s == SC_OK && direct != SC_DIRECT_GLOBAL) s = sc_condense(c);
      if (s == SC_OK && direct >= 0) s = sc_direct_factor(c, direct, nullptr, nullptr);
      if (s != SC_OK) return s;
    } else {
      MC_CUDA(sc::launch_residual(c));  // B = -R(Q) with the frozen Jacobian kept
    }
    count_launch(c);
    k_rhs<<<kBlocks, kThreads, 0, c->stream>>>(Gs, c->B, nullptr, rd + st);
    if (steady_tol > 0.0) {  // stop once the state at the start of the step is steady
      unsigned long long b = 0;
      MC_CUDA(cudaMemcpyAsync(&b, rd + st, sizeof(b), cudaMemcpyDeviceToHost, c->stream));
      MC_CUDA(cudaStreamSynchronize(c->stream));
      if (bits_to_double(b) <= steady_tol) break;
    }
    sc_solve_stats stt{};
    s = direct >= 0 ? sc_direct_solve(c, c->dQn, 1, &stt) : sc_solve(c, c->dQn, 1, &stt);
    if (s != SC_OK) return s;
    if (gmres_iters) gmres_iters[st] = stt.gmres_iters;
    count_launch(c);
    k_axpy<<<kBlocks, kThreads, 0, c->stream>>>(dofs, 1.0, c->dQn, c->Q);
    MC_CUDA(cudaEventRecord(ev[st + 1], c->stream));
    taken = st + 1;
  }
  MC_CUDA(sc::launch_residual_geo(c, Gs, c->Q, c->Q, c->Rfull));
  count_launch(c);
  MC_CUDA(cudaMemsetAsync(rd + taken, 0, sizeof(unsigned long long), c->stream));
  k_rhs<<<kBlocks, kThreads, 0, c->stream>>>(Gs, c->Rfull, nullptr, rd + taken);
  MC_CUDA(sc::launch_history(c, c->Q, c->Q));
  MC_CUDA(cudaGetLastError());
  std::vector<unsigned long long> rb(nsteps + 1);
  MC_CUDA(cudaMemcpyAsync(rb.data(), rd, (nsteps + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                          c->stream));
  MC_CUDA(cudaStreamSynchronize(c->stream));
  if (res_hist)
    for (int i = 0; i <= nsteps; ++i) res_hist[i] = i <= taken ? bits_to_double(rb[i]) : NAN;
  if (ms_hist) {
    ms_hist[0] = 0.0;
    for (int i = 1; i <= nsteps; ++i) {
      float ms = 0.f;
      if (i <= taken) MC_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[i]));
      ms_hist[i] = i <= taken ? ms : NAN;
    }
  }
  if (steps_taken) *steps_taken = taken;
  c->assembled = c->condensed = false;  // the Jacobian belongs to an earlier state
  if (!std::isfinite(bits_to_double(rb[taken]))) { c->err = "implicit march: non-finite residual"; return SC_ERR_NONFINITE; }
  return SC_OK;
}

}  // extern "C"
