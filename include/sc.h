/*
 * sc.h -- C ABI of the GB300 statically condensed GL-DGSEM Newton solver.
 *
 * One Newton linear system of the time-implicit GL-DGSEM discretisation of the 3D
 * compressible Navier-Stokes equations (Roe advective flux, BR1 viscous flux) on a
 * periodic Cartesian mesh, solved by static condensation on one GPU:
 *
 *   A dQ = B,  A = dR/dQ,  B = -R(Q)                       (Sec. 2.1, eq. NewtonLinSys1)
 *   [A_bb A_bi; A_ib A_ii] [Q_b; Q_i] = [B_b; B_i]          (Sec. 3.1, eq. StaticDGSEM_QbQiSystem)
 *   (A_bb - A_bi A_ii^-1 A_ib) Q_b = B_b - A_bi A_ii^-1 B_i (Sec. 2.2, eq. SC_step1)
 *   Q_i = A_ii^-1 (B_i - A_ib Q_b)                          (Sec. 2.2, eq. SC_step2)
 *
 * Index convention ("row-column"): A_bi has rows on element boundaries and columns
 * in element interiors; A_ib the reverse.  (The paper's names swap the two.)
 *
 * Global dof order of every vector crossing this ABI: element-major
 * (e = ex + n*(ey + n*ez)), then node (i + (N+1)*(j + (N+1)*k), i fastest), then the
 * conserved variable (rho, rho u, rho v, rho w, rho E) innermost.  All vectors are
 * double precision.  The boundary/interior permutation is internal.
 *
 * Ownership: the caller owns every array it passes; the library owns all device
 * storage it allocates (Jacobian blocks, factors, Krylov space) and frees it in
 * sc_destroy.  Every call returns an sc_status and never aborts; on failure
 * sc_last_error() describes the cause.  All device work is enqueued on the stream
 * given to sc_create; calls return after that stream has finished the call's work
 * unless stated otherwise.  A context is not thread safe.
 */
#ifndef SC_H
#define SC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sc_ctx sc_ctx;

typedef enum {
  SC_OK = 0,
  SC_ERR_ARG = 1,            /* invalid argument (null pointer, size out of range) */
  SC_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  SC_ERR_OOM = 3,            /* device allocation failed */
  SC_ERR_STATE = 4,          /* calls made out of order (e.g. solve before condense) */
  SC_ERR_SINGULAR_BLOCK = 5, /* a zero pivot in an element block factorisation */
  SC_ERR_NONFINITE = 6,      /* a NaN/Inf appeared in a result */
  SC_ERR_NOT_CONVERGED = 7   /* GMRES / refinement did not reach the tolerance */
} sc_status;

enum { SC_PREC_FP64 = 0, SC_PREC_MIXED = 1 };
enum { SC_FLUX_ROE = 0, SC_FLUX_LF = 1 };
enum { SC_VISC_BR1 = 0, SC_VISC_SIPG = 1 };
/* Preconditioners of the condensed GMRES (the paper uses point Jacobi, Sec. 4):
   SC_PC_BLOCK_JACOBI: z_e = S_ee^-1 v_e per element.
   SC_PC_RED_BLACK: one forward block Gauss-Seidel sweep over the checkerboard colouring of
     the elements (ex + ey + ez even = red): z_r = S_rr^-1 v_r for the red elements, then
     z_b = S_bb^-1 (v_b - sum_n S_bn z_n) for the black ones, the couplings from the implicit
     operator passes (the interior pass, then the boundary pass on the black elements).  About
     1.4 times the work of block Jacobi per application.  On meshes with an odd n the
     periodic wrap joins some face neighbours of one colour; their coupling is then treated as
     in block Jacobi.
   SC_PC_LEARNED (mixed arm): the red-black sweep with the black blocks corrected by a
     network, z_b = (S_bb + C_b)^-1 (...), C_b the per-node 5 x 5 corrections of the network
     (see the learned correction below); block Jacobi is its fallback.
   SC_PC_RB_SCHUR (mixed arm): the red-black sweep with each black block replaced by its
     block of the black Schur complement, D_b = S_bb + C_b,
       C_b[k,l] = -sum over the faces f of b containing k and l of
                  S_(k,k'_f) [S_mm^-1]_(k'_f,l'_f) S_(l'_f,l),
     m the red neighbour across f and k'_f the node of m at the same point as k: the
     eliminated red neighbour's whole face block of its inverse, through the co-located
     couplings.  The forward sweep's preconditioned operator has the spectrum of D^-1 times
     the black Schur complement, so this D takes the red couplings out of the black blocks
     (on the Taylor-Green systems about 0.7 times the sweep's iterations).  sc_condense forms
     the red blocks' inverses (n_b solves per red element with their factors; n_red n_b^2
     floats of device memory) and factorises the corrected black blocks; if that
     factorisation meets a singular block the plain sweep runs. */
enum { SC_PC_BLOCK_JACOBI = 0, SC_PC_NONE = 1, SC_PC_LEARNED = 2, SC_PC_RED_BLACK = 3, SC_PC_RB_SCHUR = 4 };

/* Physics and solver settings (App. B parameters; solver choices of this library). */
typedef struct {
  double gamma;          /* heat capacity ratio (1.4) */
  double Pr;             /* Prandtl number (0.72) */
  double Re;             /* reference Reynolds number */
  double Ma;             /* reference Mach number */
  double Ts;             /* Sutherland temperature / reference temperature (110.4/288.15) */
  int sutherland;        /* 1: Sutherland viscosity law, 0: mu = 1 */
  double roe_delta;      /* Harten entropy-fix width as a fraction of the Roe sound speed (0.05) */
  int precision;         /* SC_PREC_FP64 or SC_PREC_MIXED */
  int precond;           /* SC_PC_BLOCK_JACOBI, SC_PC_NONE, SC_PC_LEARNED, SC_PC_RED_BLACK or
                            SC_PC_RB_SCHUR */
  int gmres_restart;     /* Krylov dimension per cycle (e.g. 30) */
  int gmres_max_iters;   /* total iteration cap */
  int max_refine;        /* mixed arm: cap on FP64 refinement sweeps */
  double rel_tol;        /* target ||B - A dQ||_2 / ||B||_2 on the global system (1e-8) */
  double inner_tol;      /* mixed arm: relative tolerance of each inner condensed solve */
  int tensor_cores;      /* mixed arm: 1 = element Schur products and the LU trailing updates
                            of S_ee on the TF32 tensor cores (tcgen05), 0 = FP32 CUDA cores */
  double learned_min_reduction;  /* SC_PC_LEARNED: a full GMRES restart cycle (all
                            gmres_restart iterations) that reduces the condensed residual by less
                            than this factor (the learned sweep has stagnated) switches the rest
                            of the solve to block Jacobi, the fallback (1.5) */
  int factor_fp16;       /* mixed arm: 1 = keep a copy of the block-Jacobi factors in FP16 for the
                            GMRES preconditioner (FP32 arithmetic; used only when every entry is
                            within the FP16 range, else the FP32 copy), 0 = FP32 only (default 0:
                            at CFL 50 the FP16 factors nearly double the GMRES iterations) */
  int explicit_schur;    /* mixed arm, meshes with n >= 3: 1 = form the Schur blocks W_e over
                            the extended boundary sets (Sec. 2.2) in sc_condense and apply
                            S = A_bb - sum_e P_e^T W_e P_e explicitly in GMRES; 0 = implicit
                            operator (default) */
  int outer_krylov;      /* mixed arm: 0 = FP64 refinement sweeps x += A~^-1 (B - A x) (default);
                            m in [1, gmres_restart] = the inner condensed solves act as a flexible
                            preconditioner of FGMRES(m) on the global FP64 system (each outer step:
                            one inner solve, one FP64 product with A, CGS2 on global vectors).  It
                            converges where the sweeps diverge because the FP32 inner solves are
                            too inexact for the conditioning */
  int inner_iters;       /* mixed arm: cap on the GMRES iterations of one inner condensed solve
                            (0 = no cap; the inner tolerance alone ends it) */
  int interior_fp64;     /* mixed arm, n_i > 136 (N >= 5): 1 = A_ii^-1 by FP64 blocked Gauss-Jordan
                            on the FP64 own blocks, rounded to FP32 for the operator (FP32 rounding
                            instead of the ~3e-5 of the FP32 inverse at N = 6; costs the FP64 pipe
                            and n_i^2 doubles per element); 0 = FP32 Gauss-Jordan (default) */
  int adv_flux;          /* advective numerical flux: SC_FLUX_ROE (Roe with Harten's entropy fix,
                            width roe_delta; default) or SC_FLUX_LF (local Lax-Friedrichs, the
                            paper's experiment, Sec. 4: central flux minus half the larger
                            |u . n| + c of the two states times the jump) */
  int visc_flux;         /* viscous numerical flux (Sec. 2.1; the paper's experiment, Sec. 4, uses the
                            symmetric interior penalty): SC_VISC_BR1 (Bassi-Rebay 1: the average of
                            f^nu at the lifted gradients of both sides; default) or SC_VISC_SIPG
                            (compact: the average of f^nu at each side's own unlifted gradient plus
                            sigma (q- - q+), sigma = ip_penalty (N+1)^2 / (h Re), on all five
                            variables; the volume term keeps the lifted gradient with qhat = {{q}}).
                            SIPG couples an element to its six face neighbours only: the edge
                            couplings of BR1 are exact zeros */
  double ip_penalty;     /* C_IP of the interior-penalty coefficient (> 0; default 1) */
} sc_config;

/* Per-solve statistics filled by sc_solve. */
typedef struct {
  int gmres_iters;          /* total GMRES iterations */
  int refinements;          /* mixed arm: FP64 refinement sweeps, or outer FGMRES steps with
                               outer_krylov; 0 for FP64 */
  double rel_residual;      /* ||B - A dQ||_2 / ||B||_2 recomputed in FP64 after the solve */
  double cond_rel_residual; /* last condensed residual estimate / ||B||_2 */
  double ms_rhs, ms_gmres, ms_backsub, ms_refine;  /* device time per phase */
  int first_bad_element;    /* first element with a singular block, or -1 */
  int learned_fallbacks;    /* SC_PC_LEARNED: 1 if the solve fell back to block Jacobi */
} sc_solve_stats;

/* Fill *cfg with the defaults listed above (Re = 1600, Ma = 0.1, FP64, block Jacobi,
   GMRES(30), 4000 iterations, rel_tol 1e-8, tensor_cores 1, learned_min_reduction 1.5).  Never
   fails for a non-null cfg. */
sc_status sc_default_config(sc_config* cfg);

/* Create a context that enqueues all work on `cuda_stream` (a cudaStream_t, or NULL
   for the legacy default stream) of the current device.  *out receives the handle. */
sc_status sc_create(const sc_config* cfg, void* cuda_stream, sc_ctx** out);

/* Release every device and host resource of the context.  Null is ignored. */
void sc_destroy(sc_ctx* ctx);

/* Human-readable description of the last failure of this context ("" if none). */
const char* sc_last_error(const sc_ctx* ctx);

/* Mesh and order (App. C): periodic n x n x n Cartesian hexahedra on [0, L]^3,
   polynomial order N in every element (2 <= N <= 6 and 1 <= n <= 32; the FP64 arm takes
   N <= 5 and the explicit Schur operator N <= 4, else SC_ERR_ARG).  Allocates all per-mesh
   device storage (SC_ERR_OOM if it does not fit); invalidates any previous state and Jacobian. */
sc_status sc_set_mesh(sc_ctx* ctx, int n, double L, int N);

/* Physical coordinates [K][(N+1)^3][3] of the Gauss-Lobatto nodes (host array). */
sc_status sc_node_coords(sc_ctx* ctx, double* xyz);

/* Newton iterate Q and the time history (eq. ImplicitDisc): Qs = Q at time level s,
   Qsm1 = level s-1 (only read for BDF2; may be NULL for BDF1).  Arrays hold
   K*(N+1)^3*5 doubles in global dof order; on_device != 0 means device pointers. */
sc_status sc_set_state(sc_ctx* ctx, const double* Q, const double* Qs, const double* Qsm1,
                       int on_device);

/* Time step and scheme: bdf = 1 (backward Euler) or 2 (BDF2, needs Qsm1). */
sc_status sc_set_timestep(sc_ctx* ctx, double dt, int bdf);

/* Residual B = -R(Q) (eq. NeqtonEq) and the Jacobian A = dR/dQ (Sec. 2.1.1-2.1.2):
   dense per-element blocks plus the structured neighbour couplings. */
sc_status sc_assemble(sc_ctx* ctx);

/* Static condensation set-up (Sec. 3.2): A_ii^-1 per element, the element Schur
   blocks S_ee = A_bb,ee - A_bi,ee A_ii^-1 A_ib,ee and their LU factors (the block-Jacobi
   preconditioner of the condensed solve). */
sc_status sc_condense(sc_ctx* ctx);

/* Solve A dQ = B: condensed right-hand side (eq. SC_step1), right-preconditioned
   restarted GMRES on S, back-substitution (eq. SC_step2), then the FP64 global residual
   ||B - A dQ|| / ||B||.  The mixed arm wraps this in FP64 iterative refinement.
   dQ receives K*(N+1)^3*5 doubles (device pointer if on_device).  stats may be NULL.
   Returns SC_ERR_NOT_CONVERGED (dQ still written) if rel_tol is not met. */
sc_status sc_solve(sc_ctx* ctx, double* dQ, int on_device, sc_solve_stats* stats);

/* B = -R(Q) from the last sc_assemble (copy out). */
sc_status sc_get_rhs(sc_ctx* ctx, double* B, int on_device);

/* y = A x with the assembled FP64 Jacobian (global dof order). */
sc_status sc_apply_jacobian(sc_ctx* ctx, const double* x, double* y, int on_device);

/* Element e's rows of A restricted to the columns of element c (natural node order,
   row-major (N+1)^3*5 square, host array).  c must be e or a face/edge neighbour of e;
   the block sums every coupling between the two elements.  Test hook. */
sc_status sc_get_jacobian_block(sc_ctx* ctx, int e, int c, double* block);

/* Current state Q [K][(N+1)^3][5] (after sc_set_state or sc_newton_step) into Qout (device
   or host per on_device). */
sc_status sc_get_state(sc_ctx* ctx, double* Qout, int on_device);

/* Condensed right-hand side g = B_b - A_bi A_ii^-1 B_i (Sec. 2.2, eq. SC_step1) of the
   assembled system, in the condensed boundary order (element by element, boundary nodes
   in natural order, 5 variables), K * nb doubles; computed with the context's operator
   precision (FP32 blocks on the mixed arm).  After sc_condense. */
sc_status sc_condensed_rhs(sc_ctx* ctx, double* g, int on_device);

/* Back-substitution (Sec. 2.2, eq. SC_step2): given the condensed solution xb (K * nb),
   Q_i = A_ii^-1 (B_i - A_ib Q_b), and the full update dQ [K][(N+1)^3][5] with Q_b = xb.
   After sc_condense; sc_solve performs the same step internally. */
sc_status sc_backsubstitute(sc_ctx* ctx, const double* xb, double* dQ, int on_device);

/* Newton iterations on the current time step (Sec. 2.1, eq. NeqtonEq): assemble, stop if
   ||R(Q)||_2 <= newton_tol ||R(Q_0)||_2 or after max_newton updates, else condense, solve
   A dQ = -R(Q) to the configured rel_tol and set Q <- Q + dQ.  The Jacobian is recomputed
   every iteration; the history term of sc_set_state is kept.  last: statistics of the last
   linear solve (or NULL); newton_iters: updates applied; newton_rel: final
   ||R|| / ||R_0||.  SC_ERR_NOT_CONVERGED if the tolerance is not reached. */
sc_status sc_newton_step(sc_ctx* ctx, int max_newton, double newton_tol, sc_solve_stats* last, int* newton_iters,
                         double* newton_rel);

/* y_b = S x_b with the condensed operator (boundary dof vectors of length
   K * 5 * (number of boundary nodes), ordered element-major, then boundary node in
   natural order, then variable).  Device pointers.  Test hook. */
sc_status sc_condensed_matvec(sc_ctx* ctx, const double* xb, double* yb);

/* Same result as sc_condensed_matvec (the same operator passes, FP64 or mixed arm), but
   the call allocates nothing: the vectors that link the passes (the interior vector, and
   on the mixed arm the FP32 copy of xb) are kept in a fixed 8 MiB device array compiled
   into the library (held on every GPU that loads the library until the process exits)
   instead of context-owned memory.  The paper has no counterpart.  It is for callers that
   must not allocate device memory at the point of the call, e.g. a solver loop running
   under a memory pool or an allocator that forbids cudaMalloc/cudaFree once the
   simulation is running.
   Limit: the FP64 arm needs 8 K ni bytes (K * interior dofs per element <= 1,048,576;
   N = 4: up to 7,767 elements), the mixed arm 4 K (nb + ni) bytes (<= 2,097,152 floats;
   N = 4: up to 3,355 elements; explicit operator: 4 K nb bytes).  Larger meshes get
   SC_ERR_ARG with a message (checked once the mesh is set, before the condensed state).
   Every call looks up the array's device address with the current device (which must be
   the context's); the first call on a device may load the library's device code, so make
   it before any stream capture.  The call only enqueues work on the context's stream and
   returns without synchronising it.  Every call shares the one array: calls whose work
   overlaps on the GPU (other streams, other contexts, other threads) race and must be
   serialised by the caller.  The array keeps the last call's contents, which no call
   reads (each pass writes what the next one reads).
   xb, yb: device pointers as in sc_condensed_matvec. */
sc_status sc_condensed_matvec_static(sc_ctx* ctx, const double* xb, double* yb);

/* z = P v with the context's condensed preconditioner (block Jacobi, red-black sweep or
   the learned sweep; in the operator precision of the arm), boundary vectors of K nb
   doubles in the condensed order, device pointers, v != z.  After sc_condense.  Test hook. */
sc_status sc_precond_apply(sc_ctx* ctx, const double* v, double* z);

/* Sizes: number of elements, dofs per element, interior and boundary dofs per element. */
sc_status sc_sizes(const sc_ctx* ctx, int* K, int* ne, int* ni, int* nb);

/* Batched C = alpha op(A) op(B) + beta C on the TF32 tensor cores (tcgen05, FP32
   accumulation) for `batch` independent row-major FP32 problems; consecutive problems
   are strideA / strideB / strideC elements apart.  op(A) is M x K: A is stored M x K
   (lda >= K) if transA == 0, else K x M (lda >= M).  op(B) is K x N: B is stored K x N
   (ldb >= N) if transB == 0, else N x K (ldb >= K).  C is M x N (ldc >= N).  The
   building block of the mixed arm's element Schur products and of the trailing
   updates of its blocked LU (Sec. 3.2, matrix-matrix multiplications), exposed for
   testing.  Device pointers; enqueued on cuda_stream and synchronised before return.
   batch <= 65535.  Returns SC_ERR_ARG for bad sizes and SC_ERR_CUDA if a launch failed
   or a tensor-core wait timed out. */
sc_status sc_gemm_tf32(int batch, int M, int N, int K, float alpha, const float* A, long long strideA, int lda,
                       int transA, const float* B, long long strideB, int ldb, int transB, float beta, float* C,
                       long long strideC, int ldc, void* cuda_stream);

/* ---- Direct solves by dense LU (Sec. 4, Tables tab:Advantages and tab:Advantages2) ----
   The paper factorises the Jacobian once with a direct solver, either the global A or the
   condensed S of eq. SC_step1, and compares the factorisation and per-solve times of the two.
   sc_direct_factor forms the dense matrix on the GPU (A from the element blocks and the
   neighbour couplings; S column by column through the condensed operator, S e_j) and
   factorises it, P M = L U with partial pivoting (the first row of largest |a| wins), right
   looking in 64-column panels; the trailing updates run on the TF32 tensor cores on the
   mixed arm with tensor_cores, else on the CUDA cores (FP64 on the FP64 arm).  The mixed arm
   keeps FP32 factors.  ms_form / ms_factor (or NULL): device milliseconds of forming and of
   factorising.  The factors (n^2 values, n = K ne or K nb; SC_ERR_ARG beyond 64 GB) stay in
   the context until the next sc_direct_factor or sc_set_mesh: later assemblies of another
   state leave them as they are (a frozen Jacobian).  SC_ERR_SINGULAR_BLOCK on a zero pivot. */
enum { SC_DIRECT_GLOBAL = 0, SC_DIRECT_CONDENSED = 1 };
sc_status sc_direct_factor(sc_ctx* ctx, int which, double* ms_form, double* ms_factor);

/* Solve A dQ = B (B = -R(Q) of the last sc_assemble) with the factors: global, or condensed
   right-hand side (eq. SC_step1), triangular solves with the factors of S, back-substitution
   (eq. SC_step2).  Sweeps x += M^-1 (B - A x) with the FP64 global residual until rel_tol:
   at most 2 on the FP64 arm, max_refine on the mixed arm (FP32 factors).  stats: refinements
   = sweeps, rel_residual, ms_gmres = the triangular solves, ms_rhs = condensed right-hand
   sides and back-substitutions.  dQ as in sc_solve. */
sc_status sc_direct_solve(sc_ctx* ctx, double* dQ, int on_device, sc_solve_stats* stats);

/* ---- Time marching to a steady state (Sec. 4, numerical example) ------------------
   The paper drives its discretisation to a steady state, ||M^-1 H(Q)||_inf <= tol (M the
   diagonal Gauss-Lobatto mass matrix, H the spatial operator of eq. DGSEMsystem), with an
   explicit low-storage RK3 scheme and with BDF1 steps whose Newton-linearised systems reuse
   one Jacobian, solved globally or by static condensation, and reports the convergence rate
   eta = d log ||M^-1 H||_inf / d tau (tau the compute time; Table tab:Advantages2).  These
   calls march the context's state Q in place (after sc_set_mesh and sc_set_state) and leave
   the BDF1 history equal to the new state; any assembled Jacobian is invalidated. */

/* ||M^-1 H(Q)||_inf of the current state (host double). */
sc_status sc_steady_residual(sc_ctx* ctx, double* res_inf);

/* nsteps steps of Williamson's low-storage third-order Runge-Kutta scheme
   (A = 0, -5/9, -153/128; B = 1/3, 15/16, 8/15) on dQ/dt = -M^-1 H(Q).  Each step's dt is
   adapted to the state on the device: dt = min(cfl (h/N) / max(|v| + c),
   dfl (h/N)^2 / max(max(4/3, gamma/Pr) mu / (rho Re))) (dfl <= 0 drops the diffusive limit).
   res_hist (host, nsteps + 1 or NULL): ||M^-1 H||_inf after 0..nsteps steps; dt_hist (host,
   nsteps or NULL): the steps taken; ms_total: device milliseconds of the march.
   SC_ERR_NONFINITE if the state blows up. */
sc_status sc_explicit_march(sc_ctx* ctx, double cfl, double dfl, int nsteps, double* res_hist, double* dt_hist,
                            double* ms_total);

/* nsteps BDF1 steps of size dt, each one Newton-linearised solve
   A dQ = -R(Q) = -H(Q) (eq. NeqtonEq at the step's start, where Q equals the history), solved
   by sc_solve with the context's configuration (static condensation, FP64 or mixed arm; direct
   = -1) or by the dense factors of sc_direct_solve (direct = SC_DIRECT_GLOBAL: LU of A, or
   SC_DIRECT_CONDENSED: LU of S), Q <- Q + dQ.  The Jacobian is assembled (condensed, factorised)
   at the first step and then every jacobian_every steps (0 = once: the frozen Jacobian of the
   paper's experiment); the other steps only evaluate the residual.  steady_tol > 0 ends the
   march early, before the solve of the first step whose start state has
   ||M^-1 H||_inf <= steady_tol (0: all nsteps).  res_hist (host, nsteps + 1 or NULL):
   ||M^-1 H||_inf at the start of each step taken and after the last (NaN beyond); ms_hist
   (host, nsteps + 1 or NULL): device milliseconds from the start to the end of each step
   (ms_hist[0] = 0, NaN beyond the steps taken); gmres_iters (host, nsteps or NULL): GMRES
   iterations of each solve; steps_taken (or NULL).  A solve that misses rel_tol returns its
   status (SC_ERR_NOT_CONVERGED) and stops the march. */
sc_status sc_implicit_march(sc_ctx* ctx, double dt, int nsteps, int jacobian_every, int direct, double steady_tol,
                            double* res_hist, double* ms_hist, int* gmres_iters, int* steps_taken);

/* ---- Spectrum and condition-number estimate (Sec. 4, Fig. ConditionNumber) ------
   The paper approximates the L2 condition number of the global and of the condensed
   matrix by the ratio of the largest to the smallest eigenvalue modulus, both found by
   shift-and-invert Arnoldi.  sc_spectrum_estimate does the same on the assembled system:
   which = 0 for the global Jacobian A, 1 for the condensed matrix S.  The eigenvalue of
   largest modulus is the largest-modulus Ritz value of m_max Arnoldi steps (classical
   Gram-Schmidt twice) on the matrix; the eigenvalue of smallest modulus is the inverse of
   the largest-modulus Ritz value of m_min Arnoldi steps on the inverse (shift 0), each
   inverse applied by a condensed GMRES solve to relative tolerance inv_tol (A^-1: condensed
   right-hand side, GMRES on S, back-substitution; S^-1: GMRES on S).  Both start from the
   same fixed pseudo-random vector.  out[6] = {Re, Im of the largest, Re, Im of the
   smallest eigenvalue, |largest| / |smallest|, total inner GMRES iterations}.  FP64 arm,
   after sc_condense (SC_ERR_STATE otherwise); 1 <= m_max, m_min <= gmres_restart.  The
   call allocates (m + 1) vectors of the operator's size for the Arnoldi basis and frees
   them before it returns. */
sc_status sc_spectrum_estimate(sc_ctx* ctx, int which, int m_max, int m_min, double inv_tol, double* out);

/* Eigenvalues of an m x m upper Hessenberg matrix H (row-major, host) by the shifted QR
   algorithm in complex arithmetic, the step sc_spectrum_estimate applies to its Arnoldi
   matrices: re[m], im[m] (host).  Host-only; SC_ERR_NOT_CONVERGED if QR does not
   converge. */
sc_status sc_hessenberg_eigvals(int m, const double* H, double* re, double* im);

/* ---- Learned correction of the red-black sweep --------------------------------------
   Not in the paper (which preconditions GMRES on the condensed system with point Jacobi,
   Sec. 4).  With SC_PC_LEARNED the black half of the red-black sweep factorises
   D_b = S_bb + C_b, C_b block diagonal over the 5 x 5 node blocks of the black element b:
     C_k = -1/2 sum over the faces f of b containing k of S_(k,k'_f) Z_(k'_f) S_(k'_f,k),
   k'_f the co-located node of the (red) neighbour across f and Z_(k') the diagonal node block
   of the inverse of that neighbour's face block, [S_nn^-1]_(k'k') (the co-located part of the
   Schur correction that eliminating the red neighbours adds to S_bb, halved).  A network
   predicts the correction of each element's face-block inverse there: from 128 features of
   node k' it gives y, and Z = [S_nn]_(k'k')^-1 + y / ||[S_nn]_(k'k')||_F (the exact Z needs n_b
   unit solves per element); sc_condense applies the output at half weight, y/2 (shrunk
   towards the closed form: the corrected black blocks amplify the network's errors).  Layout of the parameters (shared by every call): weights
   W = [W1 (256 x 128) | W2 (256 x 256) | W3 (25 x 256)], row-major, 104,704 values, kept as
   FP32 masters and as a BF16 copy (IEEE bfloat16 bit patterns in uint16_t); biases
   b = [b1 (256) | b2 (256) | b3 (25)], FP32.  Layers: h1 = relu(W1 x + b1),
   h2 = relu(W2 h1 + b2), y = W3 h2 + b3; FP32 arithmetic.  All pointers are device pointers
   unless stated; work is enqueued on cuda_stream and synchronised before return.
   SC_ERR_ARG for null pointers or bad sizes, SC_ERR_CUDA for launch failures. */

/* y[n x 25] = net(X[n x 128]).  cache: NULL, or 4 n x 256 floats that receive z1, h1, z2,
   h2 (pre- and post-activations) for sc_mlp_backward; with NULL the call allocates
   temporaries on the stream. */
sc_status sc_mlp_forward(const uint16_t* Wbf16, const float* bias, const float* X, int n, float* Y, float* cache,
                         void* cuda_stream);

/* Accumulate the gradients of sum(dY * y) into gW (104,704) and gb (537), FP32, from the
   forward cache of the same X.  work: 2 n x 256 floats of scratch. */
sc_status sc_mlp_backward(const uint16_t* Wbf16, const float* X, const float* cache, const float* dY, int n,
                          float* gW, float* gb, float* work, void* cuda_stream);

/* Loss of Y against targets T (both n x 25): mean over samples of
   ||y - t||^2 / (||t||^2 + 1e-12).  Adds it to *loss_sum (device float) when non-NULL and
   writes its gradient to dY (n x 25) when non-NULL. */
sc_status sc_mlp_loss(const float* Y, const float* T, int n, float* dY, float* loss_sum, void* cuda_stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step >= 1 counts the
   updates) on the FP32 masters W and bias with gradients gW, gb and moments m, v
   (105,241 floats each: weights then biases); refreshes Wbf16 and zeroes gW and gb. */
sc_status sc_mlp_adam(float* W, uint16_t* Wbf16, float* bias, float* gW, float* gb, float* m, float* v, int step,
                      float lr, void* cuda_stream);

/* W16[i] = W[i] rounded to bfloat16 (nearest even), i < n: the BF16 copy of FP32 weights. */
sc_status sc_mlp_bf16(const float* W, uint16_t* Wbf16, int n, void* cuda_stream);

/* Training loop of the network (the learned correction's counterpart of sc_train_mlp):
   `epochs` passes of mini-batch Adam over device samples X [n x 128] with targets T [n x 25].
   Before every pass all n samples are shuffled (Fisher-Yates on a splitmix64 stream seeded
   by `seed`), so every batch mixes systems, elements and nodes; each batch of `batch` samples
   (the last may be smaller) runs sc_mlp_forward, sc_mlp_loss, sc_mlp_backward and one
   sc_mlp_adam step.  W, Wbf16, bias, m, v as for sc_mlp_adam; *step (host) counts the Adam
   updates and carries on across calls (start at 0).  loss_hist (host, epochs floats, or
   NULL): mean batch loss of each pass.  The call allocates its batch buffers and frees
   them before it returns. */
sc_status sc_mlp_train(float* W, uint16_t* Wbf16, float* bias, float* m, float* v, int* step, const float* X,
                       const float* T, int n, int epochs, int batch, float lr, uint64_t seed, float* loss_hist,
                       void* cuda_stream);

/* Network parameter files: the 8 bytes "SCMLP001", the counts 104,704 and 537 (int32), then
   the FP32 weights W and biases (little endian).  sc_mlp_save writes device W, bias;
   sc_mlp_load reads them into device W, its BF16 copy and bias (SC_ERR_ARG if the file is
   missing or not such a file). */
sc_status sc_mlp_save(const char* path, const float* W, const float* bias);
sc_status sc_mlp_load(const char* path, float* W, uint16_t* Wbf16, float* bias);

/* Load a saved network into the context as its SC_PC_LEARNED weights (sc_set_learned_weights
   of the file's parameters). */
sc_status sc_load_mlp(sc_ctx* ctx, const char* path);

/* Features of the learned correction for every (element e, boundary node k) of the
   condensed system, samples ordered element by element and boundary node by boundary
   node (the condensed order).  With k' the node at the same point in the neighbour n across
   the lowest-index face of e containing k (order -x,+x,-y,+y,-z,+z) and k'' the node at the
   same point in the neighbour across the lowest face of n containing k' (k itself for a node
   on one face only): F[s][128] = q_k over free-stream scales (rho, rho u, rho v, rho w over 1,
   rho E over p_inf/(gamma-1) + 1/2) | [S_ee]_kk | S_(k,k') | S_(k',k'') | [S_nn]_(k'k') (each
   row-major 5 x 5 over its Frobenius norm) | Ma, Re/1000, dt/(Ma h), N | (faces of e containing
   k) / 3 | the Frobenius norms of S_(k,k'), S_(k',k''), [S_nn]_(k'k') over that of [S_ee]_kk |
   0 x 15; snorm[s] = ||[S_ee]_kk||_F.  After sc_condense on the mixed arm (SC_ERR_STATE
   otherwise).  Device pointers, K * nbn * 128 and K * nbn floats. */
sc_status sc_learned_features(sc_ctx* ctx, float* F, float* snorm);

/* Training targets T[s][25] = ([S_ee^-1]_kk - [S_ee]_kk^-1) ||[S_ee]_kk||_F for every sample
   (row-major 5 x 5; elements of both colours): the correction of the inverse of the node block
   to the node block of the face-block inverse, [S_ee^-1]_kk from unit solves with the
   condensation's factors.  After sc_condense on the mixed arm.  Device pointer, K * nbn * 25
   floats. */
sc_status sc_learned_targets(sc_ctx* ctx, float* T);

/* Network parameters for SC_PC_LEARNED (device pointers, layout of sc_mlp_forward; copied
   into the context).  With precond = SC_PC_LEARNED, sc_condense evaluates the network on the
   features of every boundary node, assembles the black blocks' corrections C from half its
   outputs and factorises
   S_bb + C apart from the plain factors, which block Jacobi (the fallback) keeps using. */
sc_status sc_set_learned_weights(sc_ctx* ctx, const uint16_t* Wbf16, const float* bias);

/* Measurement hook for SC_PC_LEARNED: after sc_condense, assemble the black corrections from
   scale * Y instead of the network's outputs (device, K * nbn * 25 floats in the target form
   of sc_learned_targets) and refactorise the black blocks, e.g. with the exact targets, to
   measure what a perfect network would give. */
sc_status sc_set_learned_correction(sc_ctx* ctx, const float* Y, float scale);

/* ---- Batched condensation of elements of uneven order ---------------------------
   Not in the paper: the condensation set-up (A_ii^-1, Y, S_ee, LU of S_ee, solve layout;
   Sec. 2.2 eq. StaticCondBlock) of several assembled systems, each of one order N (mixed
   arm, block Jacobi, tensor cores, FP32 factors and interior inverses, implicit operator, one
   shared stream), run
   together: the per-element steps as grouped launches over all elements of all orders, the
   TF32 products per order through tables of block addresses.  After sc_batch_condense each
   system is condensed exactly as by its own sc_condense and is solved with sc_solve. */
typedef struct sc_batch sc_batch;
enum { SC_BATCH_GRAPH = 1,    /* capture the sequence into a CUDA graph once, then replay it */
       SC_BATCH_AUTOTUNE = 2  /* first call: time the N-tile widths 64/144/256 of every product on
                                 the batch's data and keep the fastest per order */ };

/* Create a batch over nctx contexts (meshes set; SC_ERR_ARG if one is not as listed above or
   uses another stream).  The contexts must outlive the batch and keep their meshes; the
   batch owns a stream of its own, ordered after the contexts' stream at every call. */
sc_status sc_batch_create(sc_ctx* const* ctxs, int nctx, sc_batch** out);

/* Condense every system of the batch (each assembled, SC_ERR_STATE otherwise); flags:
   SC_BATCH_GRAPH | SC_BATCH_AUTOTUNE.  Synchronous.  On failure the message is in
   sc_last_error of the first context. */
sc_status sc_batch_condense(sc_batch* batch, int flags);

/* Tile widths in use for order class c (classes in order of first appearance): the
   interior size ni of the class and the N-tile widths of the Y^T, S_ee and trailing-update
   products. */
sc_status sc_batch_tiles(const sc_batch* batch, int c, int* ni, int* bn_y, int* bn_s, int* bn_t);

void sc_batch_destroy(sc_batch* batch);

/* ---- One mesh of mixed polynomial order ------------------------------------------
   A periodic n^3 mesh of side L whose element e = ex + n (ey + n ez) has its own order
   orders[e] in 2..6 (the paper treats one order per mesh; this is its uneven-order case).
   A face between two orders is a mortar: the traces of both sides (state and lifted
   gradient) are interpolated to the Gauss-Lobatto nodes of the larger order, qhat (BR1)
   and fhat (Roe or local Lax-Friedrichs, cfg->adv_flux) are formed there point by point,
   and each side takes their L2 projection onto its own face polynomials (Gauss rule of
   M + 1 points).  force_mortar = 1 routes faces between equal orders through the mortar
   too.  States are ragged: element by element, (N_e+1)^3 nodes of 5 variables in natural
   node order (i fastest), flat doubles.
   Only the mixed arm: cfg->precision = SC_PREC_MIXED, cfg->precond SC_PC_BLOCK_JACOBI or
   SC_PC_NONE, cfg->visc_flux = SC_VISC_BR1; SC_ERR_ARG otherwise, or for n outside [2, 32],
   an order outside 2..6 or L <= 0.  The context keeps cuda_stream; every call is
   synchronous and reports errors as the calls above do (message: sc_mixed_last_error). */
typedef struct sc_mixed sc_mixed;
sc_status sc_mixed_create(const sc_config* cfg, void* cuda_stream, int n, double L, const int* orders,
                          int force_mortar, sc_mixed** out);
void sc_mixed_destroy(sc_mixed* m);
const char* sc_mixed_last_error(const sc_mixed* m);
/* Totals of the ragged layouts: nodes, boundary dofs, interior dofs. */
sc_status sc_mixed_sizes(const sc_mixed* m, long long* nodes, long long* nb_total, long long* ni_total);
/* Newton state Q, history Qs (and Qsm1 for BDF2), time step dt > 0, bdf 1 or 2; host
   pointers, or device pointers when on_device = 1. */
sc_status sc_mixed_set_state(sc_mixed* m, const double* Q, const double* Qs, const double* Qsm1, double dt, int bdf,
                             int on_device);
/* R(Q) of eq. NeqtonEq (time term included), ragged layout. */
sc_status sc_mixed_residual(sc_mixed* m, double* R, int on_device);
/* y = (dR/dQ)(Q) x by forward-mode dual numbers in FP64 (eq. NewtonLinSys1, exact to rounding). */
sc_status sc_mixed_jvp(sc_mixed* m, const double* x, double* y, int on_device);
/* dR_e/dQ_e of element e in FP64, natural node order, 5 (N_e+1)^3 square, row-major, into
   the host array block. */
sc_status sc_mixed_own_block(sc_mixed* m, int e, double* block);
/* Static condensation set-up (Sec. 2.2): element blocks in FP32 by five-direction duals,
   then A_ii^-1 (Gauss-Jordan), S_ee = A_bb - A_bi A_ii^-1 A_ib (TF32 tensor cores) and the
   blocked LU of S_ee, grouped over all elements of all orders.  SC_ERR_SINGULAR_BLOCK if a
   block is singular. */
sc_status sc_mixed_condense(sc_mixed* m);
/* Solve A dQ = -R(Q) (after sc_mixed_condense): FP64 iterative refinement of the global
   system to cfg->rel_tol (at most cfg->max_refine sweeps); each sweep solves the condensed
   system of the current residual by right-preconditioned GMRES(gmres_restart) to
   cfg->inner_tol, with S applied through two FP32 Jacobian-vector products and the FP32
   A_ii^-1, and back-substitutes the interior values.  SC_ERR_NOT_CONVERGED (dQ still
   written) if rel_tol is not reached. */
sc_status sc_mixed_solve(sc_mixed* m, double* dQ, int on_device, sc_solve_stats* stats);
/* Kernel launches made by the context so far. */
long long sc_mixed_launch_count(const sc_mixed* m);
/* Measurement hook (not part of the method): with on = 1, every block-Jacobi application of
   the following solves is bracketed by events (the counter restarts).  profile_read
   synchronises and returns the number of applications, their total device time and the
   bytes one application moves by its algorithm (FP32 factors n_b x lds, row permutation,
   FP64 right-hand side in and result out, summed over the elements). */
sc_status sc_mixed_profile(sc_mixed* m, int on);
sc_status sc_mixed_profile_read(sc_mixed* m, int* count, double* ms_total, double* bytes_each);

/* ---- Measurement hooks (not part of the method; used by the benchmark) ---------- */

/* Kernel ids for sc_profile_kernel / sc_kernel_work. */
enum { SC_KERNEL_COND_INTERIOR = 0, SC_KERNEL_COND_BOUNDARY = 1, SC_KERNEL_LU_SOLVE = 2,
       SC_KERNEL_LU = 3, SC_KERNEL_SCHUR_GEMM = 4, SC_KERNEL_GJ_INV = 5, SC_KERNEL_ASSEMBLE_OWN = 6,
       SC_KERNEL_GLOBAL_APPLY = 7, SC_KERNEL_EXPLICIT_GEMM = 8 /* Y_e and W_e products */,
       SC_KERNEL_EXPLICIT_APPLY = 9 /* W_e part of the explicit matvec */ };

/* Total number of kernels this context has launched since sc_create. */
sc_status sc_launch_count(const sc_ctx* ctx, long long* count);

/* Start timing every launch of one kernel with CUDA events on the context's stream
   (kernel_id = -1 stops); resets the accumulated totals. */
sc_status sc_profile_kernel(sc_ctx* ctx, int kernel_id);

/* Launches and total device milliseconds of the profiled kernel since sc_profile_kernel
   (synchronises the stream). */
sc_status sc_profile_read(sc_ctx* ctx, long long* launches, double* total_ms);

/* Elements processed by the launches of the profiled kernel since sc_profile_kernel (a
   launch over every element counts K; the red-black sweep's launches count one colour). */
sc_status sc_profile_elements(const sc_ctx* ctx, long long* elements);

/* Algorithmic work of one launch of a kernel over every element of the current mesh:
   floating-point operations and bytes that must move (matrix entries read once, vectors
   once); per element, divide by K. */
sc_status sc_kernel_work(const sc_ctx* ctx, int kernel_id, double* flops, double* bytes);

/* ---- Element partitions of a sharded run (host only; no GPU work, no context) ----
   Not in the paper.  The condensation is element-local (Sec. 2.2), so a run on several GPUs
   gives each rank whole elements; one application of the implicit condensed operator then
   needs two halo exchanges: the boundary values x_b of the face and edge neighbours of the
   owned elements (before the interior pass) and the interior values u of their face
   neighbours (before the boundary pass).  This build runs one GPU per process (replicas);
   these calls give the layout a sharded run would use. */

/* part[e] (K = n^3 ints, caller-owned) = the rank of element e = ex + n (ey + n ez): slabs of
   whole z-planes, rank r owning planes [r n / nparts, (r + 1) n / nparts).  SC_ERR_ARG unless
   1 <= nparts <= n <= 32. */
sc_status sc_partition_slabs(int n, int nparts, int* part);

/* For rank `rank` of the partition part[K]: counts[0..2] = the numbers of owned elements,
   of elements whose boundary values the owned rows need (halo_b: face and edge neighbours
   not owned) and of elements whose interior values they need (halo_u: face neighbours not
   owned); owned, halo_b, halo_u (each K ints, caller-owned) receive those element indices in
   ascending order.  SC_ERR_ARG for null pointers or a bad n. */
sc_status sc_partition_halo(int n, const int* part, int rank, int* counts, int* owned, int* halo_b, int* halo_u);

#ifdef __cplusplus
}
#endif
#endif /* SC_H */
