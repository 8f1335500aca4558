/*
 * lbo.h -- C ABI of the GB300 (sm_103a) fast Fourier spectral linearized
 * Boltzmann collision operator library (liblbo.so).
 *
 * Method: T. Yin, Z. Cai, Y. Wang, "A fast Fourier spectral method for the
 * linearized Boltzmann collision operator", arXiv 2503.09580.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  N points per velocity direction (N even; the paper's N is N/2),
 *   periodic box [-L, L]^3, spacing h = 2L/N, collocation points
 *   v_i = (i - N/2) h for i = 0..N-1 (Sec. 2.3: v_l = l L / N_p,
 *   l = -N_p..N_p-1).  A velocity field is N^3 doubles, row-major
 *   [i1][i2][i3]; a batch is [batch][i1][i2][i3].
 * Maxwellian parameters.  params[b*5 + 0..4] = (rho, u1, u2, u3, theta):
 *   M(v) = rho (2 pi theta)^{-3/2} exp(-|v-u|^2 / (2 theta))  (Sec. 2.1).
 * Collision kernel.  Variable hard spheres, B(g) = C g^{2(1-omega)} for
 *   g <= R and 0 beyond (Eq. (2.4), Sec. 2.3); C = 1/(4 pi) by default
 *   (Eq. (4.1)), R = 4L/(3+sqrt 2) by default (the dealiasing bound).
 * Memory.  Array arguments are caller-owned.  Each may be a device pointer
 *   (CUDA global memory of the plan's device) or a host pointer; host
 *   arrays are staged through plan-owned device buffers with copies on the
 *   plan's stream, and such a call returns only after the result is back
 *   in host memory.  Device-pointer calls are asynchronous on the plan's
 *   stream; the plan owns its tables and workspace.
 * Precision.  Inputs and outputs are FP64 in every mode; LBO_OPT_PRECISION
 *   selects the arithmetic of the transforms and pointwise products.
 * Errors.  Every call returns an lbo_status.  Argument errors are detected
 *   before any launch; CUDA errors map to LBO_ECUDA and the CUDA error text
 *   is available from lbo_last_error().  A plan is not thread-safe.
 */
#ifndef LBO_H
#define LBO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbo_plan lbo_plan;

typedef enum {
  LBO_OK = 0,
  LBO_EINVAL = 1,        /* bad argument (size, pointer, option value)      */
  LBO_ENOMEM = 2,        /* device or host allocation failed                */
  LBO_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed     */
  LBO_ENOTCONV = 4,      /* iterative solve stopped at its iteration cap    */
  LBO_EBREAKDOWN = 5,    /* Krylov breakdown                                */
  LBO_ENAN = 6,          /* non-finite value detected                       */
  LBO_EUNSUPPORTED = 7,  /* combination of N / precision not built          */
  LBO_ETIMEOUT = 8       /* a kernel gave up a bounded wait (tensor-core
                            path: an MMA completion); the results of the
                            call are not valid                             */
} lbo_status;

typedef enum {
  LBO_PREC_FP64 = 0,     /* FP64 transforms and products (the plain path)   */
  LBO_PREC_FP32 = 1,     /* FP32 transforms and products, FP64 in/out,
                            FP64 Maxwellians, cut-off and final combination */
  LBO_PREC_FP32X2 = 2,   /* transforms and products in pairs of FP32 numbers
                            (hi + lo, about 48 significant bits, FP32
                            exponent range) on the FP32 pipe; FP64
                            Maxwellians, ratio, cut-off and combination     */
  LBO_PREC_FP64X2 = 3,   /* transforms and products in pairs of FP64 numbers
                            (about 106 significant bits): the higher-
                            precision convolution of Sec. 3.4 (the paper
                            uses binary128), accurate without the cut-off
                            where FP64 transforms lose max|r| u digits;
                            N = 16 and 32                                  */
  LBO_PREC_BF16_SPLIT = 4,/* every transform a dense DFT contraction on the
                            tensor cores (tcgen05.mma, FP32 accumulation):
                            data and DFT matrix split into BF16 hi + lo
                            parts, three products (~2^-16 per transform);
                            FP32 fields between transforms; L only;
                            N = 16, 32, 64                                 */
  LBO_PREC_FP16_SPLIT = 5 /* the same with FP16 parts (~2^-22 per transform),
                            each pencil scaled by a power of two            */
} lbo_precision;

typedef enum {
  LBO_OPT_R = 0,           /* kernel cut-off R (double)                       */
  LBO_OPT_C = 1,           /* kernel constant C                               */
  LBO_OPT_EPS = 2,         /* cut-off level epsilon of Eq. (3.9), 1e-9        */
  LBO_OPT_CUTOFF = 3,      /* 1: apply Eq. (3.9) to r = g/M (default), 0: no  */
  LBO_OPT_MASS_FIX = 4,    /* 1: set the zero mode of the output to 0 (Sec 4.2)*/
  LBO_OPT_MOMENT_FIX = 5,  /* 1: FP64 projection of the output onto zero mass,
                              momentum and energy (least squares on the grid) */
  LBO_OPT_HEMISPHERE_P = 6,/* hemisphere rule order p: M = 2 p^2 points (4)   */
  LBO_OPT_PRECISION = 7,   /* lbo_precision                                   */
  LBO_OPT_KERNEL = 8,      /* 0: fastest built kernel set for (N, precision)
                              (default), 1: the generic plane/axis kernels,
                              2: the generic kernels with every transform a
                              two-stage shared-memory FFT (FP64 at N = 32
                              otherwise runs the hot kernels of L and of
                              Q(f,f) with one thread per pencil in
                              registers)                                      */
  LBO_OPT_JGROUPS = 9,     /* radial nodes per CTA of the fused FP32 kernel are
                              J / jgroups; 0 (default): chosen from the batch */
  LBO_OPT_Q_SINC_QUADRATURE = 10, /* Q(f,f) only.  1: the loss multiplier
                              sum_j w_j B(g_j) sinc(pi g_j |k| / L) replaced by
                              its hemisphere quadrature
                              sum_m w_m cos(pi g_j sigma_m . k / L), the
                              second mass fix of Sec. 2.3 (Eq. (2.16)): Q^_0
                              vanishes up to rounding.  Takes the generic
                              kernels (also for FP32 at N = 32); 0: off   */
  LBO_OPT_PLANES = 11      /* planes per CTA of the FP64 register plane kernel
                              at N = 32 (2, 4 or 8; 0: default, 4): the tile
                              shape lbo_plan_autotune picks for FP64        */
} lbo_option;

/* Create a plan for N^3 grids on [-box, box]^3, VHS exponent vhs_omega in
 * [0.5, 1], radial_nodes Gauss-Legendre nodes on [0, R] (Eq. (2.13)).
 * Builds the tables of Algorithm 1 (its precomputation step) on the current
 * CUDA device.  N must be 16, 24, 32, 48 or 64.  On success *out owns device memory
 * until lbo_plan_destroy.  Errors: LBO_EINVAL, LBO_EUNSUPPORTED, LBO_ENOMEM,
 * LBO_ECUDA (then *out is NULL). */
lbo_status lbo_plan_create(int N, double box, double vhs_omega, int radial_nodes,
                           lbo_plan **out);

/* Set an option.  Options that change the tables (R, C, hemisphere order)
 * rebuild them at the next apply.  LBO_EINVAL for an unknown key or an
 * out-of-range value. */
lbo_status lbo_plan_set(lbo_plan *plan, lbo_option key, double value);

/* Use this CUDA stream (a cudaStream_t passed as void*; NULL = the legacy
 * default stream) for every launch and copy of the plan. */
lbo_status lbo_plan_set_stream(lbo_plan *plan, void *stream);

/* Linearized collision operator, Algorithm 1 ("CollisionOperator"):
 *   out[b] = L_b[g[b]] = Q(M_b, g[b]) + Q(g[b], M_b),
 * M_b the Maxwellian of params[b].  params: batch*5 doubles; g, out:
 * batch*N^3 doubles (out must not alias g or params).  batch >= 0
 * (0 is a no-op).  Point values in, point values out (Sec. 3.5). */
lbo_status lbo_apply_linearized(lbo_plan *plan, const double *maxwellian_params,
                                const double *g, double *out, int batch);

/* Cache the factors of Algorithm 1 that depend on the background
 * Maxwellians only: u^_j = FFT(M^g phit_j) for every radial node and the
 * loss factor InvFFT(FFT(M) omega) (its precomputation of the gain kernel
 * and the second loss convolution, Sec. 3.5).  Later lbo_apply_linearized
 * calls with the same maxwellian_params pointer and batch, the same
 * precision and the same kernel set reuse them instead of recomputing them
 * (for the fused FP32 kernels only u^_j is cached): the Krylov products of
 * one Newton step share their Maxwellians.  params: device pointer,
 * batch*5 doubles; its contents must not change while the cache is in use
 * (the library cannot see such a change: call again, or drop the cache).
 * params = NULL or batch = 0 drops the cache (its device buffers are kept
 * for reuse).  Allocates device memory on first use and when a larger batch
 * needs it: J*batch*(N/2+1)^3 + batch*N^3 reals of the transform precision.
 * Asynchronous on the plan's stream.  Errors: LBO_EINVAL (bad plan, host
 * pointer), LBO_ENOMEM, LBO_ECUDA, LBO_EUNSUPPORTED (N not built for the
 * precision). */
lbo_status lbo_plan_cache_maxwellians(lbo_plan *plan, const double *maxwellian_params, int batch);

/* Quadratic collision operator Q(f,f) in the M-point hemisphere-quadrature
 * form of Eq. (2.14) with the plan's radial rule and a product hemisphere
 * rule of M = 2p^2 points.  f, out: batch*N^3 doubles, no aliasing.
 * Built in FP64, FP32 and the two-fold precisions (LBO_EUNSUPPORTED for the
 * split 16-bit ones). */
lbo_status lbo_apply_quadratic(lbo_plan *plan, const double *f, double *out, int batch);

/* Explicit time integration of the spatially homogeneous equation
 * (Sec. 4.2): df/dt = Q(f,f) (mode LBO_EVOLVE_QUADRATIC) or df/dt = L_M[f]
 * (LBO_EVOLVE_LINEARIZED, M_b the Maxwellian of params[b]; L[M] = 0, so this
 * is the linearized equation for f - M), with the classical fourth-order
 * Runge-Kutta scheme, nsteps steps of size dt, in place on f (device,
 * batch*N^3 doubles).  Every operator evaluation goes through the plan (its
 * precision, kernel set and the mass fixes: LBO_OPT_MASS_FIX sets the zero
 * mode of every evaluation to 0, LBO_OPT_Q_SINC_QUADRATURE the Eq. (2.16)
 * loss of Q).  The linearized form caches the Maxwellian factors for its
 * steps (and drops them afterwards unless the caller had cached them for
 * the same params).  Allocates 3 batch*N^3 stage buffers for the call and
 * synchronizes the plan's stream before returning.  Errors: LBO_EINVAL,
 * LBO_ENOMEM, LBO_ECUDA, and those of the operators. */
typedef enum { LBO_EVOLVE_QUADRATIC = 0, LBO_EVOLVE_LINEARIZED = 1 } lbo_evolve_mode;
lbo_status lbo_evolve_homogeneous(lbo_plan *plan, int mode, const double *maxwellian_params, double *f, int batch,
                                  double dt, int nsteps);

/* Wait for all work queued on the plan's stream; report the first
 * asynchronous CUDA error, if any. */
lbo_status lbo_plan_sync(lbo_plan *plan);

/* Number of kernels the last apply call launched (for accounting). */
int lbo_plan_last_launches(const lbo_plan *plan);

/* Per-kernel timing.  lbo_plan_profile(plan, 1) clears the counters and
 * from then on brackets every kernel launch of the plan with CUDA events on
 * the plan's stream; lbo_plan_profile(plan, 0) stops recording.
 * lbo_plan_profile_count synchronizes the stream, folds the recorded events
 * into per-kernel totals and returns the number of kernel names;
 * lbo_plan_profile_get reads entry i (name is a static string owned by the
 * library).  LBO_EINVAL for a bad plan or index. */
lbo_status lbo_plan_profile(lbo_plan *plan, int enable);
int lbo_plan_profile_count(lbo_plan *plan);
lbo_status lbo_plan_profile_get(lbo_plan *plan, int i, const char **name, int *launches,
                                double *total_ms);

/* ------------------------------------------------------------------------
 * Steady-state / implicit solver (Sec. 5 and the supplement).
 *
 * LBO_PROBLEM_SLAB: the 1-D steady problem v1 d_x f = Q(f,f)/Kn on
 *   (x_left, x_right), nx cells, first-order upwind finite volumes, Maxwell
 *   diffuse walls (Eq. (5.2)) through ghost cells, total mass C (Eq. (5.3)).
 *   State f: nx*N^3 doubles [cell][i1][i2][i3] (device pointer).
 *   Residual R(f) = v1^+ D^- f + v1^- D^+ f - Q(f_j,f_j)/Kn.
 *   Modified Newton (Eqs. (5.4), (5.6)): solve
 *     A g = v1^+ D^- g + v1^- D^+ g - L_j[g_j]/Kn = R
 *   with L_j linearised about the local Maxwellian of f_j, then f <- f - g.
 *   The mass mode is handled by the bordered operator A g + e m(g) with
 *   e = f/m(f), m(g) = dx h^3 sum g, and right-hand side R + e (m(f) - C).
 * LBO_PROBLEM_HOMOGENEOUS: backward Euler for df/dt = Q(f,f) on a batch of
 *   nx independent instances: F(f) = f - f_prev - dt Q(f,f), Newton with
 *   (I - dt L_M) g = F(f), M the Maxwellian of f.
 * The linear system is solved by restarted flexible GMRES with FP64 Arnoldi
 * (classical Gram-Schmidt, two passes), FP64 residuals and norms, and a right
 * preconditioner: none, the upwind sweep of the source iteration (Eq. (5.7),
 * nu_j = rho_j), or the sweep plus a learned macroscopic correction
 * (lbo_solver_set_network).  The FP64 true residual of the linear system
 * is recomputed after the solve and reported.
 * Norms are the discrete L2 norm sqrt(dx h^3 sum r^2) of Sec. 5.3 (dx = 1
 * for the homogeneous problem).
 * ------------------------------------------------------------------------ */
typedef struct lbo_solver lbo_solver;

typedef enum { LBO_PROBLEM_SLAB = 0, LBO_PROBLEM_HOMOGENEOUS = 1 } lbo_problem_kind;
/* NONE: plain FGMRES; SWEEP: the upwind sweep of the source iteration,
   Eq. (5.7); LEARNED: sweep plus a network-predicted macroscopic correction;
   MOMENT: sweep plus a Galerkin coarse correction on the five collision
   invariants of every cell (synthetic acceleration, Sec. 5.2), assembled
   from the operator once per Newton step and solved by banded LU          */
typedef enum {
  LBO_PRECOND_NONE = 0,
  LBO_PRECOND_SWEEP = 1,
  LBO_PRECOND_LEARNED = 2,
  LBO_PRECOND_MOMENT = 3
} lbo_precond;
typedef enum { LBO_WALL_FLUX_ANALYTIC = 0, LBO_WALL_FLUX_DISCRETE = 1 } lbo_wall_flux;
/* Inflow boundary (not in the paper, which treats walls only): the ghost
 * cell holds the given Maxwellian for the residual and zero for the Newton
 * correction.  An inflow side removes the mass null mode of the operator, so
 * the bordered mass constraint applies only between two walls and
 * total_mass is then ignored; nothing pins the position of a steady shock
 * between two inflow sides. */
typedef enum { LBO_BC_WALL = 0, LBO_BC_INFLOW = 1 } lbo_boundary;

typedef struct {
  int kind;               /* lbo_problem_kind                                  */
  int nx;                 /* cells (SLAB) or instances (HOMOGENEOUS)           */
  double x_left, x_right; /* SLAB domain                                       */
  double kn;              /* Knudsen number (SLAB)                             */
  double wall_left[4];    /* theta, u1, u2, u3 of the left wall (u1 must be 0)  */
  double wall_right[4];
  double total_mass;      /* C of Eq. (5.3) (SLAB; unused when a side is inflow) */
  int wall_flux;          /* lbo_wall_flux: wall density from the analytic
                             half-range flux sqrt(theta/2pi) (Eq. (5.2), the
                             default) or from its grid sum                     */
  double dt;              /* HOMOGENEOUS time step                             */
  double krylov_rtol;     /* stop when |r| <= max(rtol |r0|, atol)             */
  double krylov_atol;
  int krylov_restart;     /* m of GMRES(m), 1..200                             */
  int krylov_maxit;       /* total inner iterations cap                        */
  int precond;            /* lbo_precond                                       */
  int bc_left, bc_right;  /* lbo_boundary (SLAB): diffuse wall (default) or
                             inflow of a given Maxwellian                      */
  double inflow_left[5];  /* rho, u1, u2, u3, theta of the inflow state        */
  double inflow_right[5];
  int line_search;        /* 0..60; 0: full Newton steps (the paper's iteration);
                             k > 0: up to k halvings of the step until the
                             residual norm decreases (Armijo, c = 1e-4)      */
  double pseudo_dt;       /* SLAB: 0 for the plain modified Newton step; > 0
                             turns on pseudo-transient continuation: each step
                             solves (I/dtau + A) g = R with
                             dtau = pseudo_dt |R_first| / |R_k|, the shift
                             also entering the sweep's diagonal             */
  int coarse_moments;     /* MOMENT preconditioner: 5 (collision invariants)
                             or 13 (plus traceless stress and heat flux);
                             other values mean 5                            */
  int jacobian;           /* 0: L about the local Maxwellian of every cell, the
                             modified step of Eqs. (5.4), (5.6);
                             1: the exact derivative of the residual,
                             J v = (Q(f + s v) - Q(f - s v)) / (2 s) with
                             s = |f| / |v| (exact for the bilinear Q of
                             Eq. (2.14) up to rounding): two Q evaluations
                             in the plan's precision per Krylov product,
                             quadratic convergence near the solution      */
  int coarse_operator;    /* MOMENT preconditioner: 0 assembles and applies
                             W^T A' P with the full operator A' (Galerkin);
                             1 keeps only A''s transport, border and shift
                             parts, exact for the 5 collision invariants up
                             to the discrete collision operator's
                             conservation, and needs no collision operator
                             per Krylov iteration                         */
  int inner_solver;       /* SLAB, preconditioner not NONE.  0: restarted
                             flexible GMRES (default); 1: the source
                             iteration of Sec. 5.2 (the paper's inner
                             solver): S g_{l+1} = (nu_j/Kn + L_j/Kn) g_l + r
                             with S the upwind transport plus nu_j/Kn,
                             i.e. g += P(rhs - A g) with P the sweep of
                             Eq. (5.7) (plus the coarse or learned
                             correction when selected), from g = 0 until
                             |rhs - A g| <= max(rtol |rhs|, atol) or
                             krylov_maxit iterations; krylov_iterations
                             counts them.  It converges only when
                             nu_j + L_j is positive (see nu_scale)         */
  double nu_scale;        /* nu_j = nu_scale * rho_j in the sweep, Eq. (5.7);
                             0 means 1, the paper's choice.  The positivity
                             condition on nu_j + L_j asks for nu_j at least
                             the largest loss frequency of the cell, which
                             for hard spheres exceeds rho_j (source
                             iteration then needs nu_scale ~ 2)            */
  int device_krylov;      /* FGMRES with the modified Jacobian and the NONE
                             or SWEEP preconditioner (uniform N, not
                             collecting training pairs, plan profiling off).
                             0: Arnoldi on the host (coefficients read back
                             per iteration); 1: Gram-Schmidt coefficients,
                             norms, Givens rotations and the stopping test
                             kept on the device, each restart cycle one
                             eager iteration plus a CUDA graph whose WHILE
                             node repeats the iteration until the device-side
                             test ends the cycle (the host reads the cycle's
                             status and the restart residual only).  Same
                             arithmetic; other configurations use 0.      */
} lbo_problem;

typedef struct {
  double residual_norm;    /* |R(f)| (or |F(f)|) at the input state             */
  double rhs_norm;         /* |right-hand side of the linear system|            */
  double linear_residual;  /* FP64 true |rhs - A g| after the solve             */
  int krylov_iterations;   /* inner iterations: FGMRES steps or source iterations */
  int restarts;
  int fallbacks;           /* 1 if the learned preconditioner was replaced by the
                              plain sweep after half of krylov_maxit iterations,
                              or the MOMENT coarse operator was singular and
                              the sweep ran alone                             */
  int status;              /* lbo_status of the inner solve (LBO_ENOTCONV if the
                              cap was hit; the step is still applied)          */
  double ms_residual;      /* time in the nonlinear residual (Q evaluations)    */
  double ms_linear;        /* time in the linear solve                          */
  double step_length;      /* lambda of f <- f - lambda g (1 without line search) */
  double shift;            /* 1/dtau of the step (0 without continuation)       */
} lbo_newton_stats;

/* Create a solver on top of a plan (the plan supplies N, the box, the
 * collision kernel, the precision of L and Q and the hemisphere rule).
 * Allocates the Krylov basis ((restart+1) * nx * N^3 doubles and as many
 * preconditioned vectors).  LBO_EINVAL for inconsistent problem data. */
lbo_status lbo_solver_create(const lbo_problem *problem, lbo_plan *plan, lbo_solver **out);

/* One Newton step in place on the device state f (nx*N^3): the modified
 * step of Eqs. (5.4), (5.6) or the exact-Jacobian step (problem.jacobian),
 * with continuation and line search as the problem sets them.
 * f_prev: the previous time level (HOMOGENEOUS; ignored for SLAB).
 * stats may be NULL.  An inner solve that stops at its cap still applies
 * the step and returns LBO_ENOTCONV (also in stats->status); LBO_ENAN for a
 * non-finite residual (state unchanged), LBO_EINVAL / LBO_ECUDA for
 * argument and CUDA errors. */
lbo_status lbo_newton_step(lbo_solver *solver, double *f, const double *f_prev, lbo_newton_stats *stats);

/* Evaluate the nonlinear residual R(f) (SLAB) or F(f) (HOMOGENEOUS) into
 * out (device, nx*N^3) and return its norm in *norm (may be NULL). */
lbo_status lbo_solver_residual(lbo_solver *solver, const double *f, const double *f_prev, double *out,
                               double *norm);

/* A slab whose cells carry different velocity grids (the shock workload with
 * N chosen per cell; not in the paper, which uses one N).  plans[p] is the
 * plan of one N (one plan per N, the same box); cell j uses
 * plans[cell_plan[j]].  The state vector holds the cells one after the
 * other, cell j as N_j^3 doubles in the usual centred order;
 * lbo_solver_state_length gives its total length.  Collisions are applied
 * per cell with the cell's plan; the upwind difference of a cell uses its
 * neighbours spectrally resampled to its grid (zero padding to a finer grid,
 * truncation to a coarser one, the Nyquist term of the coarser grid a
 * cosine).  Supported: SLAB with inflow sides at both ends (LBO_EUNSUPPORTED
 * otherwise), preconditioner NONE or SWEEP (the sweep runs on the finest
 * grid), both inner solvers (source iteration with SWEEP), both Jacobians,
 * continuation and line search; per-N residual plans through
 * lbo_solver_set_residual_plan (one call per N). */
lbo_status lbo_solver_create_mixed(const lbo_problem *problem, lbo_plan *const *plans, int nplans,
                                   const int *cell_plan, lbo_solver **out);
size_t lbo_solver_state_length(const lbo_solver *solver);

/* Mixed precision: evaluate Q(f,f) of the nonlinear residual with `plan`
 * (typically an FP64 plan) while the linear operator L of the Krylov solve
 * keeps the solver's own plan (typically FP32).  The modified Newton step of
 * Eqs. (5.4), (5.6) only needs an approximate Jacobian, so the state then
 * converges to the residual's precision.  `plan` must have the solver's N
 * and box; the solver launches it on its own stream (the plan's stream is
 * set to the solver plan's stream on every residual evaluation) and does not
 * own it: keep it alive until the solver is destroyed or the call is undone
 * with plan = NULL.  LBO_EINVAL on mismatched N or box.  A mixed-N solver
 * takes one residual plan per N (the call sets the one of plan's N; NULL
 * clears all). */
lbo_status lbo_solver_set_residual_plan(lbo_solver *solver, lbo_plan *plan);

void lbo_solver_destroy(lbo_solver *solver);

/* Learned preconditioner (SLAB only; no counterpart in the paper: a learned
 * form of the synthetic acceleration the paper points to for small Kn,
 * Sec. 5.2).  A two-layer width-5 convolutional network over the cells maps
 * 13 moments per cell ({1, v, |v|^2}, the traceless stress v1v2, v1v3, v2v3,
 * v1^2-v2^2, v2^2-v3^2 and the heat flux v|v|^2) of a Krylov vector v and of
 * its upwind sweep s to a macroscopic correction,
 * z = s + sum_a c_{j,a} phi_a(v) M_j(v), phi_a in {1, v, |v|^2}.
 * Training pairs are (A z_k, z_k) from the solver's own FGMRES iterations;
 * the target of cell j solves G_j c_j = m(z_j) - m(s_j), G_j the moment
 * matrix of phi_a phi_b M_j.  Parameters: FP32, packed as
 * [W1 (H,26,5), b1 (H), W2 (5,H,5), b2 (5)]; scales: 31 floats (26 input,
 * 5 output channel scales of the normalisation).
 *
 * lbo_solver_collect(s, max_pairs): keep up to max_pairs pairs from the next
 *   solves (0 stops collecting; changing max_pairs clears the store).
 * lbo_solver_train_network: full-batch Adam on the mean squared error of the
 *   normalised targets, on the GPU; *final_loss (may be NULL) receives it.
 * hidden = 0 selects the global linear form instead: one linear
 *   convolution of width 2 nx - 1 over the cells (every cell sees the whole
 *   slab), which can represent the nonlocal macroscopic response at small
 *   Kn with 130 (2 nx - 1) + 5 parameters (lbo_solver_network_param_count).
 * lbo_network_loss_grad: loss and gradient of the same network for given
 *   device arrays x [pairs][nx][26], t [pairs][nx][5] (for checking the
 *   hand-written backward pass); grad: device array of
 *   lbo_network_param_count(hidden) floats (hidden >= 1 there). */
int lbo_network_param_count(int hidden);
lbo_status lbo_network_loss_grad(int hidden, const float *theta, const float *x, const float *t, int pairs,
                                 int nx, double *loss, float *grad);
lbo_status lbo_solver_collect(lbo_solver *solver, int max_pairs);
int lbo_solver_pair_count(lbo_solver *solver);
lbo_status lbo_solver_train_network(lbo_solver *solver, int hidden, int epochs, double lr, unsigned seed,
                                    double *final_loss);
lbo_status lbo_solver_get_network(lbo_solver *solver, int *hidden, float *params, float *scales);
lbo_status lbo_solver_set_network(lbo_solver *solver, int hidden, const float *params, const float *scales);
int lbo_solver_network_param_count(lbo_solver *solver, int hidden);

/* Allocation-free variant of lbo_apply_linearized (the paper has no
 * counterpart; this is a library facility).  For callers that cannot
 * allocate device memory when they apply the operator: solvers whose memory
 * budget is fixed at start-up, real-time loops where cudaMalloc's implicit
 * synchronisation is not allowed, hosts that forbid allocation after
 * initialisation.  Same operator, same arguments (device pointers only),
 * but its scratch comes from one static 64 MiB device array of the library
 * instead of plan-owned memory, and it calls no allocating routine.
 * - Rejects (LBO_EINVAL, nothing launched) a batch needing more than
 *   lbo_noalloc_scratch_bytes(), i.e. batch * lbo_noalloc_bytes_per_instance
 *   (1,661,320 bytes = 1.66 MB per instance at N = 32 in FP64, half that in
 *   FP32: at most 40 and 80 instances), host pointers, a call made while
 *   another device than the plan's is current, and a plan whose tables are
 *   out of date; LBO_EUNSUPPORTED with the mass or moment fix options on or
 *   a precision other than FP64 and FP32.
 * - It always runs the generic kernel set (LBO_OPT_KERNEL = 1), also where
 *   lbo_apply_linearized would pick the fused FP32 kernels.
 * - All calls share the array: calls that overlap on the GPU race and must
 *   be serialised.  Nothing in it needs to start at zero.
 * - The first call on a device (with that device current) looks up the
 *   array's address and uploads a constant table: make it before any
 *   stream capture. */
lbo_status lbo_apply_linearized_noalloc(lbo_plan *plan, const double *maxwellian_params,
                                        const double *g, double *out, int batch);
size_t lbo_noalloc_scratch_bytes(void);
size_t lbo_noalloc_bytes_per_instance(const lbo_plan *plan);

/* Launch-shape autotuner.  Times the candidate shapes of the plan's fastest
 * kernel set on the given device arrays, keeps the fastest in the plan and
 * returns it in *choice (0 when the plan has nothing to tune):
 * - fused FP32 kernels (N = 32): 1, 2, 3, 4, 6 or 8 groups of radial nodes
 *   per instance (kept as LBO_OPT_JGROUPS);
 * - FP64 register kernels (N = 32): 2, 4 or 8 planes per CTA of the plane
 *   kernel (kept as LBO_OPT_PLANES).
 * Overwrites out. */
lbo_status lbo_plan_autotune(lbo_plan *plan, const double *maxwellian_params, const double *g, double *out,
                             int batch, int *choice);

/* Groups: several plans (e.g. grids of different N, each cell with its own
 * Maxwellian) applied together.  Each member runs on its own stream forked
 * from and joined back into the group's stream, so different grid sizes
 * overlap on the GPU.  With lbo_group_use_graph(group, 1) and a non-NULL
 * group stream, the second call with the same arrays and batch sizes
 * records the whole application into a CUDA graph and later calls replay it
 * (the first call runs eagerly, so tables and workspaces exist before any
 * capture).  Arrays are device pointers; params[i], g[i], out[i], batch[i]
 * belong to member i.  Member plans must not be used concurrently
 * elsewhere. */
typedef struct lbo_group lbo_group;
lbo_status lbo_group_create(lbo_plan *const *plans, int nplans, lbo_group **out);
lbo_status lbo_group_set_stream(lbo_group *group, void *stream);
lbo_status lbo_group_use_graph(lbo_group *group, int enable);
lbo_status lbo_group_apply_linearized(lbo_group *group, const double *const *params, const double *const *g,
                                      double *const *out, const int *batch);
void lbo_group_destroy(lbo_group *group);

/* One axis pass of a batched 3-D DFT on the tensor cores (the building
 * block of the split 16-bit precisions): out = DFT along `axis` (1, 2, 3 =
 * i1, i2, i3) of each of `batch` complex fields of N^3 FP32 pairs
 * (interleaved re, im; row-major [batch][i1][i2][i3]); forward
 * exp(-2 pi i q (j - N/2) / N) from a centred index j to a cyclic frequency
 * q (inverse = 1: the conjugate, unnormalised, frequency -> centred index).
 * precision: LBO_PREC_BF16_SPLIT or LBO_PREC_FP16_SPLIT; N = 16, 32, 64;
 * in, out: device pointers (out may equal in); stream: cudaStream_t as
 * void*.  Allocates its DFT matrices for the call and synchronizes the
 * stream.  Errors: LBO_EINVAL, LBO_EUNSUPPORTED, LBO_ENOMEM, LBO_ECUDA,
 * LBO_ETIMEOUT. */
lbo_status lbo_dft_axis_tensor(int N, int precision, int inverse, int axis, const float *in, float *out, int batch,
                               void *stream);

/* ------------------------------------------------------------------------
 * Primitives on one block of cells of the 1-D slab, for a solver whose cells
 * are split over several GPUs (a contiguous block per GPU; the host driver
 * paper_2503_09580_gb300/distributed.py composes them into the modified
 * Newton / flexible GMRES iteration of Sec. 5 and the supplement, exchanging
 * boundary cells between neighbours and summing reductions over the GPUs).
 * Cells follow one another, each N^3 doubles in the centred order; every
 * array is a device pointer; everything runs on the plan's stream.  h =
 * 2 box / N is the velocity spacing, dx the cell width.
 *
 * lbo_slab_block_transport: out_j = v1^+ (v_j - v_{j-1})/dx + v1^- (v_{j+1} -
 *   v_j)/dx for the nx cells of the block, the outer values v_{-1} =
 *   ghost_left and v_nx = ghost_right (one cell each; NULL means 0): a
 *   neighbour block's boundary cell or a wall's ghost cell (Eq. (5.2)).
 * lbo_slab_block_sweep: solves (v1^+ D^- + v1^- D^+ + nu_j/kn + shift) z = r
 *   on the block (the sweep of the source iteration, Eq. (5.7)), with the
 *   incoming values z_{-1} = in_left (velocities with v1 > 0) and z_nx =
 *   in_right (v1 < 0) (NULL means 0).  direction = +1 solves only v1 >= 0,
 *   -1 only v1 < 0, 0 both: a sweep across several blocks passes each
 *   block's outgoing boundary values to the next block downstream.
 *   nu: nx doubles (device).
 * lbo_slab_block_moments: params[5 j + 0..4] = rho, u1, u2, u3, theta of
 *   cell j (Sec. 2.1; h^3 sums on the grid); nu[j] = rho (NULL allowed).
 * lbo_slab_cell_flux: *host_out = h^3 sum v1^- x (side 0) or h^3 sum v1^+ x
 *   (side 1) over one cell (the wall flux of Eq. (5.2)); synchronizes.
 * lbo_slab_maxwellian_cell: out = scale (2 pi theta)^{-3/2}
 *   exp(-|v - u|^2/(2 theta)) on one cell (u: 3 host doubles).
 * lbo_vec_dots: host_out[k] = <V + k ld, y> over len doubles, k < K (at
 *   most 512), summed in a fixed order; synchronizes.
 * lbo_vec_axpby: y = a x + b y over len doubles.
 * lbo_vec_combination: y -= sum_k c_host[k] (V + k ld), k < K (at most 512);
 *   synchronizes (c_host may be reused at once).
 * Errors: LBO_EINVAL for bad arguments, LBO_ENOMEM, LBO_ECUDA. */
lbo_status lbo_slab_block_transport(lbo_plan *plan, const double *v, const double *ghost_left,
                                    const double *ghost_right, double *out, int nx, double dx);
lbo_status lbo_slab_block_sweep(lbo_plan *plan, const double *r, const double *nu, const double *in_left,
                                const double *in_right, double *z, int nx, double dx, double kn, double shift,
                                int direction);
lbo_status lbo_slab_block_moments(lbo_plan *plan, const double *f, int nx, double *params, double *nu);
lbo_status lbo_slab_cell_flux(lbo_plan *plan, const double *cell, int side, double *host_out);
lbo_status lbo_slab_maxwellian_cell(lbo_plan *plan, double theta, const double *u, double scale, double *out);
lbo_status lbo_vec_dots(lbo_plan *plan, const double *V, size_t ld, int K, const double *y, size_t len,
                        double *host_out);
lbo_status lbo_vec_axpby(lbo_plan *plan, double *y, const double *x, double a, double b, size_t len);
lbo_status lbo_vec_combination(lbo_plan *plan, double *y, const double *V, size_t ld, int K, const double *c_host,
                               size_t len);

/* Measured ALU peaks of the current device, the denominators of the
 * library's roofline fractions for ALU-bound kernels (a measurement
 * facility; the paper has no counterpart).  Runs dense chains of FP32 FFMA
 * and FP64 DFMA (independent chains per thread, operands in registers, one
 * full wave of 64 warps per SM, about 25 ms per launch), times them with
 * CUDA events on `stream` (a cudaStream_t as void*, NULL = legacy default
 * stream) and returns the best of three launches in TFLOP/s (an FMA counts
 * 2 flops), the SM count from the device properties, and the SM clock seen
 * by the FP32 loop (clock64 cycles over the event time, MHz).  Any output pointer may be
 * NULL.  Allocates and frees a small device buffer; synchronizes `stream`.
 * Errors: LBO_ECUDA, LBO_ENOMEM. */
lbo_status lbo_measure_alu_peaks(void *stream, double *fp32_tflops, double *fp64_tflops, int *sm_count,
                                 double *sm_mhz);

/* Free a plan (NULL is allowed). */
void lbo_plan_destroy(lbo_plan *plan);

/* Static description of a status code. */
const char *lbo_status_string(lbo_status s);

/* Text of the last CUDA error seen by this thread in any lbo call ("" if
 * none). */
const char *lbo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBO_H */
