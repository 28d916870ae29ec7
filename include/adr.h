/*
 * adr.h -- C ABI of the GB300 amplitude solver for the point-source Helmholtz
 * equation (Treister & Haber, "A multigrid solver to the Helmholtz equation
 * with a point source based on travel time and amplitude").
 *
 * The library solves the complex advection-diffusion-reaction (ADR) equation
 * for the amplitude a (Eq. ADR, paper sign convention u = a exp(-i w tau),
 * Eq. new_u):
 *     Delta a - 2 i w grad(tau).grad(a) - i w (Delta tau) a
 *             - w^2 (|grad tau|^2 - kappa^2) a - i w gamma kappa^2 a = q_hat
 * discretised with the second-order upwind advection of Eq. londUpwindDiff
 * (the matrix H_2up of Eq. ADRLinSystemUpwind), by flexible GMRES
 * preconditioned with a geometric multigrid cycle on
 * (1 - beta) H_2up + beta H_1up (Eq. precADRup) whose coarse operators are
 * Galerkin products P^T A P (Eq. coarseGridMatrix).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grids are nodal, dim = 2 or 3, n[d] nodes along axis d (axis 0 fastest,
 *   the last axis is depth), spacing h[d].  Node (i0, i1[, i2]) is element
 *   i0 + n0*(i1 + n1*i2) of every array.  Every n[d] must be >= 4.
 * - Real arrays are float64.  Complex arrays are interleaved (re, im) pairs
 *   of float64 (precision ADR_F64, same layout as torch.complex128) or of
 *   float32 (ADR_F32, torch.complex64).
 * - Unless an entry point says "host", every array argument is a DEVICE
 *   pointer on the device that was current when the operator was created,
 *   allocated and owned by the caller; the library never frees it and keeps
 *   no reference to it after the call returns.
 * - The library owns the operator's hierarchy and workspace (one device
 *   arena per operator), released by adr_operator_destroy.
 * - Work is issued on the stream given at creation; calls return after the
 *   stream has been synchronised only where documented (adr_solve reads one
 *   residual estimate per iteration).
 * - Every entry point returns ADR_OK or a negative ADR_ERR_* code; the text
 *   of the most recent error of the calling thread is kept for
 *   adr_last_error.  Invalid arguments are rejected before any device work.
 */
#ifndef ADR_H_
#define ADR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADR_OK 0
#define ADR_ERR_ARG (-1)            /* invalid argument (null, size, range) */
#define ADR_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define ADR_ERR_OOM (-3)            /* device allocation failed */
#define ADR_ERR_NOT_CONVERGED (-4)  /* iteration budget spent above tolerance */
#define ADR_ERR_NAN (-5)            /* NaN or Inf met in a Krylov scalar */
#define ADR_ERR_STATE (-6)          /* operation not valid for this operator */

#define ADR_F64 0
#define ADR_F32 1

/* Discrete operators on the finest grid. */
#define ADR_SCHEME_2UP 0   /* H_2up, Eq. ADRLinSystemUpwind (the solved system) */
#define ADR_SCHEME_1UP 1   /* H_1up, Eq. 1up */
#define ADR_SCHEME_CEN 2   /* H_cen, Eq. ADRLinSystemCentral */
#define ADR_SCHEME_PREC 3  /* (1 - beta) H_2up + beta H_1up, Eq. precADRup */

/* Multigrid cycle shape (Sec. 3: Alg. TwoGrid applied recursively, Alg. Kcycle). */
#define ADR_CYCLE_V 0
#define ADR_CYCLE_K 1

/* Relaxation (Sec. 3.1). */
#define ADR_RELAX_JACOBI 0  /* damped Jacobi with the fixed weight jacobi_weight[l] */
#define ADR_RELAX_MR 1      /* one step of Jacobi-preconditioned GMRES per sweep:
                               Jacobi with the minimal-residual complex weight */

#define ADR_MAX_LEVELS 8

typedef struct adr_params {
  int levels;                          /* maximum number of grid levels (>= 1) */
  double beta;                         /* blend of Eq. precADRup */
  int cycle;                           /* ADR_CYCLE_V or ADR_CYCLE_K */
  int relax;                           /* ADR_RELAX_JACOBI or ADR_RELAX_MR */
  int pre_sweeps[ADR_MAX_LEVELS];      /* relaxations before restriction, per level */
  int post_sweeps[ADR_MAX_LEVELS];     /* relaxations after the correction, per level */
  double jacobi_weight[ADR_MAX_LEVELS];/* ADR_RELAX_JACOBI weight per level */
  int coarse_iterations;               /* fixed Jacobi-GMRES steps on the coarsest grid */
  int kcycle_iterations;               /* inner FGMRES steps of the K-cycle */
  int restart;                         /* outer FGMRES restart length m (1..64) */
  int precond_precision;               /* ADR_F64 or ADR_F32: arithmetic of the cycle */
  int near_source;                     /* rows within this Chebyshev distance of the
                                          source use central advection (Sec. 2.2 says
                                          "distance of one node"; 1..4, default 1) */
  double reorth_eta;                   /* Gram-Schmidt of the outer FGMRES and of the
                                          coarsest-grid GMRES (one launch per step, or
                                          the cooperative form): the second classical
                                          pass runs only when the first left less than
                                          reorth_eta |w| (Daniel-Gragg-Kaufman-Stewart
                                          test); >= 1: always (CGS2).  The single-block
                                          and cluster coarsest forms always run it.
                                          Default 0.1 */
  int adjoint;                         /* 1: also build the conjugate-transposed
                                          operator and its hierarchy (adr_adjoint_solve,
                                          adr_apply_adjoint, adr_vcycle_adjoint); about
                                          doubles the operator's memory.  Default 0 */
  int relax_blocks;                    /* grid of the fused relaxation applies (blocks
                                          per problem, grid-stride beyond); 0 selects
                                          2432 (16 per SM).  The bulk-copy applies
                                          (tma) run one block per SM, or relax_blocks
                                          blocks when that is smaller.  A launch shape,
                                          not arithmetic: results do not depend on it
                                          beyond rounding order.  0..10240 */
  int coarse_solver;                   /* form of the coarsest-grid GMRES (same arithmetic):
                                          ADR_COARSE_AUTO picks by size; the others force
                                          one (cluster and grid need <= 32 iterations) */
  int tma;                             /* 1: the float32 relaxation applies of the stored-
                                          stencil levels stream their coefficients into
                                          shared memory with bulk copies (16 warps, one
                                          buffer each); 2: the same with 8 warps, two
                                          buffers each; 3: 16 warps, one buffer each
                                          refilled in halves (box entries, two-point
                                          entries; the coarsest grid's GMRES step keeps
                                          whole tiles); 4: the same in quarters; 0:
                                          plain loads.  Same products;
                                          the sums' order and the weight's block sums
                                          follow the kernel.  Default 3 */
  double shift;                        /* complex shift alpha of the cycle's operator
                                          (Eq. shift): the multigrid hierarchy is built
                                          from the preconditioner minus i alpha w^2
                                          kappa^2 on its diagonal, the outer operator is
                                          unchanged.  With tau1 = 0 this is the shifted-
                                          Laplacian preconditioner of the standard
                                          Helmholtz matrix (Sec. 3, alpha = 0.2 in
                                          Sec. 4).  0..100, default 0 (no shift) */
  int scheme;                          /* the solved system (outer FGMRES operator):
                                          ADR_SCHEME_2UP (Eq. ADRLinSystemUpwind, default),
                                          ADR_SCHEME_1UP (Eq. 1up) or ADR_SCHEME_CEN
                                          (Eq. ADRLinSystemCentral) */
  int prec_scheme;                     /* the cycle's finest-grid operator before the
                                          shift: ADR_SCHEME_PREC (the blend of
                                          Eq. precADRup, default; beta = 1 gives H_1up)
                                          or ADR_SCHEME_2UP / 1UP / CEN */
  int rescale;                         /* 1: the cycle is built on M A M^{-1}, M =
                                          diag(exp(-i w tau)) (the system rescaled as
                                          Helmholtz, Eq. ADRcenRescaled), and applied as
                                          z = M^{-1} K (M v); the outer iteration stays on
                                          the amplitude.  Stage 2 of Alg. ADRlong is
                                          scheme = prec_scheme = ADR_SCHEME_CEN, shift =
                                          0.2, rescale = 1.  Default 0 */
  double kcycle_threshold;             /* early exit of the K-cycle's inner FGMRES
                                          (Alg. Kcycle; Sec. 4.2 uses 0.1 on the coarse
                                          grids): an inner solve whose residual falls to
                                          this fraction of the restricted residual stops
                                          and its later steps do not enter the result.
                                          0 (default): the fixed kcycle_iterations steps.
                                          0..1e6 */
  int outer_df;                        /* 1 (default): with a float32 cycle (not
                                          rescaled) and adjoint = 0, the outer
                                          iteration runs in double-float arithmetic
                                          (pairs of float32 values, float32 pipe; about
                                          2^-46 relative per operation against
                                          float64's 2^-53): A z_j on the float32 z_j,
                                          the Gram-Schmidt passes, the normalisation and
                                          x += Z y.  The solution, the Hessenberg
                                          matrix and the residual at every restart stay
                                          float64.  0: all outer work in float64 */
} adr_params_t;

#define ADR_COARSE_AUTO 0      /* cluster up to 32768 nodes, else one block up to 8192, else kernels */
#define ADR_COARSE_KERNELS 1   /* one launch per step (reductions across launches) */
#define ADR_COARSE_CTA 2       /* one 1024-thread block per problem */
#define ADR_COARSE_CLUSTER 3   /* one thread-block cluster per problem (DSMEM reductions) */
#define ADR_COARSE_GRID 4      /* one cooperative launch over all SMs (grid barriers) */

typedef struct adr_level_info {
  int n[3];            /* nodes per axis (n[2] = 1 in 2D) */
  int64_t nodes;
  int stencil_points;  /* 0 on the finest level (matrix-free), 21 (2D) or 81 (3D) */
} adr_level_info_t;

typedef struct adr_op_info {
  int dim;
  int levels;
  adr_level_info_t level[ADR_MAX_LEVELS];
  int64_t arena_bytes;     /* device bytes owned by the operator */
  int problems;            /* problems of a batched operator (1 otherwise) */
} adr_op_info_t;

typedef struct adr_solve_info {
  int iterations;          /* outer FGMRES iterations performed */
  int restarts;            /* completed restart cycles */
  double rel_residual;     /* |q - H_2up a| / |q|, recomputed explicitly at exit */
  double rel_estimate;     /* last Givens estimate |g_{j+1}| / |q| */
  int status;              /* ADR_OK, ADR_ERR_NOT_CONVERGED or ADR_ERR_NAN */
} adr_solve_info_t;

typedef struct adr_op_s* adr_op_t;

/* Fills *p with the defaults: 5 levels, beta = 0.25 (Sec. 4.2), K-cycle with
 * ADR_RELAX_MR, l+1 pre/post relaxations on level l counted from 1 (Sec. 4.2),
 * 10 coarsest-grid iterations (Sec. 4.2), 2 inner K-cycle steps (Alg. Kcycle),
 * restart 20, FP32 cycle.  Returns ADR_ERR_ARG if p is NULL. */
int adr_params_default(adr_params_t* p);

/* Builds the operator for one point source (Sec. 2.1 coefficients,
 * Eq. travel_time_coeff; Sec. 3 hierarchy, Eq. coarseGridMatrix).
 *   kappa, tau1, gamma: device float64[N], slowness, travel-time factor
 *       (tau = |x - x0| * tau1) and absorbing-layer profile; read during the
 *       call only.
 *   src: node index per axis of the source x0 (inside the grid).
 *   omega > 0: angular frequency.  params: NULL selects the defaults.
 *   stream: cudaStream_t used for all work of this operator (NULL = legacy
 *       default stream).
 * On success *out receives a handle to destroy with adr_operator_destroy.
 * Errors: ADR_ERR_ARG for bad sizes/pointers/parameters, ADR_ERR_OOM,
 * ADR_ERR_CUDA. */
int adr_operator_create(int dim, const int* n, const double* h, const int* src, double omega,
                        const double* kappa, const double* tau1, const double* gamma,
                        const adr_params_t* params, void* stream, adr_op_t* out);

/* adr_operator_create for a travel time given as plain nodal values tau
 * (device float64[N]) instead of the factor tau1 of tau = |x - x0| tau1: the
 * coefficients of Eq. travel_time_coeff take d_d tau and d_dd tau by finite
 * differences of tau itself (central inside, first-order / second-order
 * one-sided on the boundary), the source row (Eq. helmADR2) and the
 * reconstruction use tau directly.  tau must be the travel time from the
 * source (zero at src).  Next to the source, where tau has its conical kink,
 * the differences are only first-order accurate: the factored form of
 * adr_operator_create is the more accurate input (Sec. 2.1).  Everything
 * else (arguments, ownership, errors) as adr_operator_create;
 * adr_operator_update on this operator takes plain tau in its tau1
 * argument. */
int adr_operator_create_tau(int dim, const int* n, const double* h, const int* src, double omega,
                            const double* kappa, const double* tau, const double* gamma,
                            const adr_params_t* params, void* stream, adr_op_t* out);

/* Rebuilds the coefficients and the whole Galerkin hierarchy of an existing
 * operator for a new source, frequency and medium on the same grid, inside
 * the operator's arena (no allocation, no synchronisation).  Arguments as in
 * adr_operator_create.  Errors: ADR_ERR_ARG, ADR_ERR_CUDA. */
int adr_operator_update(adr_op_t op, const int* src, double omega, const double* kappa, const double* tau1,
                        const double* gamma);

/* A batch of `problems` independent point-source problems on one grid (the
 * same dim, n, h and params), each with its own source, frequency, slowness,
 * travel time and absorbing profile; the paper has no batched form.  Every
 * operation of the operator then runs all problems at once: each kernel
 * launch covers every problem's nodes (one launch per step of the cycle and
 * of the Krylov iteration), and the problems' flexible GMRES iterations
 * advance in lockstep, a problem that meets its tolerance being frozen.
 *   src: int[3 * problems] (3 entries per problem, unused axes 0);
 *   omega: double[problems] (host arrays);
 *   kappa, tau1, gamma: device float64[problems * N], problem-major.
 * Vectors of the other entry points become problem-major arrays of
 * problems * N entries; adr_solve fills `problems` info entries;
 * adr_coefficients / adr_level_stencil write one block per problem.  The
 * adjoint (params.adjoint) is built for single problems only (ADR_ERR_ARG).
 * problems in [1, 65535]. */
int adr_batch_create(int dim, const int* n, const double* h, int problems, const int* src, const double* omega,
                     const double* kappa, const double* tau1, const double* gamma, const adr_params_t* params,
                     void* stream, adr_op_t* out);

/* A batch whose problems have grids of their own (sizes and spacings), the
 * paper has no batched form: the many-source, many-frequency setting where
 * each frequency gets the coarsest grid that keeps its points per wavelength.
 * Every kernel launch of the cycle and of the Krylov iteration still covers
 * all problems (grid.y = problem; a problem smaller than the largest leaves
 * the surplus blocks idle), the problems' FGMRES iterations advance in
 * lockstep as in adr_batch_create, and each problem's arithmetic is that of
 * its own single-problem operator up to the rounding order of reductions.
 *   n: int[3 * problems], nodes per axis per problem (unused axes 1);
 *   h: double[3 * problems], spacing per axis per problem;
 *   src: int[3 * problems]; omega: double[problems] (host arrays);
 *   kappa, tau1, gamma: device float64 arrays of sum_p N_p entries, problem
 *   p's N_p = n0 n1 n2 entries after the earlier problems' (the same layout
 *   for every vector of the other entry points and for adr_coefficients,
 *   whose per-problem blocks are (2 dim + 3) N_p).
 * Every problem's grid must allow the same number of levels up to
 * params.levels (the hierarchy stops where any problem stops).  The
 * persistent cooperative coarsest form is not used for these batches.
 * Errors as adr_batch_create. */
int adr_batch_create_grids(int dim, int problems, const int* n, const double* h, const int* src, const double* omega,
                           const double* kappa, const double* tau1, const double* gamma, const adr_params_t* params,
                           void* stream, adr_op_t* out);

/* adr_operator_update for a batch (arrays as in adr_batch_create); the
 * single-problem adr_operator_update refuses batches (ADR_ERR_STATE). */
int adr_batch_update(adr_op_t op, const int* src, const double* omega, const double* kappa, const double* tau1,
                     const double* gamma);

/* Releases the operator and its device arena (after synchronising its stream). */
int adr_operator_destroy(adr_op_t op);

/* Describes the hierarchy built for op. */
int adr_operator_info(adr_op_t op, adr_op_info_t* info);

/* Copies the fine-level coefficients (Eq. travel_time_coeff and the reaction
 * term of Eq. ADR) to the device float64 array out of (2*dim + 3) * N values:
 * d_d tau for each axis, d_dd tau for each axis, Re rho, Im rho, tau. */
int adr_coefficients(adr_op_t op, double* out);

/* y = A x on the finest grid for scheme ADR_SCHEME_* (Eqs. ADR, londDiff,
 * londUpwindDiff, 1up, precADRup), complex vectors of N entries in the given
 * precision (ADR_F32 uses the float32 copies of the coefficients). */
int adr_apply(adr_op_t op, int scheme, int precision, const void* x, void* y);

/* Copies the Galerkin stencil of level l >= 1 (precision of the cycle) to the
 * device array out: stencil_points * nodes complex values, point-major
 * (entry for point p of node j at p * nodes + j).  Point p enumerates the
 * offsets (o0, o1[, o2]) in [-2, 2]^dim with at most one |o_d| = 2, axis 0
 * fastest, in lexicographic order of (o_{dim-1}, ..., o0). */
int adr_level_stencil(adr_op_t op, int level, void* out);

/* One application of the multigrid preconditioner: z = B^{-1} r on the
 * finest grid (complex, precision of the cycle).  z may not alias r. */
int adr_vcycle(adr_op_t op, const void* r, void* z);

/* q_hat = delta_{x0} / prod(h) (float64 complex, N entries, Sec. 4.1). */
int adr_point_source_rhs(adr_op_t op, void* q);

/* Solves A a = rhs by right-preconditioned flexible GMRES(m), A the system
 * params.scheme selects (H_2up by default; "H_2up" below stands for it).
 *   rhs: float64 complex device vector, or NULL for the point source.
 *   a: float64 complex device vector; input initial guess if use_x0 != 0,
 *      output solution.
 *   Stops when |rhs - H_2up a| / |rhs| <= tol (checked on the Givens estimate
 *   inside a cycle and explicitly at the end of each cycle) or after maxit
 *   iterations (then ADR_ERR_NOT_CONVERGED, a still holds the iterate).
 *   info may be NULL; for a batch it receives one entry per problem, and the
 *   return code is ADR_ERR_NOT_CONVERGED if any problem missed the tolerance. */
int adr_solve(adr_op_t op, const void* rhs, void* a, int use_x0, double tol, int maxit,
              adr_solve_info_t* info);

/* Alg. ADRlong, the two-stage solve: stage 1 runs FGMRES on stage1's system
 * from a zero guess until its relative residual is <= tol1 or maxit1
 * iterations have run (Sec. 4.2 uses 1e-2 and 5; ending at maxit1 is not an
 * error); its iterate starts stage 2, which runs to tol / maxit.  For the
 * central ADR system, stage1 is scheme = ADR_SCHEME_1UP with the cycle on
 * H_1up (prec_scheme ADR_SCHEME_PREC, beta = 1) and stage2 is scheme =
 * prec_scheme = ADR_SCHEME_CEN, shift = 0.2, rescale = 1.
 *   The two operators must share grid, spacing, problems, sources and
 *   frequencies (else ADR_ERR_ARG).  rhs: NULL for the point source, else a
 *   float64 complex device vector of B*N entries.  a: float64 complex, B*N,
 *   output.  info: NULL or 2*B entries (stage 1's B, then stage 2's B).
 *   Returns stage 2's status (as adr_solve), or stage 1's error other than
 *   ADR_ERR_NOT_CONVERGED. */
int adr_solve_two_stage(adr_op_t stage1, adr_op_t stage2, const void* rhs, void* a, double tol1, int maxit1,
                        double tol, int maxit, adr_solve_info_t* info);

/* u = a exp(-i w tau) (Eq. new_u), float64 complex device vectors. */
int adr_reconstruct(adr_op_t op, const void* a, void* u);

/* The whole pipeline on HOST buffers: copies kappa, tau1, gamma (host
 * float64[N]) to the device, builds the operator, solves for the point
 * source from a zero guess, reconstructs u, and copies u (and a, if not
 * NULL) back to host float64 complex arrays of N entries.  Host buffers may
 * be pageable or pinned.  The operator is destroyed before returning. */
int adr_solve_host(int dim, const int* n, const double* h, const int* src, double omega,
                   const double* kappa, const double* tau1, const double* gamma,
                   const adr_params_t* params, double tol, int maxit, void* stream,
                   double* u_host, double* a_host, adr_solve_info_t* info);

/* ---------------------------------------------------------------------------
 * Adjoint state and slowness gradient.  The paper has no adjoint; this is the
 * standard adjoint-state gradient of a receiver misfit through its operator:
 * with u = M a, M = diag(exp(-i w tau)) (Eq. new_u), receivers R, data d and
 * J = 1/2 |R u - d|^2, the travel time held fixed,
 *     H_2up^H lambda = M^H R^T (R u - d),
 *     dJ/dkappa_j = -Re( conj(lambda_j) (2 w^2 kappa_j - 2 i w gamma_j kappa_j) a_j ),
 * because kappa enters H_2up only through its reaction diagonal
 * w^2 kappa^2 - i w gamma kappa^2 (Eq. ADR).  The entry points below need an
 * operator created with params.adjoint = 1 (else ADR_ERR_STATE), except
 * adr_receivers and adr_kappa_gradient.
 * ------------------------------------------------------------------------- */

/* Solves H_2up^H lambda = rhs (device complex128[N], not aliasing lambda) by
 * the same flexible GMRES as adr_solve, preconditioned by the cycle on the
 * conjugate-transposed hierarchy (coarse operators P^T A^H P).  use_x0, tol,
 * maxit, info and the error codes as in adr_solve. */
int adr_adjoint_solve(adr_op_t op, const void* rhs, void* lambda, int use_x0, double tol, int maxit,
                      adr_solve_info_t* info);

/* y = H_2up^H x, complex128[N] (the conjugate transpose of the float64
 * operator that adr_apply(op, ADR_SCHEME_2UP, ADR_F64, ...) applies). */
int adr_apply_adjoint(adr_op_t op, const void* x, void* y);

/* One application of the cycle on the conjugate-transposed hierarchy:
 * z = B_H^{-1} r in the precision of the cycle (as adr_vcycle). */
int adr_vcycle_adjoint(adr_op_t op, const void* r, void* z);

/* Receiver sampling: rec (device int64[nrec]) node indices, d (device
 * complex128[nrec]) data, u (device complex128[N]) the wavefield.  Writes, for
 * the pointers that are not NULL: res (device complex128[nrec]) = u[rec] - d;
 * rhs (device complex128[N]) = M^H R^T res (zero elsewhere; repeated receivers
 * add up); *misfit (host) = 1/2 |res|^2 (synchronises the stream).  A receiver
 * index outside [0, N) contributes nothing and, when misfit is requested,
 * makes the call return ADR_ERR_ARG. */
int adr_receivers(adr_op_t op, int nrec, const int64_t* rec, const void* d, const void* u, void* res, void* rhs,
                  double* misfit);

/* grad (device float64[N]) -= Re(conj(lambda) (2 w^2 kappa - 2 i w gamma kappa) a)
 * elementwise: adds this source's term of dJ/dkappa.  kappa, gamma: device
 * float64[N] (those the operator was last built with); a, lambda: device
 * complex128[N] (amplitude and adjoint state). */
int adr_kappa_gradient(adr_op_t op, const double* kappa, const double* gamma, const void* a, const void* lambda,
                       double* grad);

/* Travel-time factor for the point source at node src (input preparation,
 * not part of the solve): tau1 (device float64[N], output) with
 * tau = |x - x0| * tau1 solving the first-order upwind (Godunov)
 * discretisation of the factored eikonal equation
 * |tau0 grad tau1 + tau1 grad tau0|^2 = kappa^2 (Eq. factoredEikonal),
 * relaxed in place on the device until no node changes (at most max_sweeps
 * sweeps; *sweeps_done, if not NULL, receives the count).  kappa: device
 * float64[N] slowness.  Returns ADR_ERR_NOT_CONVERGED if max_sweeps was
 * reached while values still changed, ADR_ERR_ARG / ADR_ERR_OOM /
 * ADR_ERR_CUDA on failure.  Allocates (and frees) one int of device memory. */
int adr_traveltime(int dim, const int* n, const double* h, const int* src, const double* kappa, double* tau1,
                   int max_sweeps, void* stream, int* sweeps_done);

/* adr_traveltime with a choice of order.  order 1 is adr_traveltime.  order 2
 * continues from that first-order fixed point with the second-order
 * one-sided differences of the factored fast marching (Sec. 2.1): along each
 * axis (3 t_j - 4 t_nb + t_nb2) / 2h where the node two steps out on the
 * upwind side has the smaller travel time, first order at Chebyshev distance
 * 1 from the source, the larger root of the local quadratic, axes dropped
 * while the root would fall below a neighbour's travel time.  That phase
 * iterates Jacobi sweeps (deterministic) until no node moves by more than a
 * relative 1e-12, at most max_sweeps more sweeps; *sweeps_done counts both
 * phases.  Allocates one int, one pinned int and (order 2) N float64 of
 * device memory for the call.  Errors as adr_traveltime; ADR_ERR_ARG for
 * another order. */
int adr_traveltime_order(int dim, const int* n, const double* h, const int* src, const double* kappa, double* tau1,
                         int order, int max_sweeps, void* stream, int* sweeps_done);

/* adr_traveltime without any allocation.  The paper has no counterpart: this
 * is a deployment variant of the same computation, with the same arguments,
 * result and error codes as adr_traveltime.
 *
 * It is for callers that must not allocate during the call: a process whose
 * device memory is held by a caching allocator (where cudaMalloc can fail
 * although the caller's pool has room), or one that keeps other streams busy
 * (cudaFree waits for the whole device; pinning host memory is slow).  No
 * cudaMalloc, cudaFree, cudaMallocHost or allocating library routine runs in
 * this call.  The per-sweep convergence flags live in a fixed device array of
 * ADR_TRAVELTIME_STATIC_MAX_SWEEPS ints (32 KiB) inside the library; the call
 * zeroes the first max_sweeps of them on `stream` before its first sweep, so
 * nothing needs to be zero beforehand.  The host reads the flags into stack
 * memory every 16 sweeps (a synchronisation of `stream`).
 *
 * - max_sweeps above ADR_TRAVELTIME_STATIC_MAX_SWEEPS is rejected with
 *   ADR_ERR_ARG before any device work.
 * - The first call on a device looks up the array's device address on the
 *   current device (which may load the library's module there); it must not
 *   run while any stream of the process is being captured.
 * - The array is shared by every call on a device: calls that overlap in time
 *   on one device (from other threads or streams) race on it and must be
 *   serialised by the caller. */
#define ADR_TRAVELTIME_STATIC_MAX_SWEEPS 8192
int adr_traveltime_static(int dim, const int* n, const double* h, const int* src, const double* kappa, double* tau1,
                          int max_sweeps, void* stream, int* sweeps_done);

/* Kernel classes that adr_profile_kernel can time. */
#define ADR_PROF_NONE 0
#define ADR_PROF_LEVEL1_RELAX 1   /* minimal-residual apply on level 1 (stored stencil) */
#define ADR_PROF_FINE_RELAX 2     /* minimal-residual apply on the finest level */
#define ADR_PROF_OUTER_APPLY 3    /* float64 H_2up apply of the outer iteration */
#define ADR_PROF_COARSEST 4       /* coarsest-grid solve */
#define ADR_PROF_CYCLE 5          /* one whole preconditioner application (the
                                     captured cycle, every level's kernels) */

/* Instrumentation: brackets every launch of one kernel class of op with CUDA
 * events on the stream it runs on (inside the captured cycle as well) and
 * accumulates their durations at the synchronisation points of adr_solve.
 * Changing the class discards the captured cycle (recaptured on next use).
 * adr_profile_read returns the launches timed and their total milliseconds
 * since the class was set.  Errors: ADR_ERR_ARG, ADR_ERR_CUDA. */
int adr_profile_kernel(adr_op_t op, int kernel_class);
int adr_profile_read(adr_op_t op, long long* launches, double* total_ms);

/* Number of CUDA kernels the library has launched since it was loaded (all
 * threads, all operators); an instrumentation counter, never reset. */
long long adr_kernel_launches(void);

/* Text of the calling thread's most recent error ("" if none). */
const char* adr_last_error(void);

/* Library version, e.g. "0.1.0". */
const char* adr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ADR_H_ */
