/*
 * dngd.h - C ABI of the GB300 (sm_103a) Dual Natural Gradient Descent step.
 *
 * The library computes one damped Gauss-Newton (Levenberg-Marquardt) step of
 * a tanh-MLP physics-informed network in residual space, as defined by
 * Jnini & Vella, "Dual Natural Gradient Descent for Scalable Training of
 * Physics-Informed Neural Networks" (TMLR 2025):
 *
 *   residuals r(theta) in R^m, classes scaled by 1/sqrt(N_gamma)   (Sec. 2.2)
 *   Jacobian  J = dr/dtheta in R^{m x n}                            (Sec. 2.2)
 *   residual Gramian K = J J^T                                      (Def. 3.1)
 *   dual system (K + lambda I) alpha = r, v = -J^T alpha            (Thm. 3.1,
 *        push-through form of Eq. dual-system / dual-recovery)
 *   geodesic acceleration: f_vv = d^2/dt^2 r(theta + t v), (K + lambda I)
 *        beta = f_vv, a = -J^T beta, accept v + a/2 when 2||a||/||v|| <= 0.5
 *                                  (Sec. 3.2, Prop. 3.2, Alg. DenseDualSolve)
 *   Nystrom-preconditioned CG for large m                       (Sec. 3.3,
 *        Eq. spec_precond_nystrom_main_final, Alg. PCGStep)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - theta layout: for each affine layer l in order, W_l [w_l x w_{l-1}]
 *   row-major followed by b_l [w_l].  Hidden layers use tanh, the output
 *   layer (width 1) is affine.
 * - X is [m x d_in] row-major float64; rows are grouped by residual class in
 *   the order of dngd_problem_desc.classes.  target is [m] float64.
 * - The step returned in delta_out is the increment to ADD to theta.
 * - Unless a function says otherwise, pointer arguments may be device
 *   pointers (used in place) or host pointers (pageable or pinned; the
 *   library stages them through its own device buffers).  The caller owns
 *   every pointer it passes.  The library owns its workspace, allocated in
 *   dngd_create.
 * - All device work is ordered on the stream given to dngd_create.  A call
 *   returns after the work is enqueued, except where it must read a result
 *   on the host (dngd_step with info != NULL, host output pointers), in which
 *   case it synchronises that stream.
 * - Errors: functions return DNGD_OK (0) or a negative dngd_status.  Device
 *   side failures (non-SPD pivot, non-finite values, bounded-wait timeouts)
 *   are recorded in a device status word and reported by the next call that
 *   synchronises.  No entry point traps the GPU.
 */
#ifndef DNGD_H
#define DNGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int dngd_status;

enum {
  DNGD_OK = 0,
  DNGD_ERR_INVALID_ARG = -1,  /* bad descriptor, size or pointer */
  DNGD_ERR_NOT_SPD = -2,      /* Cholesky pivot <= 0; info->not_spd_column */
  DNGD_ERR_NO_CONVERGE = -3,  /* CG / refinement hit its iteration cap */
  DNGD_ERR_NONFINITE = -4,    /* NaN/Inf in r, K, the factor or the step */
  DNGD_ERR_BUDGET = -5,       /* serving admission refused (HBM budget) */
  DNGD_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
  DNGD_ERR_CUDA = -7,         /* CUDA runtime/driver error */
  DNGD_ERR_STATE = -8,        /* call out of order (e.g. solve before step) */
  DNGD_ERR_OOM = -9           /* device allocation failed */
};

enum dngd_precision {
  DNGD_FP64 = 0,        /* every stage in float64 */
  DNGD_MIXED_BF16 = 1,  /* FP32 jets/J, BF16 tensor-core Gram (FP32 accum),
                           FP32 Cholesky of K + (lambda+mu) I and its explicit
                           inverse as the preconditioner of PCG refinement on
                           the FP32-J operator with double-float accumulation */
  DNGD_MIXED_TF32 = 2,  /* as MIXED_BF16 with a TF32 tensor-core Gram */
  DNGD_MIXED_OZ = 3,    /* FP32 jets/J; exact Gram of the FP32 J from four
                           8-bit integer slices per row on the BF16 tensor
                           cores (13 slice products; the three leading levels
                           in exact FP32 chunks, the two trailing ones rounded
                           within 2^-39 of the row scales times n; chunks
                           summed in double-float: K accurate to ~2^-33 of the
                           row scales); the FP32 factor of K + (lambda+mu) I (as
                           MIXED_BF16) preconditions PCG whose operator is the
                           exact FP64 Gram (one m x m GEMV per iteration
                           instead of two over J) */
  DNGD_MIXED_OZ64 = 4   /* as MIXED_OZ for an FP64 Jacobian: FP64 jets,
                           residuals, J, f_vv and map-back J^T x; the exact
                           Gram from the same four 8-bit slices per entry
                           with the products of levels g = s + t <= 5 (15 of
                           16; the dropped level is what limits an accurate
                           J's Gram, not the slicing); K accurate to ~2^-33
                           of the row scales, the Gram of J rounded to 32
                           bits below each row's largest entry; FP32
                           preconditioning factor and PCG on the exact Gram
                           as MIXED_OZ; line-search trial losses in FP32 */
};

enum dngd_solver {
  DNGD_DENSE = 0,  /* form K, factor, solve (Alg. DenseDualSolve) */
  DNGD_PCG = 1     /* matrix-free: J never formed; Nystrom-preconditioned CG on
                      K + lambda I (Alg. PCGStep); precision must be a mixed mode
                      (FP32 jets and FP32 factor-form operator) */
};

/* Trailing updates of the exact-Gram modes' factorisation
 * (dngd_problem_desc.factor_update) */
enum dngd_factor_update {
  DNGD_FACTOR_SLICED = 0,       /* the first 64 columns of each step's update
                                   in double-float, the rest exact products
                                   of six 8-bit slices on the tensor cores,
                                   on a side stream (look-ahead) */
  DNGD_FACTOR_DF = 1            /* the whole update in double-float
                                   arithmetic, no look-ahead: what a batch of
                                   exact-Gram instances uses, all instances'
                                   steps in one launch per kernel; a single
                                   context with this setting computes the
                                   same factor as its batch */
};

/* Which form of the damped Gauss-Newton system the dense FP64 solver
 * factors (dngd_problem_desc.solve_space).  Both give the same step: the
 * dual (K + lambda I) y = r, v = -J^T y with K = J J^T [m x m] (Thm. 3.1,
 * push-through), or the primal (J^T J + lambda I) v = -J^T r [n x n]
 * (Prop. 3.1), and likewise the geodesic acceleration (Prop. 3.2: primal
 * (J^T J + lambda I) a = -J^T f_vv; dual, in the push-through form this
 * library uses, a = -J^T (K + lambda I)^{-1} f_vv).  The primal form costs
 * O(m n^2 + n^3) time and n x n memory, the dual O(m^2 n + m^3) and m x m
 * (Sec. 4.4), so the smaller of m and n decides which is cheaper. */
enum dngd_solve_space {
  DNGD_SPACE_DUAL = 0,          /* residual space (m x m) */
  DNGD_SPACE_PRIMAL = 1,        /* parameter space (n x n); precision
                                   DNGD_FP64 with solver DNGD_DENSE only */
  DNGD_SPACE_AUTO = 2           /* primal when precision is DNGD_FP64, the
                                   solver DNGD_DENSE and n < m; else dual */
};

/* GEMMs of the matrix-free operator (dngd_problem_desc.pcg_operator) */
enum dngd_pcg_operator {
  DNGD_PCG_OP_TC3 = 0,          /* 3xTF32 on the tensor cores */
  DNGD_PCG_OP_COMPENSATED = 1   /* FP32 SIMT, compensated accumulation */
};

#define DNGD_MAX_LAYERS 12
#define DNGD_MAX_DIM 8
#define DNGD_MAX_CLASSES 4

/* One residual class gamma (Sec. 2.2): N_gamma points and the linear
 * operator Op u = c_val u + sum_k c_grad[k] d_k u + c_lap sum_{k: lap_mask[k]} d_kk u.
 * The class residual is (Op u(x_i) - target_i) / sqrt(count). */
typedef struct {
  int count;
  double c_val;
  double c_grad[DNGD_MAX_DIM];
  double c_lap;
  int lap_mask[DNGD_MAX_DIM];
} dngd_class_desc;

typedef struct {
  int n_layers;                      /* affine layers (hidden + output), >= 1 */
  int widths[DNGD_MAX_LAYERS + 1];   /* widths[0] = d_in, widths[n_layers] = 1 */
  int n_classes;
  dngd_class_desc classes[DNGD_MAX_CLASSES];
  int precision;                     /* enum dngd_precision */
  int solver;                        /* enum dngd_solver */
  double lambda;                     /* Levenberg-Marquardt damping, > 0;
                                        FP64 contexts also accept a finite
                                        lambda <= 0, with which K + lambda I
                                        may be indefinite: the factorisation
                                        then reports DNGD_ERR_NOT_SPD and the
                                        failing column */
  int use_ga;                        /* geodesic acceleration on/off */
  double eps_norm;                   /* GA guard: accept only if ||v|| > eps_norm */
  double ga_ratio_max;               /* GA threshold on 2||a||/||v|| (paper: 0.5) */
  /* mixed precision refinement (ignored for DNGD_FP64) */
  int refine_max_it;                 /* PCG iterations per solve, e.g. 200 */
  double refine_tol;                 /* stop at ||rhs - A x|| <= tol ||rhs|| */
  double shift_mu;                   /* extra diagonal shift of the factored
                                        preconditioner K_lowp + (lambda+mu) I */
  /* matrix-free PCG solver (DNGD_PCG) */
  int pcg_rank;                      /* landmarks ell (<= m; default 512) */
  double pcg_tol;                    /* stop at ||rhs - A x|| <= tol ||rhs|| */
  int pcg_max_it;
  uint64_t pcg_seed;                 /* reserved (landmarks come from
                                        dngd_set_landmarks or are evenly spaced) */
  int keep_gram;                     /* keep K + lambda I for dngd_get_stage(6)
                                        (debug; one extra m x m buffer) */
  double lambda_cap;                 /* > 0: the damping rule of the paper's
                                        experiments (App. A.3 tables),
                                        lambda_k = min(L(theta_k), lambda_cap)
                                        with L = 1/2 ||r(theta_k)||^2, taken by
                                        every synchronous step (dngd_step)
                                        right after the residuals; lambda (or
                                        dngd_set_lambda) is then ignored by
                                        those steps.  A loss that is zero or
                                        not finite gives lambda_cap.  The
                                        asynchronous and batched steps keep
                                        the lambda of the last synchronous
                                        step.  0: fixed lambda. */
  int pcg_operator;                  /* enum dngd_pcg_operator (DNGD_PCG): the
                                        GEMMs of the factor-form operator
                                        K v = J (J^T v) and of the landmark
                                        columns.  0: 3xTF32 on the
                                        tensor cores (operands split into two
                                        TF32 terms, three products; TMEM
                                        chunks of 128 K-elements added in
                                        round-to-nearest FP32);
                                        1: FP32 SIMT with compensated
                                        (Kahan) accumulation and FP64 row
                                        reductions, slower and more
                                        accurate (see dngd_kvp). */
  int factor_update;                 /* enum dngd_factor_update (exact-Gram
                                        modes, DNGD_DENSE): how the factor's
                                        trailing updates are computed.  Both
                                        keep ~2^-47 of each entry (the
                                        factor preconditions a refinement on
                                        the exact Gram).  Batches of
                                        exact-Gram instances always use
                                        DNGD_FACTOR_DF. */
  int solve_space;                   /* enum dngd_solve_space.  With the
                                        primal space, the system dimension
                                        of dngd_solve and of stages 6 and 7
                                        is n instead of m, and stages 1 and
                                        4 (the dual vectors) do not exist. */
} dngd_problem_desc;

typedef struct {
  double loss;              /* 1/2 ||r(theta)||^2 */
  double norm_v;            /* ||v|| */
  double norm_a;            /* ||a|| (0 when GA is off) */
  double ga_ratio;          /* 2||a||/||v|| */
  int ga_accepted;
  int solve_iters[2];       /* CG/refinement iterations for r and for f_vv */
  double solve_relres[2];   /* final ||rhs - A x|| / ||rhs|| */
  int not_spd_column;       /* failing pivot column, or -1 (a parameter
                               index in the primal space, whose factored
                               system is J^T J + lambda I) */
  int device_status;        /* raw device status word */
  float phase_ms[8];        /* jets+J, Gram, factor, solve r, f_vv, solve f_vv,
                               finish, total (filled when timing is enabled) */
  double shift_used;        /* diagonal shift mu of the factored preconditioner
                               (mixed paths).  Starts at max(shift_mu, the
                               shift that factored in the previous step) and
                               is raised x3 (at least to 1e-6 trace(K)/m) on
                               a failed low-precision factorisation, up to 12
                               tries; the refinement keeps the exact lambda. */
  int factor_attempts;      /* low-precision factorisations this step (mixed) */
  float jt_ms, j_ms;        /* durations of the first J^T p and J u launches of
                               the refinement (mixed, timing enabled): each
                               reads the FP32 J once */
  double lambda_used;       /* the damping this step solved with */
  float gram_kernel_ms;     /* duration of the Gram's product kernel alone
                               (tensor-core modes, timing enabled; without
                               the slicing and the split-K reduction) */
} dngd_step_info;

typedef struct dngd_ctx dngd_ctx;

/* Human-readable message for a status code. */
const char* dngd_status_string(dngd_status s);

/* Library version string. */
const char* dngd_version(void);

/* Number of CUDA kernel launches this library has issued so far (all
 * contexts, host-side counter).  Differences bracket a region of interest. */
uint64_t dngd_launch_count(void);

/* Number of parameters n of the MLP described by desc (Sec. 2.1 layout). */
int64_t dngd_num_params(const dngd_problem_desc* desc);

/* Create a step context for one problem shape.  Allocates the workspace
 * (J, K / factor, jet buffers, Krylov vectors) with cudaMalloc on the current
 * device.  stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: INVALID_ARG for an inconsistent descriptor, OOM, CUDA. */
dngd_status dngd_create(dngd_ctx** out, const dngd_problem_desc* desc, void* stream);

/* Device bytes dngd_create would allocate for desc. */
dngd_status dngd_workspace_bytes(const dngd_problem_desc* desc, size_t* bytes);

dngd_status dngd_destroy(dngd_ctx* ctx);

/* Enable (1) or disable (0) per-phase CUDA-event timing in dngd_step_info. */
dngd_status dngd_set_timing(dngd_ctx* ctx, int enable);

/* Override the damping lambda for the following calls (> 0; FP64 contexts
 * also accept a finite lambda <= 0, as dngd_create).  A context whose
 * descriptor sets lambda_cap applies the paper's rule lambda_k = min(L, cap)
 * in each synchronous step instead. */
dngd_status dngd_set_lambda(dngd_ctx* ctx, double lambda);

/* One D-NGD step (Alg. DenseDualSolve or PCGStep; push-through recovery).
 *   theta [n], X [m x d_in], target [m]: inputs (float64).
 *   delta_out [n]: the step to add to theta (float64).
 *   info: optional (NULL allowed); when given, the call synchronises the
 *   stream and fills it.
 * Keeps r, J, the factor / preconditioner and v for dngd_solve and the
 * stage accessors below until the next step. */
dngd_status dngd_step(dngd_ctx* ctx, const double* theta, const double* X, const double* target,
                      double* delta_out, dngd_step_info* info);

/* Solve (K + lambda I) x = rhs with the factor / preconditioner of the last
 * dngd_step (Remark 3.1: the GA solve reuses the same operator).
 * rhs [m] -> x [m], float64; a context in the primal space solves
 * (J^T J + lambda I) x = rhs, rhs [n] -> x [n].  Errors: STATE if no step
 * was taken. */
dngd_status dngd_solve(dngd_ctx* ctx, const double* rhs, double* x_out);

/* The space a context's dense solver works in (enum dngd_solve_space:
 * DNGD_SPACE_AUTO resolved at dngd_create), or -1 for a NULL context. */
int dngd_solve_space_of(const dngd_ctx* ctx);

/* Loss L(theta + eta_j delta) = 1/2 ||r||^2 for k step sizes (the line search
 * of Alg. D-NGD Workflow).  etas [k] host array; loss_out [k] host array.
 * delta may be NULL (then every entry is L(theta)).  Synchronises. */
dngd_status dngd_loss(dngd_ctx* ctx, const double* theta, const double* X, const double* target,
                      const double* delta, const double* etas, int k, double* loss_out);

/* Grid line search and update: picks eta* = argmin over etas of
 * L(theta + eta delta) (first minimum in the given order) and writes
 * theta_out = theta + eta* delta.  theta_out may alias theta.  eta_out host. */
dngd_status dngd_line_search(dngd_ctx* ctx, const double* theta, const double* X, const double* target,
                             const double* delta, const double* etas, int k, double* theta_out,
                             double* eta_out);

/* The same line search without synchronising: the k losses, the argmin and
 * theta += eta* delta all stay on the device (theta, X, target, delta must be
 * device pointers; theta is updated in place; etas is a host array, k <= 64,
 * copied before the call returns).  The losses are 2x the loss (||r||^2). */
dngd_status dngd_line_search_async(dngd_ctx* ctx, double* theta, const double* X, const double* target,
                                   const double* delta, const double* etas, int k);

/* ---- the optimizer loop ------------------------------------------------------
 * D-NGD training (Alg. "D-NGD Workflow"): each iteration takes one step
 * (dngd_step, so the descriptor's damping rule lambda_k = min(L, cap) of
 * App. A.3 applies) and the grid line search with the update of theta, until
 * max_iters iterations, the wall-clock budget or the loss target.  Between
 * iterations the collocation points may be resampled (the paper redraws them
 * for several problems): the callback rewrites X [m x d] and target [m] in
 * place, every `resample_every` iterations, and must have finished its writes
 * when it returns.  A step that reports NO_CONVERGE is still taken; any other
 * failure ends the loop with that status (theta then holds the last iterate).
 */
typedef dngd_status (*dngd_resample_fn)(void* user, int iteration, double* X, double* target);

typedef struct {
  int max_iters;              /* > 0 */
  double time_budget_s;       /* wall clock, checked before each iteration (0: none) */
  double loss_target;         /* stop once L(theta) <= loss_target (0: none) */
  int resample_every;         /* resample before iteration i when i > 0 and
                                 i % resample_every == 0 (0: never) */
  dngd_resample_fn resample;  /* required when resample_every > 0 */
  void* user;                 /* passed to resample */
  const double* etas;         /* line-search grid, host [k]; NULL: 2^-j, j = 0..30 */
  int k;                      /* grid size (<= 64) when etas is given */
} dngd_train_cfg;

enum dngd_train_stop {
  DNGD_STOP_ITERS = 0,   /* max_iters iterations done */
  DNGD_STOP_BUDGET = 1,  /* wall-clock budget spent */
  DNGD_STOP_LOSS = 2     /* loss target reached */
};

typedef struct {
  int iters;          /* iterations completed */
  int stop;           /* enum dngd_train_stop */
  double loss;        /* L(theta) of the final iterate (on the last X, target) */
  double elapsed_s;   /* wall clock of the loop */
} dngd_train_result;

/* theta [n], X, target: device pointers (theta is updated in place);
 * loss_history: host [max_iters] or NULL, L(theta_i) at the start of
 * iteration i; result: host.  Synchronises once per iteration (the step's
 * damping rule reads the loss). */
dngd_status dngd_train(dngd_ctx* ctx, double* theta, double* X, double* target, const dngd_train_cfg* cfg,
                       double* loss_history, dngd_train_result* result);

/* Residuals and Jacobian at theta (Sec. 2.2) through the step's own kernels
 * and precision.  r_out [m] float64; J_out [m x n] row-major float64 or NULL. */
dngd_status dngd_residual_jacobian(dngd_ctx* ctx, const double* theta, const double* X,
                                   const double* target, double* r_out, double* J_out);

/* Second directional derivative f_vv = d^2/dt^2 r(theta + t v)|_0 (Sec. 3.2)
 * through the step's f_vv kernel.  v [n] -> fvv_out [m], float64. */
dngd_status dngd_fvv(dngd_ctx* ctx, const double* theta, const double* X, const double* target,
                     const double* v, double* fvv_out);

/* Stage outputs of the last dngd_step, copied to dst (host or device):
 * which = 0 r [m], 1 alpha [m], 2 v [n], 3 f_vv [m], 4 beta [m], 5 a [n],
 *         6 lower triangle of K + lambda I [m x m] row-major (dense, before
 *           factorisation; the upper triangle is left as zero),
 *         7 Cholesky factor L [m x m] row-major (dense solver),
 *           (6 and 7 in the primal space: J^T J + lambda I and its factor,
 *           [n x n]; 1 and 4 then give DNGD_ERR_STATE),
 *         8 landmark columns K_{:,I} [m x ell] row-major (PCG solver),
 *         9 exact Gram J J^T [m x m] row-major, full symmetric, no lambda
 *           (DNGD_MIXED_OZ, DNGD_MIXED_OZ64),
 *        10 the preconditioner's explicit inverse factor L^{-1} [m x m]
 *           row-major lower (mixed paths, FP32 values),
 *        11 the FP64 Cholesky factor of the exact Gram + (lambda + mu) I
 *           [m x m] row-major lower (DNGD_MIXED_OZ, DNGD_MIXED_OZ64).
 * Values are converted to float64. */
dngd_status dngd_get_stage(dngd_ctx* ctx, int which, double* dst);

/* Landmarks of the Nystrom preconditioner (Sec. 3.3.1: a landmark is one
 * scalar residual; Alg. "Nystrom construction" picks the set I).  idx [ell]
 * host array of residual indices in [0, m), ell <= the desc's pcg_rank.
 * Without this call the context uses ell evenly spaced residuals.
 * PCG contexts only; INVALID_ARG otherwise. */
dngd_status dngd_set_landmarks(dngd_ctx* ctx, const int64_t* idx, int ell);

/* Kernel-vector product w = J (J^T v) + lambda v (Def. 3.3) with the stream
 * factors of the last dngd_step, J never formed.  v [m] -> w_out [m].
 * PCG contexts only (STATE before the first step).  Accuracy: the 3xTF32
 * operator's products keep about 2^-22 of each FP32 operand (the split drops
 * the third TF32 term) and sum in FP32 chunks; the compensated operator
 * rounds each FP32 product once and sums with Kahan compensation.  CG with
 * an inexact product converges on its recursive residual, while the true
 * residual ||rhs - (K + lambda I) x|| stalls near the product's error times
 * cond(K + lambda I). */
dngd_status dngd_kvp(dngd_ctx* ctx, const double* v, double* w_out);

/* Nystrom preconditioner of the last step: z = P^{-1} x with
 * P^{-1} = U (Lambda_hat + lambda I)^{-1} U^T + (I - U U^T) / lambda
 * (Eq. spec_precond_nystrom_main_final), applied as (K_hat + lambda I)^{-1}
 * through the Woodbury identity.  x [m] -> z_out [m].  PCG contexts only. */
dngd_status dngd_precond_apply(dngd_ctx* ctx, const double* x, double* z_out);

/* ---- asynchronous stepping and batches of independent instances --------
 * A dense context can step without any host synchronisation: the step reads
 * its inputs from the context's own staging buffers, runs the refinement for
 * a fixed budget of iterations (twice the last synchronous step's count plus
 * two, at least 8 and at most refine_max_it; each kernel of an iteration is
 * a no-op once the device-side convergence flag is set, so results equal the
 * synchronous step's) and factors the low-precision Gram once with the shift
 * of the previous synchronous step.  That step is captured once into a CUDA
 * graph and replayed (re-captured when lambda, the shift or the budget
 * changes).  The first asynchronous step of a context, and the step after a
 * failed factorisation or after a captured solve that stopped at its budget
 * above refine_tol, runs synchronously. */

/* Enqueue one step on the context's stream (inputs are copied first; pointers
 * may be host or device; delta_out is written when the stream reaches it).
 * Dense solver only. */
dngd_status dngd_step_async(dngd_ctx* ctx, const double* theta, const double* X, const double* target,
                            double* delta_out);

/* Wait for the last dngd_step_async and fill info (may be NULL).  Returns the
 * step's device status (NOT_SPD means: call again, the next step re-searches
 * the shift). */
dngd_status dngd_step_wait(dngd_ctx* ctx, dngd_step_info* info);

/* A batch of independent D-NGD instances of different shapes (e.g. many
 * small PINNs of uneven m and n).  Every instance has its own context and
 * stream; one batch step is ONE CUDA-graph launch that forks to all instance
 * streams (each runs its asynchronous step) and joins.  When every instance
 * is an exact-Gram mode (DNGD_MIXED_OZ / OZ64), the instances' steps run in
 * two halves around one batched factorisation: per 64-column step, one
 * launch each for all instances' diagonal blocks, panel solves and trailing
 * updates (double-float; such instances are created with factor_update =
 * DNGD_FACTOR_DF, also for their synchronous steps).  The per-instance
 * arithmetic never depends on the batch, so each result equals the instance
 * stepped alone with the same descriptor (factor_update = DNGD_FACTOR_DF for
 * exact-Gram modes).  An instance whose captured step failed its factor or
 * stopped its refinement at the captured budget above tolerance is redone
 * synchronously and the graph is re-captured. */
typedef struct dngd_batch dngd_batch;

/* descs [count] (dense solver); stream: master stream or NULL (own stream). */
dngd_status dngd_batch_create(dngd_batch** out, const dngd_problem_desc* descs, int count, void* stream);
dngd_status dngd_batch_destroy(dngd_batch* batch);
int dngd_batch_size(const dngd_batch* batch);

/* One step of every instance: arrays of count pointers (host or device), the
 * same conventions as dngd_step.  infos [count] or NULL.  Synchronises the
 * master stream; returns the first failing instance's status.  The first call
 * steps each instance synchronously; later calls launch the batch graph. */
dngd_status dngd_batch_step(dngd_batch* batch, const double* const* theta, const double* const* X,
                            const double* const* target, double* const* delta_out, dngd_step_info* infos);

/* The context of instance i (for dngd_get_stage, dngd_line_search, ...). */
dngd_ctx* dngd_batch_context(dngd_batch* batch, int i);

/* Failure detection check (no counterpart in the paper): runs one bounded
 * device-side wait that cannot be satisfied (a grid barrier missing one
 * arrival) with a limit of limit_ms (0 < limit_ms <= 1000).  The wait runs
 * out, the kernel records its timeout and returns, and the call reports
 * DNGD_ERR_TIMEOUT; the context stays usable.  The same bounded waits guard
 * every device-side wait of the library (TMA / MMA / epilogue mbarriers, the
 * persistent PCG's grid barriers). */
dngd_status dngd_check_wait_expiry(dngd_ctx* ctx, double limit_ms);

/* ---- serving: a request loop over PINN solve jobs ------------------------
 * A job is one PINN solve: a problem, initial parameters, collocation data
 * and a number of D-NGD iterations (step + 31-point line search + update).
 * Jobs are admitted first come, first served when a slot is free and their
 * device footprint fits in what is left of the HBM budget (a job that can
 * never fit is rejected with DNGD_ERR_BUDGET).  Admitted jobs keep their
 * state on the device and always have their next iteration in flight on their
 * own stream, so iterations of different jobs overlap on the GPU (continuous
 * batching); a finished job releases its memory and slot at once.  A failing
 * job is marked FAILED without affecting others.  One worker thread owns all
 * device work of the server; submit / poll / cancel / stats are thread-safe. */
typedef struct dngd_server dngd_server;

typedef struct {
  size_t hbm_budget_bytes;  /* 0: 80% of the free device memory at creation */
  int max_slots;            /* jobs running at once (>= 1) */
  int line_search_points;   /* grid eta_j = 2^-j, j < points (0: 31) */
} dngd_server_cfg;

typedef struct {
  dngd_problem_desc desc;   /* dense solver */
  const double* theta0;     /* [n] host or device; copied at submit */
  const double* X;          /* [m x d] host or device; copied at submit */
  const double* target;     /* [m] host or device; copied at submit */
  int n_steps;              /* D-NGD iterations to run */
} dngd_job_desc;

enum dngd_job_states { DNGD_JOB_QUEUED = 0, DNGD_JOB_RUNNING = 1, DNGD_JOB_DONE = 2, DNGD_JOB_FAILED = 3,
                       DNGD_JOB_CANCELLED = 4 };

typedef struct {
  int state;                /* enum dngd_job_states */
  int steps_done;
  dngd_status status;       /* failure reason (FAILED) */
  double loss;              /* 1/2 ||r||^2 at the start of the last step */
  double queue_s, run_s;    /* time queued / running so far */
} dngd_job_state;

typedef struct {
  double steps_per_s;       /* completed iterations / time since the first submit */
  double p50_ms, p99_ms;    /* per-iteration latency on the device (step + line search) */
  long long steps_total;
  int admitted, rejected, done, failed, running, queued;
  size_t hbm_used_bytes, hbm_budget_bytes;
} dngd_serving_stats;

dngd_status dngd_server_create(dngd_server** out, const dngd_server_cfg* cfg);
dngd_status dngd_server_destroy(dngd_server* server);   /* cancels running jobs */
dngd_status dngd_submit(dngd_server* server, const dngd_job_desc* job, uint64_t* job_id);
/* theta_out [n] (host or device, may be NULL) is filled once the job is DONE. */
dngd_status dngd_poll(dngd_server* server, uint64_t job_id, dngd_job_state* state, double* theta_out);
dngd_status dngd_cancel(dngd_server* server, uint64_t job_id);
dngd_status dngd_server_stats(dngd_server* server, dngd_serving_stats* stats);
/* Block until no job is queued or running (TIMEOUT after timeout_s). */
dngd_status dngd_server_drain(dngd_server* server, double timeout_s);

/* Gram matrix without any device allocation (the paper has no counterpart:
 * this is a library facility).  K = J J^T + shift I for a BF16 matrix J on the
 * tcgen05 tensor cores, the same kernels as the step's Gram.
 *   J      device, [m x ld] row-major bfloat16, 16-byte aligned, ld >= n and
 *          ld * 2 a multiple of 16 bytes; columns n..ld-1 are ignored.
 *   K      device, [m x ldk] float32 output: the lower triangle with the
 *          diagonal is written, the strict upper triangle is set to 0.
 *   stream a cudaStream_t (NULL = legacy default stream).
 * For callers that cannot call cudaMalloc at this point (their framework owns
 * every device allocation, or an allocation would disturb the surrounding
 * work).  The call allocates nothing: its scratch (split-K partial tiles, the
 * tile list, a status word) is one static 16 MiB device array that every GPU
 * which loads this library keeps until the process exits, so m is limited to
 * 2000; larger m returns DNGD_ERR_INVALID_ARG with a message on stderr.
 * The first call on each device looks up the array's device address (with
 * that device current).
 * All calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU (other streams, other threads) race on it.  The call
 * synchronises the stream and returns DNGD_ERR_TIMEOUT if a bounded wait in
 * the kernel gave up. */
dngd_status dngd_gram_bf16_noalloc(const void* J, int m, int n, long long ld, float* K, long long ldk,
                                   double shift, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DNGD_H */
