/*
 * liblqr: segment-parallel Riccati recursion for discrete-time, time-varying,
 * finite-horizon LQR on one GB300 GPU (sm_103a).
 *
 * Problem (Section II, Eq. 1-2 of Laine & Tomlin, "The Parallelization of
 * Riccati Recursion"):
 *     minimise  sum_{t<T} 1/2 x_t'Q_t x_t + u_t'S_t x_t + 1/2 u_t'R_t u_t + q_t'x_t + r_t'u_t
 *               + 1/2 x_T'Q_T x_T + q_T'x_T
 *     subject to x_{t+1} = A_t x_t + B_t u_t + c_t,  x_0 = x0.
 * The paper's names: Q_xx = Q, Q_uu = R, Q_ux = S (m x n), q_x1 = q, q_u1 = r,
 * F_x = A, F_u = B, f_1 = c, x_init = x0. R_t must be positive definite and the
 * problem strictly convex (Section II, assumption after Eq. 2).
 *
 * Method (Sections II-A to II-C): the horizon is split into K segments. Every
 * segment but the last runs the constraint-explicit backward sweep of Section
 * II-B with its end state x_term as a parameter; the last runs a plain Riccati
 * sweep from the terminal cost. The segment summaries are coupled through the
 * link equations of Eq. 10-11 (a block-tridiagonal FP64 system in the K-1 link
 * states), whose backward elimination yields the global value function at the
 * segment boundaries. A second, exact sweep per segment (the smoothing pass of
 * Section III-A, started from that global value function) then gives the serial
 * feedback policies K_t, k_t, and a forward rollout per segment from its link
 * state gives x_t, u_t and the multipliers lambda_t of Eq. 3.
 *
 * Memory and layout. All problem and solution arrays are DEVICE pointers owned
 * by the caller, row-major, stage-major and contiguous:
 *     A[T][n][n]  B[T][n][m]  c[T][n]  Q[T+1][n][n] (slot T = Q_T)
 *     R[T][m][m]  S[T][m][n] (NULL means S = 0)  q[T+1][n] (slot T = q_T)
 *     r[T][m]     x0[n]
 *     K[T][m][n]  k[T][m]  x[T+1][n]  u[T][m]  P[T+1][n][n]  p[T+1][n]  lam[T+1][n]
 * Q and R are read symmetrised, 1/2 (M + M'). The element type is double for
 * LQR_FP64 and LQR_MIXED_*, float for LQR_FP32.
 *
 * Streams and errors. Every call validates its arguments on the host first and
 * returns LQR_ERR_INVALID_ARG without touching the GPU when they are wrong.
 * Solves are enqueued on the caller's stream (a cudaStream_t passed as void*;
 * NULL = the legacy default stream) and return before the GPU finishes.
 * Conditions found on the device (a non positive-definite pivot, a segment that
 * cannot absorb its end constraint, non-finite values) are recorded in a status
 * word of the handle and read back by lqr_report(), which synchronises the
 * stream. No call traps or aborts. A handle must not be used from two host
 * threads at once; solves on one handle are stream-ordered on the stream given.
 */
#ifndef LQR_H
#define LQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LQR_OK = 0,
  LQR_ERR_INVALID_ARG = 1,        /* bad pointer, size or option (host check)              */
  LQR_ERR_NOT_PD = 2,             /* R_t + B_t'P B_t or a link block not positive definite */
  LQR_ERR_SEGMENT_INFEASIBLE = 3, /* a segment cannot absorb its end-point constraint      */
  LQR_ERR_NONFINITE = 4,          /* NaN or Inf produced                                   */
  LQR_ERR_NO_CONVERGENCE = 5,     /* iterative refinement did not reach opts.tol           */
  LQR_ERR_TIMEOUT = 6,            /* a bounded device wait ran out                         */
  LQR_ERR_CUDA = 7,               /* a CUDA runtime call failed                            */
  LQR_ERR_OOM = 8,                /* workspace allocation failed                           */
  LQR_ERR_UNSUPPORTED = 9,        /* valid request this build does not implement           */
  LQR_ERR_CAPACITY = 10           /* larger than a fixed-capacity entry point accepts      */
} lqr_status;

typedef enum {
  LQR_FP64 = 0,       /* all arithmetic in FP64 (the plain method)                          */
  LQR_FP32 = 1,       /* FP32 data and arithmetic, sweeps and link solve alike               */
  LQR_MIXED_TF32 = 2, /* FP64 data; FP32 sweeps, FP64 factor/link solve, FP64 KKT refinement */
  LQR_MIXED_BF16 = 3, /* reserved (LQR_ERR_UNSUPPORTED)                                      */
  LQR_MIXED_FP32 = 4  /* FP64 data and solution; the solve runs the LQR_FP32 path on an FP32
                         copy of the data (LQR_FORM_MULTIPLIER only) and the FP64 KKT residual
                         drives iterative refinement to opts.tol. Where the FP32 fast sweeps
                         apply, each correction reuses the solve's K_t, P_t and M_uu^-1
                         (vector-only passes over the same segments; the handle then holds
                         (T+1) n^2 + T m^2 + K n^2 more floats), else it is a whole FP32 solve */
} lqr_precision;

/* How a segment carries its unknown end state (both reach the same summary
 * of Eq. 9 in exact arithmetic):
 *  LQR_FORM_MULTIPLIER  - the end-point constraint x_T = x_term is dualised: the
 *      sweep carries its multiplier mu (the mu of Eq. 10) as the parameter,
 *      starting from V = 0, dV/dx = mu. Every stage is a plain Riccati stage.
 *      The link solve works with these dual summaries. Default.
 *  LQR_FORM_CONSTRAINED - the constraint-explicit sweep of Section II-B
 *      (Eq. 9-16): x_term is the parameter and the first ceil(n/m) stages from
 *      the segment end absorb the end-point constraint by range/null-space
 *      splits. Its x_term blocks lose accuracy like cond(R_L)^2 * eps, where
 *      R_L is the ceil(n/m)-stage reachability matrix at the segment end. */
typedef enum { LQR_FORM_MULTIPLIER = 0, LQR_FORM_CONSTRAINED = 1 } lqr_form;

/* How the link system of Section II-A (neighbouring segments' multipliers
 * related through the unknown link points, Eq. 10-11) is solved. Both give the
 * same Pi_j, pi_j and link points in exact arithmetic.
 *  LQR_LINK_CHAIN - block elimination from the last link to the first
 *      (K-1 dependent steps), each step spread over a cluster of CTAs.
 *  LQR_LINK_SCAN  - the segment summaries composed pairwise as an associative
 *      suffix scan (ceil(log2 K) levels of independent compositions, one CTA
 *      each), then the link feedback of every segment in one parallel pass;
 *      LQR_FP32 with LQR_FORM_MULTIPLIER only (else LQR_ERR_UNSUPPORTED), and
 *      n up to the shared-memory limit (about 80; larger n: LQR_ERR_UNSUPPORTED).
 *      The paper does not use a scan: it solves the link system directly.
 *  LQR_LINK_AUTO  - the scan where it applies, else the chain. */
typedef enum { LQR_LINK_AUTO = 0, LQR_LINK_CHAIN = 1, LQR_LINK_SCAN = 2 } lqr_link;

typedef struct lqr_handle lqr_handle;

/* One problem: dimensions and device pointers (layout above). */
typedef struct {
  int n, m, T;
  const void *A, *B, *c, *Q, *R, *S, *q, *r, *x0;
} lqr_problem;

/* Outputs: caller-allocated device arrays; any may be NULL except where noted.
 * x and u are written when non-NULL; lam needs x and u. */
typedef struct {
  void *K, *k, *x, *u, *P, *p, *lam;
} lqr_solution;

typedef struct {
  lqr_precision prec;
  int num_segments;   /* K >= 1; 0 = choose automatically                         */
  double tol;         /* refinement target on |KKT w - b|_inf / |b|_inf            */
  int max_refine;     /* iterative-refinement corrections allowed (double data only);
                         needs K, k, x, u and lam in the solution                   */
  int debug_checks;   /* reserved, 0                                              */
  lqr_form form;      /* segment parametrisation, see lqr_form                    */
  int residual;       /* 1 = compute the FP64 KKT residual of the returned solution
                         (needs x, u, lam); implied by max_refine > 0              */
  lqr_link link;      /* link-system solver, see lqr_link (0 = automatic)         */
  long long spin_limit; /* polls (about 32 ns apart) of a bounded device wait before it
                         gives up with LQR_ERR_TIMEOUT: the tensor-core sweep's waits
                         for its own products (it then releases its tensor memory and
                         returns; 0 = 2^26, about two seconds) and the refinement
                         corrections' waits for their own bulk copies (the copies
                         still in flight then get one more wait at the default limit;
                         0 = 2^25)                                                  */
  int refine_plain;   /* mixed modes: 0 = the refinement loop runs as one CUDA graph
                         (a WHILE node around one iteration, ended on the device at
                         convergence) where the graph can be built; 1 = the loop's
                         kernels are launched one by one from the host, every
                         iteration up to max_refine (a converged one returns at once
                         on the device). Same kernels and results either way.     */
} lqr_opts;

/* Scalars of the last solve, read back by lqr_report(). */
typedef struct {
  int status;          /* lqr_status of the device side of the last solve */
  int num_segments;    /* K used                                          */
  int refine_iters;    /* refinement iterations run                       */
  int bad_stage;       /* first stage index a device check flagged, or -1 */
  double cost;         /* optimal objective J* (Eq. 1) along x, u         */
  double kkt_residual; /* normwise backward error of Eq. 3 when computed, else -1:
                          |KKT w - b|_inf / (|KKT|_inf |w|_inf + |b|_inf)        */
  double kkt_rel;      /* |KKT w - b|_inf / |b|_inf when computed, else -1 */
} lqr_report_t;

/* Per-segment summary written by lqr_segment_summaries (FP64, per segment j),
 * five blocks S0[n][n], S1[n][n], S2[n][n], s3[n], s4[n]:
 *  LQR_FORM_CONSTRAINED: Vxx, Vzx, Vzz, vx, vz, the quadratic
 *      cost_to_go_{b_j}(x, x_term) of Eq. 9 at the segment start.
 *  LQR_FORM_MULTIPLIER: P, Z, -W, p, w of the dual value
 *      G(x, mu) = 1/2 x'P x + mu'Z x - 1/2 mu'W mu + p'x + w'mu (the segment cost
 *      plus mu'x_end, minimised over the controls), related to Eq. 9 by
 *      Vzz = W^-1, Vzx = -W^-1 Z, Vxx = P + Z'W^-1 Z, vz = -W^-1 w, vx = p + Z'W^-1 w.
 * The last segment stores its plain Riccati value (P at its start in S0, p in
 * s3, zeros elsewhere). */
#define LQR_SUMMARY_DOUBLES(n) (3 * (size_t)(n) * (size_t)(n) + 2 * (size_t)(n))

/* Create a handle on CUDA device `device`. workspace_hint (bytes) pre-sizes the
 * device workspace; 0 = grow on first use. The handle owns the workspace. */
lqr_status lqr_create(lqr_handle **h, int device, size_t workspace_hint);

/* Free the handle and its workspace (synchronises the device first). */
lqr_status lqr_destroy(lqr_handle *h);

/* Segment boundaries b_0 = 0 < b_1 < ... < b_K = T used for K segments:
 * b_j = floor(j*T/K). Writes K+1 ints to bounds (host memory). Fails with
 * LQR_ERR_SEGMENT_INFEASIBLE when some segment would be shorter than
 * ceil(n/m) stages, the least a segment needs to reach an arbitrary end state
 * (Section II-B, the feasibility remark after Eq. 16). */
lqr_status lqr_partition(int n, int m, int T, int K, int *bounds);

/* Solve one problem (Sections II-A..II-C). Asynchronous on `stream`. */
lqr_status lqr_solve(lqr_handle *h, const lqr_problem *prob, const lqr_opts *opts,
                     const lqr_solution *sol, void *stream);

/* The same solve with HOST problem and solution pointers: copies the inputs
 * to the handle's device staging area, solves, copies the requested outputs
 * back and synchronises `stream` before returning. Host buffers should be
 * pinned for full copy bandwidth. */
lqr_status lqr_solve_host(lqr_handle *h, const lqr_problem *prob_host, const lqr_opts *opts,
                          const lqr_solution *sol_host, void *stream);

/* Many independent problems of uneven n, m, T in one solve (a batch). Two
 * schedules:
 *  - persistent: one launch; resident CTAs take the problems from a queue
 *    ordered by decreasing work (longest first) and solve each one whole as
 *    one segment (Riccati sweep, rollout, multipliers, objective). Used for
 *    LQR_FP32 multiplier-form batches that request x and u and fit the FP32
 *    sweep and rollout plans (n up to about 64, m up to 32), with
 *    opts->num_segments 0 or 1;
 *  - per step: one launch per step over all (problem, segment) units, the
 *    segment count of each problem from the batch shape (one segment per
 *    problem when the batch has at least one problem per SM, else about two
 *    units per SM) unless opts->num_segments > 0 fixes it.
 * With opts->num_segments = 0 and both schedules possible, the first batch of
 * a shape bucket (problem count and largest horizon by powers of two, largest
 * n and m) is solved with each schedule and timed (that call synchronises
 * `stream`); the handle keeps the faster schedule for the bucket.
 * probs and sols are HOST arrays of nprob entries whose pointers are device
 * arrays (layout above); all problems share opts (precision, form
 * LQR_FORM_MULTIPLIER; no refinement). segments (host, nprob ints, or NULL)
 * receives the segment count used per problem. Otherwise asynchronous on
 * `stream`; the host arrays may be reused as soon as the call returns. */
lqr_status lqr_solve_batched(lqr_handle *h, int nprob, const lqr_problem *probs, const lqr_opts *opts,
                             const lqr_solution *sols, int *segments, void *stream);

/* Synchronise `stream` and read back per-problem status (lqr_status) and
 * objective J* of the last lqr_solve_batched call (host arrays of nprob
 * entries; cost may be NULL). */
lqr_status lqr_report_batched(lqr_handle *h, void *stream, int nprob, int *status, double *cost);

/* Gradients of a scalar loss L(x, u) of the optimal trajectory with respect to
 * every problem datum (implicit function theorem on the KKT system of Eq. 3;
 * the KKT matrix is symmetric, so its transpose solve is one more
 * segment-parallel Riccati solve with the same matrices and the linear costs
 * -dL/dx, -dL/du, c = 0, x0 = 0, recomputing the segment value functions).
 * prob: the forward problem; sol: its solution (x, u, lam required, from
 * lqr_solve with the same opts); grad_x [T+1][n] = dL/dx, grad_u [T][m] = dL/du
 * (device; NULL = 0). grads: device output arrays laid out like the problem
 * (A..x0, n/m/T equal to prob's; any pointer NULL = not wanted), receiving
 * dL/dA ... dL/dx0; dL/dQ and dL/dR are symmetric (Q and R enter symmetrised).
 * Asynchronous on `stream`; the handle's status covers the adjoint solve. */
lqr_status lqr_backward(lqr_handle *h, const lqr_problem *prob, const lqr_opts *opts,
                        const lqr_solution *sol, const void *grad_x, const void *grad_u,
                        const lqr_problem *grads, void *stream);

/* lqr_backward for a batch (host arrays of nprob entries; grad_x / grad_u are
 * host arrays of device pointers, or NULL). The adjoint solves run as one
 * batched solve; per-problem status through lqr_report_batched. */
lqr_status lqr_backward_batched(lqr_handle *h, int nprob, const lqr_problem *probs, const lqr_opts *opts,
                                const lqr_solution *sols, const void *const *grad_x,
                                const void *const *grad_u, const lqr_problem *grads, void *stream);

/* KKT residual of a given solution with NO device allocation. The paper has
 * no counterpart: this serves callers that may not allocate device memory
 * once running, such as hard real-time control loops (a model-predictive
 * controller whose cycle budget forbids cudaMalloc after start-up) and code
 * executing inside another framework's stream capture, and that hold no
 * liblqr handle (a handle owns a growable workspace).
 * Computes, for the solution sol (x, u, lam required) of prob, the same
 * quantities lqr_solve reports with opts.residual = 1: out[0] = normwise
 * backward error eta, out[1] = |KKT w - b|_inf / |b|_inf, out[2] = objective
 * J along (x, u). out is a caller-allocated DEVICE buffer of 3 doubles; prec
 * gives the element type of the data (float for LQR_FP32, else double).
 * Scratch memory is a fixed file-scope device array of
 * LQR_NOALLOC_MAX_STAGES + 9 doubles (about 512 KB) that every GPU loading the
 * library holds until exit; problems with T > LQR_NOALLOC_MAX_STAGES are
 * rejected with LQR_ERR_CAPACITY. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. The call only enqueues a
 * memset of the array's reduction slots and one kernel on `stream`. All calls
 * share the array, so calls whose executions overlap on the GPU (different
 * streams, or different host threads) race: serialise them. */
#define LQR_NOALLOC_MAX_STAGES 65536
lqr_status lqr_kkt_residual_noalloc(const lqr_problem *prob, const lqr_solution *sol, lqr_precision prec,
                                    double *out, void *stream);

/* Self-test of the tensor-core product unit the segment sweeps use on device
 * `device` (the tcgen05 TF32 products of Section II-B's stage terms, in the
 * operand forms the sweep issues: A from shared memory and from tensor
 * memory, 128-row tiles at row offsets 0 and 64, N = 64, 128, 192, and
 * accumulation with a negated A), against CUDA-core FP32 products of the same
 * operands, one CTA on deterministic data. errs (host, 5 doubles) receives
 * four normwise relative differences and a wait flag: [0] shared x shared
 * (N = 128), [1] tensor-memory A (N = 192), [2] tensor-memory A (N = 64, the
 * rows from 128 on), [3] |X - X| / |X| with the second product negated,
 * [4] 1 if a bounded completion wait ran out (then LQR_ERR_TIMEOUT).
 * TF32 operands carry 10 mantissa bits, so [0]-[2] are of order 1e-3 and
 * [3] of order 1e-6. Synchronous; allocates and frees a small device buffer. */
lqr_status lqr_tc_selftest(int device, double* errs);

/* The FP64 pivot reciprocal of the FP64 factorisations (the pivots of the
 * Cholesky / LDL' factors of R + B'PB and of the link blocks, Section II-B),
 * y[i] = 1 / d[i] from the FP32 hardware reciprocal refined by two
 * Newton-Raphson steps y <- y + y (1 - d y) (the division itself outside the
 * FP32 exponent range), exported so that its accuracy can be checked against
 * IEEE division. d, y: DEVICE arrays of count doubles. Asynchronous on stream. */
lqr_status lqr_rcp_newton_check(const double* d, double* y, int count, void* stream);

/* FP64 -> FP32 conversion of `count` values (DEVICE arrays), rounding to
 * nearest with ties to even as IEEE prescribes, computed with integer
 * operations on the bit patterns (the conversion instruction would occupy the
 * FP64 pipe): the kernel that makes the FP32 working copies of the mixed
 * modes. Asynchronous on `stream`. */
lqr_status lqr_convert_f64_to_f32(const double *src, float *dst, long long count, void *stream);

/* ---- Trajectory-optimisation outer loop --------------------------------------
 * Section I: trajectory optimisation reduces to a sequence of LQR subproblems.
 * lqr_sqp_solve runs Gauss-Newton multiple-shooting SQP on the nonlinear
 * tracking model
 *   x_{t+1} = A x_t + B u_t + beta tanh(C x_t),  x_0 = x0,
 *   J = sum_t 1/2 (x_t - xref_t)'Q (x_t - xref_t) + 1/2 u_t'R u_t
 *       + 1/2 (x_T - xref_T)'Q_T (x_T - xref_T),
 * each iteration: the LQR subproblem in the step (dx, du) at the iterate
 * (dynamics linearised at every stage, c_t the defect f(x_t, u_t) - x_{t+1},
 * the objective's exact quadratic model; one kernel), its solution by the
 * segment-parallel solver (the options in opts->sub), the l1 merit
 * J + nu D (D the defects' l1 norm, nu = max(nu_min, 2 max|lambda|)) at the
 * step lengths 0, 1, 1/2, ..., 1/128 (one kernel for all), the first length
 * with Armijo decrease phi(a) <= phi(0) + 1e-4 a (g'd - nu D(0)) (the full
 * step once |g'd - nu D(0)| <= 1e-12 max(1, |phi(0)|); 1/128 when none), and
 * the step (one kernel). Stops after max_iters iterations or once
 * a max|(dx, du)| <= tol max(1, max|(x, u)|) and D(a) <= tol.
 * Model arrays: DEVICE FP64, row-major; Q, R, Q_T symmetric positive definite.
 * x [T+1][n], u [T][m]: DEVICE FP64, the starting iterate on entry (need not
 * satisfy the dynamics), the last iterate on return. lam [T+1][n], K [T][m][n],
 * k [T][m]: DEVICE FP64 or NULL: the last subproblem's multipliers (those of
 * the nonlinear problem at convergence) and feedback policy (the stabilising
 * policy of Section I's model-predictive-control use). hist: HOST, NULL or
 * max_iters * LQR_SQP_HIST doubles, per iteration (a, J(a), D(a), merit, step,
 * nu). opts->sub.prec: LQR_FP64 or LQR_MIXED_FP32 (else LQR_ERR_UNSUPPORTED).
 * Synchronous: returns after the loop (each iteration reads its merit values
 * back). A failed subproblem returns its status. Workspace owned by the handle. */
typedef struct {
  int n, m, T;
  const double *A, *B, *C; /* n x n, n x m, n x n */
  double beta;
  const double *Q, *R, *QT; /* n x n, m x m, n x n */
  const double *xref;      /* [T+1][n] */
  const double *x0;        /* [n] */
} lqr_nl_model;

typedef struct {
  int max_iters;
  double tol;
  double nu_min;
  lqr_opts sub;            /* options of every LQR subproblem solve */
} lqr_sqp_opts;

typedef struct {
  int iters;               /* iterations taken */
  int converged;           /* 1 when the stopping test held */
  double cost, defect;     /* J and D at the returned iterate */
  double alpha, step;      /* the last step length and a max|(dx, du)| */
} lqr_sqp_report;

#define LQR_SQP_HIST 6

lqr_status lqr_sqp_solve(lqr_handle *h, const lqr_nl_model *model, const lqr_sqp_opts *opts, double *x, double *u,
                         double *lam, double *K, double *k, lqr_sqp_report *report, double *hist, void *stream);

/* The global policy and cost to go of every stage reconstructed in parallel
 * from the segments' parametric values (Section II-B with the global value of
 * Section III-A), in place of the sequential policy sweep of step A4.
 * The constraint-explicit sweeps give, at every stage t of segment j < K-1,
 * the cost to go of the rest of the segment as a function of (x_t, z) (Eq. 9
 * at stage t; z the segment's end state) and the stage's policy
 * u_t = Kx x + Kz z + k1; the link solve gives the global value
 * 1/2 z'P_e z + p_e'z at the segment's end. At every stage whose
 * constraint_to_go has no rows left, independently (one CTA per stage):
 *   P_t = Vxx - Vzx'(Vzz + P_e)^-1 Vzx,  p_t = vx - Vzx'(Vzz + P_e)^-1 (vz + p_e),
 *   K_t = Kx - Kz (Vzz + P_e)^-1 Vzx,     k_t = k1 - Kz (Vzz + P_e)^-1 (vz + p_e).
 * The few stages at each segment end whose constraint_to_go still has rows
 * (about ceil(n/m)) come from the policy sweep started at the segment end, and
 * the last segment's stages from its Riccati sweep. The result equals the
 * serial recursion's up to rounding; P_t is a difference of terms that grow
 * towards the segment end, so there the rounding error is larger than the
 * sequential sweep's (the cancellation this reconstruction trades for its
 * parallelism).
 * prob and opts as for lqr_solve with opts->prec = LQR_FP64 and
 * opts->form = LQR_FORM_CONSTRAINED, no refinement (else
 * LQR_ERR_UNSUPPORTED). Outputs (DEVICE, FP64, caller-allocated): K [T][m][n],
 * k [T][m], P [T+1][n][n] and p [T+1][n] (both NULL = not wanted).
 * Workspace: T (m (2n+1) + 3n^2 + 2n) doubles beyond the solve's (plus
 * T (2n^2 + n) when the per-stage factor does not fit in shared memory), owned
 * by the handle. Asynchronous on `stream`; device conditions through lqr_report. */
lqr_status lqr_global_policy_parallel(lqr_handle *h, const lqr_problem *prob, const lqr_opts *opts, void *K,
                                      void *k, void *P, void *p, void *stream);

/* The residual of the KKT system of Eq. 3 at (x, u, lambda), as the right-hand
 * side of the correction solve of iterative refinement (Section II-C): with
 * rx_t = Q_t x_t + S_t'u_t + q_t + lambda_t - A_t'lambda_{t+1},
 * rx_T = Q_T x_T + q_T + lambda_T, ru_t = S_t x_t + R_t u_t + r_t - B_t'lambda_{t+1},
 * rd_t = x_{t+1} - A_t x_t - B_t u_t - c_t, r0 = x_0 - x0 (Q, R read
 * symmetrised), writes q~ = -rx [T+1][n], r~ = -ru [T][m], c~ = rd [T][n] and
 * x0~ = r0 [n] (DEVICE FP64, caller-allocated). FP64 data and solution; the
 * products run in double-FP32 arithmetic (each FP64 value split into an FP32
 * pair, compensated accumulation: about 47 significant bits), the kernel of the
 * mixed-precision refinement's early passes. n, m <= 128 (else
 * LQR_ERR_UNSUPPORTED). Asynchronous on `stream`. */
lqr_status lqr_kkt_residual_vectors(lqr_handle *h, const lqr_problem *prob, const lqr_solution *sol, double *q_out,
                                    double *r_out, double *c_out, double *x0_out, void *stream);

/* The multipliers of every segment problem from the least-squares system of
 * Section II-B ("Lagrange Multipliers"), at the trajectory (x, u) (the optimum
 * lqr_solve returns, or any other): a check on the multipliers of Eq. 3 that
 * lqr_solve returns (lambda_t = -(P_t x_t + p_t)).
 * Segment j (the K-way split of lqr_partition; K = opts->num_segments, or the
 * automatic count when 0) is the problem of the constraint-explicit section:
 * its first state fixed, the dynamics, and for j < K-1 its end state fixed
 * (multiplier mu_j) with no terminal cost; the last segment has the terminal
 * cost. Its stationarity conditions in the multipliers are over-determined
 * ((n + m) L + n equations, (L + 1) n (+ n) unknowns for L stages) and are
 * solved in the least-squares sense through their block-tridiagonal normal
 * equations (block Cholesky, one CTA per segment, FP64), as the paper states.
 * At the optimum the system is consistent and the result is the exact
 * multiplier vector; elsewhere it is the least-squares one.
 * prob: FP64 device arrays as for lqr_solve; opts->prec = LQR_FP64, no
 * refinement (else LQR_ERR_UNSUPPORTED). x [T+1][n], u [T][m]: DEVICE FP64.
 * Outputs (DEVICE FP64, caller-allocated): lam [T+1][n] (lambda_t of the
 * segment holding stage t; lambda_T from the last segment), lam_end [K-1][n]
 * (segment j's own multiplier of the dynamics into its end state, which is
 * segment j+1's lambda at its first stage), mu [K-1][n]; lam_end and mu may be
 * NULL only when K = 1. Workspace: (longest segment + 2)(2n^2 + 2n) doubles per
 * segment, owned by the handle. Asynchronous on `stream`; a block that is not
 * positive definite is reported through lqr_report (LQR_ERR_NOT_PD). */
lqr_status lqr_ls_multipliers(lqr_handle *h, const lqr_problem *prob, const lqr_opts *opts, const double *x,
                              const double *u, double *lam, double *lam_end, double *mu, void *stream);

/* Step A1 alone: the per-segment parametric backward sweeps (Section II-B,
 * Eq. 9-16). Writes K summaries of LQR_SUMMARY_DOUBLES(n) doubles each to the
 * device array `summaries` (FP64). */
lqr_status lqr_segment_summaries(lqr_handle *h, const lqr_problem *prob, const lqr_opts *opts,
                                 double *summaries, void *stream);

/* The paper's own feedback policies (Section III-A), beside the serial ones
 * lqr_solve returns. The constraint-explicit segment sweeps (Section II-B)
 * give, for every stage t of segment j, u_t = Kx_t x_t + Kz_t x_term + k1_t
 * with x_term the segment's end link point (Eq. 9-16; the last segment, which
 * has a terminal cost and no end constraint, its plain Riccati policy with
 * Kz = 0); the link solve gives the link points z_j (z_0 = x0).
 *  smooth = 0: these unsmoothed segment policies. Applied with the link
 *      points they reproduce the optimal trajectory; their gains differ from
 *      the serial ones, as the segment ends are held at the link points.
 *  smooth = 1: the smoothing pass: each segment j < K-1 re-swept without end
 *      constraint from the next segment's cost to go J_{j+1}(x, z_{j+2}) (its
 *      own end pinned at its link point; the last segment's value for
 *      j = K-2): u_t = Kx_t x_t + k1_t, Kz = 0.
 * prob and opts as for lqr_solve with opts->prec = LQR_FP64 and
 * opts->form = LQR_FORM_CONSTRAINED (else LQR_ERR_UNSUPPORTED), no
 * refinement. Outputs (DEVICE, FP64, caller-allocated): Kx [T][m][n],
 * Kz [T][m][n] (NULL = not wanted), k1 [T][m], z [K+1][n] (NULL = not
 * wanted; K the segment count used, lqr_report's num_segments).
 * Asynchronous on `stream`; device conditions through lqr_report. */
lqr_status lqr_segment_policies(lqr_handle *h, const lqr_problem *prob, const lqr_opts *opts, int smooth,
                                void *Kx, void *Kz, void *k1, void *z, void *stream);

/* Synchronise `stream` and read back the scalars of the last solve on h. */
lqr_status lqr_report(lqr_handle *h, void *stream, lqr_report_t *out);

/* Human-readable name of a status code (static string). */
const char *lqr_status_string(lqr_status s);

/* Number of kernels the last lqr_solve / lqr_segment_summaries /
 * lqr_solve_batched call enqueued. */
int lqr_last_launch_count(const lqr_handle *h);

/* Phase profiling with CUDA events recorded on the solve's own stream.
 * Phases: the parametric segment sweeps (A1), the link solve (A3), the policy
 * sweeps (A4), rollout + multipliers + cost (A5/A6), refinement (A7/A8).
 * lqr_global_policy_parallel records A1, A3, the policy sweep of the segment
 * ends (policy slot) and the per-stage reconstruction kernel (rollout slot). */
#define LQR_NUM_PHASES 5
enum { LQR_PHASE_SWEEP = 0, LQR_PHASE_LINK = 1, LQR_PHASE_POLICY = 2, LQR_PHASE_ROLLOUT = 3,
       LQR_PHASE_REFINE = 4 };

/* Start (enable=1) or stop recording; enabling resets the accumulated times.
 * At most 256 solves are recorded per enable. */
lqr_status lqr_profile_enable(lqr_handle *h, int enable);

/* Sum of each phase's device time (ms) over the recorded solves, and their
 * count. Waits for the recorded events. phase_ms has LQR_NUM_PHASES entries. */
lqr_status lqr_profile_read(lqr_handle *h, double *phase_ms, int *solves);

#ifdef __cplusplus
}
#endif

#endif /* LQR_H */
