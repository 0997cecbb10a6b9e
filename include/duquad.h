/*
 * duquad.h -- C ABI of the GB300 (sm_103a) DuQuad solver.
 *
 * Solves convex QPs of the form (Necoara & Patrascu, arXiv 1504.05708,
 * Sec. 2, eq. original_primal):
 *
 *     min_{u in [lb, ub]}  F(u) = 1/2 u'Qu + q'u     s.t.  Gu + g in K,
 *
 * with K = R^p_- (inequalities, DQ_CONE_INEQ) or K = {0} (equalities,
 * DQ_CONE_EQ), by the inexact (augmented) dual first-order method DFOM
 * (Sec. 3): an outer projected dual (fast) gradient loop -- DGM / DFGM with
 * rho = 0 (Case 1), ADGM / ADFGM with rho > 0 (Case 2) -- around an inner
 * projected (fast) gradient solve of the (augmented) Lagrangian over the box
 * (Algorithm FOM, Sec. 2.1), returning the last primal iterate (eq.
 * last_primal) and/or the averaged primal iterate (eq. average_primal).
 *
 * Conventions for every entry point:
 *   - Return value is a dq_status; nothing throws or aborts across the ABI.
 *     A negative status means nothing was written to the caller's outputs;
 *     dq_last_error() then returns a message for the calling thread.
 *   - Matrices are dense row-major: Q is n x n (symmetric), G is p x n.
 *   - Host arrays are always double.  Device arrays have the element type of
 *     the problem's precision (double for DQ_FP64, float for DQ_FP32 and
 *     DQ_BF16X3) and must stay valid while a handle borrows them.
 *   - The caller owns every buffer it passes.  The library owns the handles
 *     and the device memory it allocates for them (released by *_destroy).
 *   - All GPU work is issued on the context's CUDA stream.  Entry points that
 *     return host results synchronise that stream before returning.
 */
#ifndef DUQUAD_H
#define DUQUAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Algorithm of the outer loop (Sec. 3, Algorithm DFOM and its DGM/DFGM rules).
 * DQ_ADGM / DQ_ADFGM use the augmented Lagrangian (rho > 0, Case 2). */
typedef enum { DQ_DGM = 0, DQ_DFGM = 1, DQ_ADGM = 2, DQ_ADFGM = 3 } dq_algorithm;

/* Which primal output(s) to compute and test (eq. last_primal, eq. average_primal). */
typedef enum { DQ_OUT_LAST = 1, DQ_OUT_AVERAGE = 2, DQ_OUT_BOTH = 3 } dq_output;

/* Arithmetic of the solve.  DQ_FP64: everything in double.  DQ_FP32: iterates
 * and matrix products in float, constants and final residuals in double.
 * DQ_BF16X3: shared-matrix batches only; matrix products on tensor cores with
 * bf16 hi/lo split operands (three products) and float accumulation. */
typedef enum { DQ_FP64 = 0, DQ_FP32 = 1, DQ_BF16X3 = 2 } dq_precision;

/* Inner stopping rule: DQ_INNER_GAP stops the inner loop of Algorithm FOM when
 * a certificate of eq. duquad_in (an upper bound on L_rho(x, mu) - d_rho(mu))
 * is <= eps_in; DQ_INNER_FIXED runs exactly fixed_inner iterations. */
typedef enum { DQ_INNER_GAP = 0, DQ_INNER_FIXED = 1 } dq_inner_stop;

/* Certificate of DQ_INNER_GAP.  DQ_CERT_POINT: at the iterate x^k, the
 * gradient-mapping bound <grad, x - x+> + ||L (x - x+)||^2 (1/(2 sigma) -
 * 1/(2 L)) when sigma > 0, else the Frank-Wolfe gap; it needs the gradient at
 * x^k (one more G' product when rho > 0).  DQ_CERT_STEP: when sigma > 0, the
 * bound ||L (y - x^k)||^2 (1/(2 sigma) - 1/(2 L)) of the step y^k -> x^k that
 * the iteration makes anyway (no extra product); where sigma = 0, in the
 * two-pass grid form, the tensor-core batch and FP32 thread-block solves, the
 * point certificate is used.
 * DQ_CERT_AUTO (0, the default): the step certificate in the single-pass grid
 * engine, the point certificate in the thread-block engine.  (The gradient at
 * y comes from Q y = Q x^k + beta (Q x^k - Q x^{k-1}), which carries about
 * (1 + 2 beta) times the rounding of one product; the step certificate
 * squares it, and on FP32 instances with kappa(Q) ~ 1e4 that floor stayed
 * above eps_in.) */
typedef enum { DQ_CERT_AUTO = 0, DQ_CERT_POINT = 1, DQ_CERT_STEP = 2 } dq_inner_cert;

typedef enum { DQ_CONE_INEQ = 0, DQ_CONE_EQ = 1 } dq_cone;
typedef enum { DQ_HOST = 0, DQ_DEVICE = 1 } dq_memory;

/* Engine selection (DQ_ENGINE_AUTO picks by size and batch). */
typedef enum {
  DQ_ENGINE_AUTO = 0,
  DQ_ENGINE_CTA = 1,   /* whole solve inside one thread block per instance   */
  DQ_ENGINE_GRID = 2,  /* one large instance spread over the whole GPU        */
  DQ_ENGINE_TC = 3     /* shared-matrix batch on tensor cores (DQ_BF16X3)     */
} dq_engine;

typedef enum {
  DQ_OK = 0,             /* converged (or fixed counts completed)             */
  DQ_NOT_CONVERGED = 1,  /* max_outer reached; outputs hold the last iterates */
  DQ_PENDING = 2,        /* dq_poll: the ticket is still running              */
  DQ_ERR_INVALID = -1,   /* bad argument; message in dq_last_error()          */
  DQ_ERR_NOMEM = -2,     /* device allocation failed                          */
  DQ_ERR_CUDA = -3,      /* CUDA runtime error                                */
  DQ_ERR_NONFINITE = -4, /* NaN/Inf appeared in the iterates                  */
  DQ_ERR_DIVERGED = -5,  /* infeasible: certified d_lb > max of F on the box  */
  DQ_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up                */
  DQ_ERR_REJECTED = -7   /* serving: admission refused (footprint / queue)    */
} dq_status;

typedef struct dq_context dq_context;
typedef struct dq_problem dq_problem;

/* How lambda_max(Q) and ||G||^2 = lambda_max(G'G) are found when
 * dq_problem_desc leaves them NaN (they set L_L of Sec. 3 Step 1 and L_d of
 * eq. Ld, which Algorithm FOM's step 1/L_L and both inner certificates need
 * as upper bounds of the Lipschitz constants).
 *   DQ_LIP_LANCZOS (0, default): the Lanczos method on the GPU from a
 *     pseudo-random (SplitMix64) start vector for k = ceil((ln(1.648 sqrt(n) /
 *     1e-3) / 0.1 + 1) / 2) steps (all n when n is smaller), products in the
 *     problem's precision, the tridiagonal eigenproblem in FP64, returning
 *     max(theta + 2 r, theta / 0.99) for the top Ritz value theta and its
 *     residual r.  By Kuczynski and Wozniakowski's bound for random starts
 *     (SIAM J. Matrix Anal. Appl. 13(4), 1992) theta >= 0.99 lambda_max except
 *     with probability <= 1e-3, so the value is an upper bound except with
 *     that probability, and about 1 % above lambda_max.
 *   DQ_LIP_BOUND: guaranteed bounds, min(Gershgorin row sum, ||Q||_F) and
 *     min(||G||_1 ||G||_inf, ||G||_F^2) in FP64; often far above the true
 *     values (slower convergence), for callers that need a certain bound. */
typedef enum { DQ_LIP_LANCZOS = 0, DQ_LIP_BOUND = 1 } dq_lipschitz;

/* Problem description (eq. original_primal).  batch > 1 describes `batch`
 * instances that share Q and G and differ in q (batch x n) and g (batch x p),
 * all row-major.  lmax_Q, lmin_Q, normG2: NaN means "compute"; lmax_Q and
 * normG2 are then found on the GPU as `lipschitz` says, lmin_Q is taken as 0
 * (valid for rho > 0 only).  A given value is used verbatim; lmin_Q must be a
 * lower bound of lambda_min(Q) (it sets sigma_L and L_d of eq. Ld). */
typedef struct {
  int32_t n, p;            /* variables, linear constraints (p >= 0)           */
  int32_t batch;           /* >= 1                                             */
  int32_t cone;            /* dq_cone                                          */
  int32_t prec;            /* dq_precision                                     */
  int32_t memory;          /* dq_memory of the arrays below                    */
  const void *Q, *q, *G, *g, *lb, *ub;
  double lmax_Q, lmin_Q, normG2;
  int32_t lipschitz;       /* dq_lipschitz (default DQ_LIP_LANCZOS)            */
} dq_problem_desc;

/* Solve options.  NaN / 0 fields take the documented defaults. */
typedef struct {
  int32_t alg;             /* dq_algorithm                                     */
  int32_t output;          /* dq_output (default DQ_OUT_BOTH)                  */
  int32_t inner_stop;      /* dq_inner_stop                                    */
  int32_t engine;          /* dq_engine                                        */
  double eps_out;          /* outer certificate tolerance (default 1e-3)       */
  double eps_in;           /* inner certificate tolerance (default: eq. choose_ein,
                              eps_out/4 for (A)DGM, eps_out^1.5/(8 sqrt(2 L_d))
                              for (A)DFGM with R_d = 1)                       */
  double rho;              /* NaN: 0 for DGM/DFGM, 1/||G||^2 for ADGM/ADFGM    */
  int32_t fixed_outer;     /* > 0: run exactly this many outer iterations      */
  int32_t fixed_inner;     /* inner iterations for DQ_INNER_FIXED              */
  int32_t max_outer;       /* cap in certificate mode (default 10000)          */
  int32_t max_inner;       /* cap per inner solve in gap mode (default 5000)   */
  int32_t check_every;     /* outer iterations between certificate checks (1)  */
  int32_t inner_check_every; /* inner iterations between gap checks (1)        */
  int32_t warm_start;      /* 1: start from the handle's last x and lambda     */
  int32_t kd_literal;      /* 1: K_d = R^p when lmin_Q == 0 (paper's literal)  */
  double Ld, LL, sigma;    /* NaN: derive from the problem's constants         */
  int32_t fresh_constants; /* 1: recompute lambda_max(Q) and ||G||^2 in this
                              solve instead of reusing the handle's (given
                              values in dq_problem_desc are always kept)       */
  int32_t inner_cert;      /* dq_inner_cert (default DQ_CERT_AUTO)             */
  int32_t stop_fstar;      /* 1: outer stop on |F(u) - f_star| <= eps_out and
                              dist_K(Gu+g) <= eps_out instead of the certificate
                              (the paper's experiments, Sec. 6, for a known F*;
                              thread-block and grid engines)                   */
  double f_star;           /* F* for stop_fstar                                */
} dq_solve_opts;

/* Result of one solve (one instance). */
typedef struct {
  int32_t status;          /* dq_status of this instance                       */
  int32_t outer_iters;
  int64_t inner_iters;     /* all inner iterations, extra last-iterate solves included */
  int32_t converged_last, converged_avg;
  double f_last, infeas_last;  /* FP64 F(u) and dist_K(Gu+g) of the outputs  */
  double f_avg, infeas_avg;
  double d_lb;             /* FP64 lower bound on F* from the certificate      */
  double Ld, LL, sigma, rho, alpha; /* constants used (alpha = 1/(2 L_d))       */
} dq_result;

/* Output buffers.  NULL pointers are skipped.  memory = DQ_HOST: double
 * arrays; DQ_DEVICE: device arrays of the precision's element type.  For a
 * batch, arrays hold batch x n (x_last, x_avg) or batch x p (lambda) values. */
typedef struct {
  void *x_last, *x_avg, *lambda;
  int32_t memory;
} dq_outputs;

/* Create a context bound to CUDA device `device` issuing work on the CUDA
 * stream `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * Errors: DQ_ERR_INVALID (bad device), DQ_ERR_CUDA. */
dq_status dq_context_create(int device, void *cuda_stream, dq_context **out);
/* Stops serving and releases the context; when problem handles of the
 * context still exist the release happens when the last one is destroyed
 * (the context must not be used after this call either way). */
dq_status dq_context_destroy(dq_context *ctx);

/* Create a problem handle.  memory = DQ_HOST: the arrays are copied to the
 * device (converted to the precision's element type).  memory = DQ_DEVICE:
 * Q and G are borrowed (the caller keeps them alive and unchanged until
 * dq_problem_destroy); vectors are copied.  The library also keeps a
 * transposed copy of G and FP64 constants.  Validation: n >= 1, p >= 0,
 * batch >= 1, and on the device for host and device data alike: finite
 * values, lb <= ub, and Q symmetric (|Q_ij - Q_ji| <= tol sqrt(|Q_ii Q_jj|),
 * tol = 1e-10 for FP64, 1e-6 for FP32 and DQ_BF16X3); otherwise DQ_ERR_INVALID
 * with a message.  Errors: DQ_ERR_NOMEM, DQ_ERR_CUDA. */
dq_status dq_problem_create(dq_context *ctx, const dq_problem_desc *desc, dq_problem **out);

/* Sparse problems (CSR).  When Q and G are sparse, every step of the method
 * is still a matrix-vector product and costs O(nnz) instead of O(n^2)
 * (Sec. 5, the remark on sparse QPs).  Q is given as the full symmetric n x n
 * matrix (both triangles), G as p x n, each in CSR: row offsets rowptr[rows+1]
 * (rowptr[0] = 0, rowptr[rows] = nnz), column indices strictly increasing
 * within a row, values; offsets and indices are int32 (nnz < 2^31).
 * memory = DQ_HOST: values and vectors are doubles; DQ_DEVICE: every array is
 * a device array (values and vectors of the precision's element type), copied
 * to the host once for validation and for building G'.  prec: DQ_FP64 or
 * DQ_FP32; one instance (batch 1), solved by the grid engine (DQ_ENGINE_AUTO
 * or DQ_ENGINE_GRID; other engines return DQ_ERR_INVALID).  The library
 * copies everything (nothing is borrowed).  Validation: consistent offsets,
 * columns in range and increasing, finite values, lb <= ub, Q symmetric in
 * structure and values (|Q_ij - Q_ji| <= tol sqrt(|Q_ii Q_jj|), tol as for
 * dense problems); else DQ_ERR_INVALID.  G' is built on the host by a stable
 * counting sort, so every product sums in a fixed order.  lipschitz:
 * DQ_LIP_LANCZOS (Lanczos on the CSR products) or DQ_LIP_BOUND (the bounds of
 * dq_lipschitz, computed from the CSR arrays in FP64 on the host). */
typedef struct {
  int32_t n, p;
  int32_t cone;            /* dq_cone                                          */
  int32_t prec;            /* DQ_FP64 or DQ_FP32                               */
  int32_t memory;          /* dq_memory of every array below                   */
  int32_t nnz_Q, nnz_G;
  const int32_t *Q_rowptr, *Q_col;
  const void *Q_val;
  const int32_t *G_rowptr, *G_col;
  const void *G_val;
  const void *q, *g, *lb, *ub;
  double lmax_Q, lmin_Q, normG2; /* as in dq_problem_desc                      */
  int32_t lipschitz;       /* dq_lipschitz                                     */
} dq_sparse_desc;

dq_status dq_problem_create_sparse(dq_context *ctx, const dq_sparse_desc *desc, dq_problem **out);

/* Replace q and/or g (NULL keeps the current one) of all `batch` instances;
 * arrays as in dq_problem_desc with the given memory kind. */
dq_status dq_problem_set_vectors(dq_problem *prob, const void *q, const void *g, int32_t memory);

/* FP64 constants held by the handle (lambda_max(Q), lambda_min bound, ||G||^2). */
dq_status dq_problem_constants(dq_problem *prob, double *lmax_Q, double *lmin_Q, double *normG2);

dq_status dq_problem_destroy(dq_problem *prob);

/* Solve the problem (all instances of a batch) with Algorithm DFOM (Sec. 3).
 * results: one dq_result per instance (batch entries).  Outputs are written
 * for status >= 0.  Returns the worst instance status (error < not converged
 * < ok).  Synchronises the context's stream. */
dq_status dq_solve(dq_problem *prob, const dq_solve_opts *opts, const dq_outputs *out,
                   dq_result *results);

/* Solve `count` independent problems of any sizes in one persistent launch
 * (one CTA-resident solve per instance, a device work queue, longest
 * instances first), issued as a captured CUDA graph that is replayed while
 * the inputs (handles, options, warm-start flags) stay the same.  The launch
 * shape is the one dq_autotune chose for this size mix, else 256 threads and
 * the device's shared-memory maximum.  opts, out are arrays of `count`
 * entries; results holds one entry per instance (batches expand). */
dq_status dq_solve_many(dq_problem *const *probs, int32_t count, const dq_solve_opts *opts,
                        const dq_outputs *out, dq_result *results);

/* Solve one FP64 or FP32 instance without allocating memory.  The paper has
 * no counterpart: this is for callers that cannot allocate device memory
 * while running -- a real-time loop (e.g. model-predictive control solving
 * one QP per sampling period) whose timing must not depend on an allocator,
 * or a process whose memory pool has already reserved the GPU, so that a
 * further cudaMalloc fails.  It runs the same whole-solve-per-thread-block
 * kernel as dq_solve's CTA engine on the caller's device arrays and keeps
 * its scratch (instance descriptor, work-queue counter, result, constants and
 * a transposed copy of G) in one fixed 8 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 * desc: memory must be DQ_DEVICE, batch 1, prec DQ_FP64 or DQ_FP32 (arrays of
 * double or float).  out (nullable): DQ_DEVICE arrays of the same type.
 * Limits: n * p elements of G must fit the scratch (8 MiB minus 4 KiB:
 * n * p <= 1048064 for FP64, 2096128 for FP32) and the instance's vectors one
 * thread block's shared memory; otherwise DQ_ERR_INVALID with a message.
 * No warm start.
 * Set-up: the first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress, with that device current).  Under CUDA's default
 * lazy module loading that first call (or the first launch) is also when the
 * library's kernels and the 8 MiB array are placed on the device, so it can
 * fail with an out-of-memory error if the caller's pool has already reserved
 * the GPU: make one call per device before any pool reserves device memory
 * (or run with CUDA_MODULE_LOADING=EAGER, which places them when the library
 * loads).  After that first call, calls allocate nothing.
 * Every call copies its descriptor from host memory and synchronises
 * `stream` before returning.  Every call shares the one
 * scratch array (which keeps the last call's contents), so calls whose GPU
 * work overlaps (other streams or threads on the same device) race:
 * serialise them.  stream: cudaStream_t (NULL = legacy default). */
dq_status dq_solve_noalloc(int device, const dq_problem_desc *desc, const dq_solve_opts *opts,
                           const dq_outputs *out, dq_result *result, void *cuda_stream);

/* Autotune the launch shape dq_solve_many uses for this mix of problems:
 * times short fixed-count solves (2 outer x 25 inner iterations) of up to
 * `sample` instances spread over the mix under each candidate block size
 * (128, 256, 512 threads) and shared-memory cap (48 KB, 112 KB, the device
 * maximum) with CUDA events, keeps the fastest for the context under a
 * signature of the size histogram, and persists it (file named by
 * DQ_AUTOTUNE_CACHE, else autotune.txt next to the library).  The sampled
 * handles' warm-start state is overwritten.  threads_out / smem_cap_out
 * (nullable) receive the choice (smem cap 0 = device maximum). */
dq_status dq_autotune(dq_problem *const *probs, int32_t count, const dq_solve_opts *opts, int32_t sample,
                      int32_t *threads_out, int32_t *smem_cap_out);

/* ---- serving (continuous batching) ----------------------------------------
 * dq_serve_start launches the context's persistent request loop with `slots`
 * device request slots and a device-memory budget of `hbm_budget_bytes` for
 * admitted requests.  dq_submit enqueues a solve of `prob` (which must stay
 * alive until the ticket is polled) with new q/g vectors (host double, NULL
 * keeps the handle's) and warm start from the handle's last lambda; it
 * returns DQ_ERR_REJECTED when the request can never fit the budget or the
 * loop's per-request limits (FP32 instances with n <= 512, p <= 1024).
 * dq_poll returns DQ_PENDING until the ticket completes, then the result and
 * the outputs (host double).  dq_serve_stop drains and stops the loop. */
dq_status dq_serve_start(dq_context *ctx, int32_t slots, int64_t hbm_budget_bytes);
dq_status dq_submit(dq_context *ctx, dq_problem *prob, const dq_solve_opts *opts,
                    const double *q, const double *g, uint64_t *ticket);
dq_status dq_poll(dq_context *ctx, uint64_t ticket, double *x_last, double *x_avg,
                  double *lambda, dq_result *result);
dq_status dq_serve_stop(dq_context *ctx);

/* ---- measurement ----------------------------------------------------------
 * Counters of the kernels a context launched.  With profiling enabled the
 * grid engine brackets every inner-iteration GEMV launch (the streaming
 * matrix pass that dominates the method, Sec. 5 "main computational
 * bottleneck") with CUDA events on the context's stream; launches that
 * returned early because the inner loop had already stopped are not counted.
 * gemv_bytes counts each matrix element once plus the vectors read and
 * written once (the algorithmic bytes of those launches).  The single-pass
 * form also times its per-iteration partial-sum reduction (reduce_*). */
typedef struct {
  int64_t launches;        /* all kernels launched by this context            */
  int64_t gemv_launches;   /* timed inner-iteration GEMV launches             */
  double gemv_ms;          /* their summed device time                        */
  double gemv_bytes;       /* their algorithmic bytes                         */
  int64_t reduce_launches; /* timed partial-sum reductions (single-pass form) */
  double reduce_ms;        /* their summed device time                        */
} dq_stats;

/* enable != 0 turns per-launch event timing of the GEMV on. */
dq_status dq_context_profile(dq_context *ctx, int32_t enable);
/* Copy the counters; reset != 0 zeroes them afterwards. */
dq_status dq_context_stats(dq_context *ctx, dq_stats *out, int32_t reset);

/* ---- theory mode ----------------------------------------------------------
 * Iteration counts that the paper's analysis prescribes for a target
 * accuracy eps (host arithmetic only; needs no GPU).  With R_d an estimate of
 * the distance from lambda^0 to the optimal multipliers and D_U the box
 * diameter ||ub - lb||_2:
 *   rho     given, or (NaN) rho* = 8 R_d^2 / eps for ADGM/ADFGM (the optimal
 *           smoothing of Sec. 5) and 0 for DGM/DFGM;
 *   L_L = lmax_Q + rho normG2,  sigma_L = lmin_Q,
 *   L_d = normG2 / (lmin_Q + rho normG2)                         (eq. Ld);
 *   eps_in, k_out                                        (eq. choose_ein):
 *     DGM/ADGM   eps / 4,                        8 L_d R_d^2 / eps
 *     DFGM/ADFGM eps^{3/2} / (8 R_d sqrt(2 L_d)),  sqrt(8 L_d R_d^2 / eps);
 *   k_in, Algorithm FOM's count for eps_in (Sec. 5):
 *     sigma_L = 0: sqrt(2 L_L D_U^2 / eps_in),
 *     sigma_L > 0: sqrt(L_L / sigma_L) log(L_L D_U^2 / eps_in) + 1;
 * k_out and k_in are rounded up (at least 1).  A solve with inner_stop =
 * DQ_INNER_FIXED, fixed_inner = k_in, fixed_outer = k_out, rho = rho and
 * eps_in = eps_in runs the method exactly as analysed.  DQ_ERR_INVALID: eps,
 * R_d or D_U not positive and finite, lmax_Q or normG2 not finite, lmin_Q
 * negative, rho negative, or L_d undefined (DGM/DFGM with lmin_Q = 0). */
typedef struct {
  int32_t alg;                    /* dq_algorithm                              */
  double eps;                     /* target accuracy (> 0)                     */
  double Rd;                      /* estimate of R_d (> 0)                     */
  double D_U;                     /* box diameter (> 0)                        */
  double lmax_Q, lmin_Q, normG2;  /* spectrum constants                        */
  double rho;                     /* NaN: the default above                    */
} dq_theory_in;

typedef struct {
  double rho, LL, sigma, Ld;      /* the constants the counts use              */
  double eps_in;                  /* inner accuracy (eq. choose_ein)           */
  int64_t k_out, k_in, k_total;   /* outer, inner per outer, their product     */
} dq_theory_out;

dq_status dq_theory(const dq_theory_in *in, dq_theory_out *out);

/* Theory-mode solve: the method run with the counts of the analysis (Sec. 5,
 * eq. choose_ein) for one instance (batch 1), with an estimate of R_d where
 * the caller has none (the paper leaves the R_d search open).
 *   R_d: Rd > 0 is used as given.  Rd NaN: a certified solve of the same
 *     instance (algorithm alg, eps_out = eps, default eps_in and rho, from
 *     lambda^0 = 0) gives multipliers lambda, and R_d = safety *
 *     max(||lambda||_2, eps) (safety NaN: 2).  A certified lambda can lie short
 *     of the optimal multipliers, which the safety factor covers.
 *   D_U = ||ub - lb||_2 of the problem; lmax_Q and normG2 as
 *     dq_problem_constants gives them; lmin_Q as given at creation (NaN: 0,
 *     which only ADGM/ADFGM accept).
 *   rho: NaN takes rho* = 8 R_d^2 / eps for ADGM/ADFGM (0 for DGM/DFGM).
 * Then a solve with inner_stop = DQ_INNER_FIXED, fixed_outer = k_out,
 * fixed_inner = k_in, eps_in, rho, L_L, sigma_L and L_d from dq_theory, from
 * lambda^0 = 0 (no warm start), on `engine` (DQ_ENGINE_AUTO picks as dq_solve),
 * outputs as in dq_solve.  max_total (0: 1e8) bounds k_out * k_in: larger
 * counts return DQ_ERR_INVALID before any fixed-count work.  counts and Rd_used
 * (either may be NULL) receive dq_theory's output and the R_d taken. */
typedef struct {
  int32_t alg;          /* dq_algorithm                                      */
  double eps;           /* target accuracy (> 0)                             */
  double Rd;            /* > 0, or NaN: estimate                             */
  double safety;        /* factor on the estimate (NaN: 2)                   */
  double rho;           /* NaN: rho* (ADGM/ADFGM) or 0                       */
  int64_t max_total;    /* cap on k_out * k_in (0: 1e8)                      */
  int32_t engine;       /* dq_engine                                         */
} dq_theory_solve_opts;

dq_status dq_solve_theory(dq_problem *P, const dq_theory_solve_opts *opts, const dq_outputs *out,
                          dq_result *result, dq_theory_out *counts, double *Rd_used);

/* Message of the last failing call on this thread ("" if none). */
const char *dq_last_error(void);

/* Library version string. */
const char *dq_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DUQUAD_H */
