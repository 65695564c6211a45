/*
 * spmesl.h - C ABI of libspmesl: sparse precision matrix estimation via the
 * scaled lasso (SPMESL), solved by GPU-parallel coordinate descent on one
 * NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are dense and row-major.  "p x p" buffers are p*p elements with
 *    leading dimension p unless a leading-dimension argument says otherwise.
 *  - Pointers are DEVICE pointers unless the argument name ends in `_host`.
 *    The caller allocates and owns every buffer it passes; the library never
 *    frees or keeps a caller pointer after the call's stream work completes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued on it; calls return without synchronising unless
 *    the description says otherwise.
 *  - Errors come back as spmesl_status codes; nothing throws across the ABI.
 *    Invalid arguments are rejected on the host before any work is enqueued.
 *    Conditions found on the device (non-finite input, sigma floor, iteration
 *    caps, a bounded wait that ran out) are written to a status word in the
 *    workspace and reported by spmesl_fit_result (or by spmesl_fit itself
 *    when `stats` is non-NULL).
 *  - Precision: SPMESL_FP64 takes FP64 data and works in FP64 throughout.
 *    SPMESL_FP32 and SPMESL_MIXED take FP32 data, run the coordinate-descent
 *    sweeps in FP32, and keep sigma, the convergence decisions on sigma and
 *    the final Theta in FP64.  SPMESL_MIXED builds the Gram matrix with
 *    split-BF16 tensor-core products and FP32 accumulation.
 *
 * Index convention for the result: Theta[j*p + k] = omega_jk.  Before
 * symmetrisation column k of Omega comes from regression k (Eq. (4)):
 * omega_kk = 1/sigma_k^2, omega_jk = -b_jk / sigma_k^2, where b_jk is the
 * coefficient of x_j in the regression of x_k on the other columns.
 */
#ifndef SPMESL_H
#define SPMESL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPMESL_OK = 0,
    SPMESL_NOT_CONVERGED = 1,   /* an iteration cap was hit; outputs hold the last iterate */
    SPMESL_EINVAL = -1,         /* bad argument (sizes, pointers, tolerances, workspace) */
    SPMESL_ENOMEM = -2,         /* workspace too small / allocation or budget refused */
    SPMESL_ENONFINITE = -3,     /* NaN/Inf in the input, or S_jj <= 0 */
    SPMESL_EDEGENERATE = -4,    /* some sigma_j^2 reached the floor 1e-12 * S_jj (perfect fit) */
    SPMESL_ETIMEOUT = -5,       /* a bounded device-side wait ran out */
    SPMESL_ECUDA = -6,          /* a CUDA runtime call failed */
    SPMESL_EBUSY = -7,          /* request still running / no free slot */
    SPMESL_ENOTFOUND = -8       /* unknown ticket */
} spmesl_status;

typedef enum {
    SPMESL_FP64 = 0,
    SPMESL_FP32 = 1,
    SPMESL_MIXED = 2
} spmesl_precision;

/* Penalty level lambda0 (Section 2.1 and Section 2.3, Eqs. (10)-(11)). */
typedef enum {
    SPMESL_LAMBDA_GIVEN = 0,    /* use the lambda0 argument as is */
    SPMESL_LAMBDA_UNIV = 1,     /* sqrt(2 log(p) / n)                         (Section 2.1) */
    SPMESL_LAMBDA_UNIV_PM1 = 2, /* sqrt(2 log(p-1) / n)                       (Section 4.1) */
    SPMESL_LAMBDA_UB = 3,       /* sqrt(4 log(p) / n)                         (Eq. (10), A = 1) */
    SPMESL_LAMBDA_PB = 4        /* sqrt(2) L_n(k/p), k = L_1^4(k/p)+2L_1^2(k/p) (Eq. (11)) */
} spmesl_lambda_rule;

/* Inner stopping rule of the lasso subproblems. */
typedef enum {
    SPMESL_INNER_JOINT = 0,     /* ||B_next - B_cur||_inf over all active columns (Algorithm 3) */
    SPMESL_INNER_COLUMN = 1     /* per column ||b_next - b_cur||_inf (Algorithms 1-2) */
} spmesl_inner_rule;

/* How the per-column rule keeps g_j = S_.j - S b_j during a sweep.  Both solve
 * Algorithm 1's column problems to the same tolerance.  The lazy solver also
 * sweeps each column's support alone before every certifying sweep, so its
 * iterates take another path to the same solution. */
typedef enum {
    SPMESL_GRADIENT_AUTO = 0,   /* lazy, and the block solver for heavy columns: those whose
                                   heat exceeds opts.heavy_heat in fits of at least
                                   opts.heavy_min_p columns (from the start, beside the lazy
                                   launch) and those whose support outgrows the lazy solver's
                                   32-coordinate active-set phase (after it, continuing from
                                   the lazy solver's iterate) */
    SPMESL_GRADIENT_EAGER = 1,  /* g_j and b_j stored in shared memory, rank-1 update of the
                                   whole g_j after every coordinate move */
    SPMESL_GRADIENT_LAZY = 2    /* only the support of b_j stored; each 128-coordinate slice of
                                   g_j formed from S rows when the sweep reaches it; the block
                                   solver only for supports beyond the lazy list (256) */
} spmesl_gradient;

typedef struct {
    int32_t precision;          /* spmesl_precision */
    int32_t standardize;        /* 1 (default): fit on S^C = C S C, C = diag(S_jj^-1/2), and
                                   return C Omega^C C (Proposition 1); 0: fit on S itself with
                                   update b_kj = Soft(c, lambda0 sigma_j) / S_kk */
    int32_t center;             /* spmesl_gram / spmesl_solve: subtract column means (Section 2.2) */
    int32_t lambda_rule;        /* spmesl_lambda_rule */
    int32_t inner_rule;         /* spmesl_inner_rule (default SPMESL_INNER_COLUMN) */
    int32_t warps_per_block;    /* 0 = chosen from p and shared-memory capacity */
    int32_t record_phase_times; /* 1: record CUDA events around the fit's phases on `stream`;
                                   spmesl_fit_result then fills ms_cd and ms_theta */
    int32_t use_graph;          /* spmesl_batch_run: capture the batch's launches once into a
                                   CUDA graph and replay it on later runs */
    int32_t gradient;           /* spmesl_gradient: how a column keeps its gradient (column rule) */
    int32_t diagnostics;        /* 1: after the fit, one more launch checks every column's
                                   (b_j, sigma_j) in FP64 on the device and fills kkt_viol,
                                   dual_gap and err_est of spmesl_stats (0: not computed) */
    int32_t heavy_heat;         /* SPMESL_GRADIENT_AUTO on a standardised fit: a column whose
                                   heat (off-diagonal |S^C_jk| above lambda0) exceeds this goes to
                                   the block solver from the start; 0 = 32, at most 62 */
    int32_t heavy_min_p;        /* ... only in fits with p >= heavy_min_p (0 = 4096; < 0: never).
                                   In any fit a column whose support outgrows the lazy solver's
                                   32-coordinate active-set phase is handed over to it */
    int32_t count_rows;         /* measurement: 1 fills spmesl_stats.rows_moved */
    int32_t handover;           /* SPMESL_GRADIENT_AUTO: the lazy solver hands a column to the
                                   block solver when its support exceeds this at the start of an
                                   active-set phase (0 = 32, the phase's size; at most 256, above
                                   32 such columns sweep without the phase) */
    int32_t reserved[2];
} spmesl_opts;

typedef struct {
    int32_t status;             /* spmesl_status of the fit */
    int32_t outer_iters;        /* max over columns of sigma iterations (joint rule: global count) */
    int64_t inner_sweeps;       /* sum over columns of full sweeps, the block solver's certifying
                                   passes over every coordinate included (joint rule: global count) */
    int64_t moves;              /* coordinate updates that changed some b_kj (one S-row axpy each) */
    int64_t nnz_B;              /* nonzero off-diagonal b_jk at exit */
    int32_t n_not_converged;    /* columns that hit an iteration cap */
    int32_t n_degenerate;       /* columns whose sigma^2 hit the floor */
    double max_db;              /* largest |delta b| of the last sweep (joint rule) */
    double lambda0;             /* penalty level actually used */
    float ms_gram;              /* device time of the Gram step (spmesl_solve only), ms */
    float ms_fit;               /* device time of the whole fit, ms */
    float ms_cd;                /* coordinate-descent kernel alone (record_phase_times), ms */
    float ms_theta;             /* Theta assembly kernel alone (record_phase_times), ms */
    int32_t max_col_sweeps;     /* largest number of sweeps any one column ran */
    int32_t max_col_outer;      /* largest number of sigma iterations any one column ran */
    float ms_queue;             /* serving: submit -> admitted into a batch, ms (host clock) */
    float ms_total;             /* serving: submit -> completion seen by the context, ms */
    int32_t batch_size;         /* serving: requests in the batch this one ran in */
    int32_t reserved32;
    int64_t active_sweeps;      /* sum over columns of sweeps over the support only (lazy solver) */
    int64_t active_moves;       /* coordinate updates in those sweeps (no S-row read: the support's
                                   block of S is held in shared memory) */
    int32_t block_columns;      /* columns solved by the block solver (heavy columns and those the
                                   lazy solver handed over; SPMESL_GRADIENT_AUTO / LAZY) */
    int32_t diagnostics;        /* 1 when the three fields below were computed (opts.diagnostics) */
    double kkt_viol;            /* largest violation of the lasso subgradient conditions of any
                                   column, relative to its penalty lambda0 sigma_j, in FP64 on the
                                   working matrix (Section 2.1; Algorithm 1's fixed point) */
    double dual_gap;            /* largest relative duality gap (P - D) / P of any column's lasso
                                   subproblem at its final sigma, in FP64 on the working matrix */
    double err_est;             /* estimated max |dTheta| / max |Theta| of the result against the
                                   exact estimator: the first-order effect of the measured
                                   gradient residuals and sigma fixed-point residuals, plus the
                                   rounding bound of the working matrix (see spmesl_opts) */
    int64_t rows_moved;         /* opts.count_rows: for each full-sweep index m (the m-th full
                                   sweep of a column, m < 64), the number of distinct coordinates
                                   k that moved in sweep m of any column, summed over m: the rows
                                   of S a row-synchronous schedule reads for its rank-1 updates */
} spmesl_stats;

/* A helper (no passage of the paper): fill `opts` with the defaults: FP32,
 * standardize = 1, center = 0,
 * lambda_rule = GIVEN, inner_rule = COLUMN, warps_per_block = 0. */
void spmesl_default_opts(spmesl_opts* opts);

/* A helper (no passage of the paper): static text for a status code. */
const char* spmesl_status_string(int status);

/* A helper (no passage of the paper): library ABI version
 * (major * 10000 + minor * 100 + patch). */
int spmesl_version(void);

/* Penalty level for a rule (host computation; Section 2.1, Eqs. (10)-(11),
 * Section 4.1).  Returns NaN for SPMESL_LAMBDA_GIVEN or invalid n, p. */
double spmesl_lambda(int rule, int n, int p);

/*
 * Gram matrix S = X'X / n (Section 2.2), optionally of the column-centred X.
 *   X          n x p, leading dimension ldx >= p; FP64 for SPMESL_FP64,
 *              FP32 otherwise.  Read only.
 *   S          p x p output, leading dimension lds >= p, same element type as
 *              X.  Both triangles are written.
 *   workspace  device scratch of at least spmesl_gram_workspace_bytes(n, p,
 *              precision) bytes (may be NULL when that is 0).
 * SPMESL_FP64 and SPMESL_FP32 accumulate in the input precision on the CUDA
 * cores; SPMESL_MIXED splits X = hi + lo into two BF16 parts and forms
 * hi'hi + hi'lo + lo'hi on the tensor cores (tcgen05, TMEM accumulators)
 * with FP32 accumulation.
 * Errors: EINVAL for n < 1, p < 1, ldx < p, lds < p, NULL pointers, a short
 * workspace; ECUDA if a launch fails.
 */
size_t spmesl_gram_workspace_bytes(int n, int p, int precision);
spmesl_status spmesl_gram(const void* X, int n, int p, int ldx, int precision, int center,
                          void* S, int lds, void* workspace, size_t ws_bytes, void* stream);

/*
 * One SPMESL fit on a covariance matrix (Algorithm 2 / Algorithm 3):
 *   1. S^C = C S C (standardize = 1, Section 2.2 and Proposition 1);
 *   2. for every column j, the scaled lasso of Eq. (5) by cyclic ascending
 *      coordinate descent with warm start (Algorithm 1): all columns run in
 *      parallel, each keeping its gradient g_j = S_.j - S b_j on chip and
 *      applying the rank-1 update g_j -= S_.k delta_kj after every coordinate
 *      that moves (Proposition 2 written on S); sigma_j^2 =
 *      S_jj - 2 b_j'S_.j + b_j'S b_j in FP64 (Eq. (14)); columns whose sigma
 *      changed by less than tol are retired (Section 3.3).
 *      With the per-column rule and the lazy gradient, each column sweeps
 *      its current support (up to 32 coefficients) to convergence before
 *      every certifying sweep. That sweep holds the support and updates the
 *      other coordinates; the lasso at one sigma has converged when both moved
 *      nothing by tol. Heavy columns (up to 64 support coefficients in the
 *      phase) let the coordinates such a sweep would move join the next
 *      phase together instead of entering one at a time; with none the lasso
 *      at that sigma has converged. The per-column solvers take a safeguarded secant step
 *      on the fixed point sigma = F(sigma) of Eq. (14) after its first step.
 *      The stop tests and the returned (b, sigma) pair are those of
 *      Algorithm 1, so the fit ends at the same fixed point within tol;
 *   3. Omega_1 = -B D (Eq. (4)), min-magnitude symmetrisation (Eq. (9)), and
 *      Omega^o = C Omega^C C.
 *   S          p x p covariance (FP64 for SPMESL_FP64, FP32 otherwise), read only.
 *   n          sample size; used only by lambda rules other than GIVEN (may be 0
 *              with SPMESL_LAMBDA_GIVEN).
 *   lambda0    penalty level (> 0) when opts->lambda_rule is GIVEN.
 *   tol        the tolerance delta of both stopping tests (> 0).
 *   maxit      cap on inner sweeps per lasso subproblem and, separately, on
 *              sigma iterations (>= 1).
 *   opts       may be NULL for the defaults; opts->precision selects the path.
 *   Theta      p x p FP64 output (row-major, symmetric).
 *   sigma      p FP64 output, sigma_j in the original scale.
 *   stats      host pointer or NULL.  Non-NULL makes the call synchronise on
 *              `stream` and fill it; the return value is then the fit's status.
 *   workspace  device scratch of at least spmesl_fit_workspace_bytes(p,
 *              precision) bytes, 256-byte aligned.  It holds the standardised
 *              S, the coefficients B and the fit's control block, and must not
 *              be reused until the fit has completed on `stream`.
 * Returns OK once the work is enqueued (stats == NULL) or the fit's status.
 * Errors: EINVAL (p < 2, lambda0 <= 0, tol <= 0, maxit < 1, NULL pointers,
 * misaligned or short workspace, p above spmesl_max_p(precision)); ECUDA.
 * Device-detected: ENONFINITE (non-finite S or S_jj <= 0; Theta untouched),
 * EDEGENERATE, NOT_CONVERGED, ETIMEOUT.
 */
size_t spmesl_fit_workspace_bytes(int p, int precision);
int spmesl_max_p(int precision);
spmesl_status spmesl_fit(const void* S, int n, int p, double lambda0, double tol, int maxit,
                         const spmesl_opts* opts, double* Theta, double* sigma,
                         spmesl_stats* stats, void* workspace, size_t ws_bytes, void* stream);

/*
 * spmesl_fit without any device allocation and without a caller workspace.
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc or give the library scratch memory (for example a plugin whose
 * host application owns all device memory, or real-time code that forbids
 * allocation after start-up).
 *   Arguments, outputs and device-side status are those of spmesl_fit, except
 *   that there is no workspace: the fit's scratch is one 64 MiB __device__
 *   array inside the library.  record_phase_times is ignored.
 *   The first call on each device (with that device current) looks up the
 *   array's device address; that lookup loads the library's module, which
 *   commits the 64 MiB on the device, and the device holds it until the
 *   process exits.  Make that first call at start-up, and before any stream
 *   capture.  If the device has no room for the array, SPMESL_ENOMEM.
 *   Size limit: the fit's scratch must fit in 64 MiB, i.e. p <= 2351 for
 *   SPMESL_FP32 / SPMESL_MIXED and p <= 1664 for SPMESL_FP64; larger p returns
 *   SPMESL_ENOMEM before any work is enqueued.
 *   All calls share the array and it keeps the last call's contents (each fit
 *   clears what must start at zero).  Calls whose work overlaps on the GPU
 *   race on the array: issue them on one stream or order them.
 *   stats non-NULL synchronises `stream` and fills everything except the
 *   timing fields (lambda0 included).  No cudaMalloc, cudaFree or allocating
 *   library routine is called.
 */
spmesl_status spmesl_fit_noalloc(const void* S, int n, int p, double lambda0, double tol,
                                 int maxit, const spmesl_opts* opts, double* Theta, double* sigma,
                                 spmesl_stats* stats, void* stream);

/* The fit's outcome (Algorithm 2): synchronise `stream` and read the status
 * and counters of the last fit that
 * ran in `workspace` (p and precision as given to spmesl_fit).  Returns the
 * fit's status. */
spmesl_status spmesl_fit_result(const void* workspace, int p, int precision,
                                spmesl_stats* stats, void* stream);

/*
 * One SPMESL fit from the data in the residual form, without the Gram matrix
 * (Algorithm 3's residual matrix E = X - X B and the rank-1 update of
 * Proposition 2, run per column with the cyclic order and the per-column
 * stopping rule of Algorithm 1).  Column j keeps its residual
 * e_j = x_j - X b_j; the gradient of coordinate k is x_k' e_j / n and a move
 * updates e_j -= x_k delta.  sigma_j^2 = ||e_j||^2 / n (Eq. (14)) in FP64 from
 * a residual recomputed from the data.  The estimate is the one spmesl_gram +
 * spmesl_fit computes; the iterates are plain cyclic sweeps (the covariance
 * form also sweeps the current support alone before each full sweep).
 * Memory: the scaled data twice (n x p and p x n) and the p x p coefficients,
 * against S, the standardised S and two p x p matrices in the covariance form.
 *   X          n x p data, row-major with leading dimension ldx >= p, device,
 *              FP64 for SPMESL_FP64, FP32 otherwise (SPMESL_MIXED runs as
 *              SPMESL_FP32: there is no Gram to build).  Read only.
 *   n          sample size, 1 <= n <= 16384.
 *   lambda0, tol, maxit, Theta, sigma, stats: as spmesl_fit.
 *   opts       precision, standardize (columns scaled to unit variance and
 *              the result mapped back, Proposition 1), center (subtract
 *              column means, Section 2.2), lambda_rule, warps_per_block,
 *              record_phase_times; inner_rule must be SPMESL_INNER_COLUMN.
 *   workspace  spmesl_fit_residual_workspace_bytes(n, p, precision) bytes,
 *              256-byte aligned, owned by the caller; must not be reused
 *              until the fit has completed on `stream`.  spmesl_fit_result
 *              reads its status; spmesl_fit_coefficients does not apply.
 * A column whose support outgrows 256 coefficients stops and reports
 * NOT_CONVERGED with its last iterate.
 * Errors: EINVAL (NULL pointers, p < 2, n outside [1, 16384], ldx < p,
 * lambda0 <= 0, tol <= 0, maxit < 1, inner_rule JOINT, short or misaligned
 * workspace, sizes whose per-warp shared memory exceeds the block limit);
 * ECUDA.  Device-detected: ENONFINITE (non-finite X or a column of zero
 * variance; Theta untouched), EDEGENERATE, NOT_CONVERGED.
 */
size_t spmesl_fit_residual_workspace_bytes(int n, int p, int precision);
spmesl_status spmesl_fit_residual(const void* X, int n, int p, int ldx, double lambda0,
                                  double tol, int maxit, const spmesl_opts* opts, double* Theta,
                                  double* sigma, spmesl_stats* stats, void* workspace,
                                  size_t ws_bytes, void* stream);

/* The regression coefficients of Eq. (5) (b_j of each column problem,
 * Algorithm 2): copy the coefficients of the last fit in `workspace` to B (p x p FP64
 * device buffer, original scale, B[j*p + k] = b_jk, zero diagonal). */
spmesl_status spmesl_fit_coefficients(const void* workspace, int p, int precision, double* B,
                                      void* stream);

/*
 * Optimality check of an estimate (Section 2.1: the scaled-lasso optimality
 * conditions of each column problem of Eq. (5); Eq. (14)): for every column k
 * of B, with lambda = lambda0 sigma_k on the working matrix (S^C when
 * opts->standardize, else S) and g = S_.k - S b_k formed in FP64 on the device,
 *   kkt_viol  = max over k and j != k of |g_j - lambda sign(b_jk)| (b_jk != 0)
 *               or (|g_j| - lambda)_+ (b_jk = 0), divided by lambda;
 *   dual_gap  = max over k of (P - D) / P of the lasso subproblem, with
 *               rr = S_kk - b'S_.k - b'g, yr = S_kk - b'S_.k,
 *               s = min(1, lambda / ||g||_inf), P = rr / 2 + lambda ||b||_1,
 *               D = s yr - s^2 rr / 2;
 *   err_est   = the first-order estimate of max |dTheta| / max |Theta| that
 *               these residuals and the sigma fixed-point residual imply, with
 *               the rounding bound of a working matrix built in
 *               opts->precision from n samples added (spmesl_stats).
 * The same check runs after a fit with opts->diagnostics = 1.  The paper has
 * no such routine; it defines the conditions checked.
 *   S       p x p covariance as for spmesl_fit (read only).
 *   n       sample size for the rounding bound (and lambda rules); 0 = 1.
 *   B       p x p FP64 coefficients in the original scale, B[j*p + k] = b_jk
 *           (the layout of spmesl_fit_coefficients); sigma: p FP64 values.
 *   stats   host, required: status, lambda0, diagnostics = 1, kkt_viol,
 *           dual_gap and err_est are written; the call synchronises `stream`.
 *   workspace  spmesl_fit_workspace_bytes(p, precision), 256-byte aligned.
 * Errors: EINVAL (NULL pointers, p < 2 or above spmesl_max_p, short or
 * misaligned workspace, no usable lambda0), ENONFINITE (non-finite S or
 * S_jj <= 0), ECUDA.
 */
spmesl_status spmesl_diagnose(const void* S, int n, int p, double lambda0, const double* B,
                              const double* sigma, const spmesl_opts* opts, spmesl_stats* stats,
                              void* workspace, size_t ws_bytes, void* stream);

/*
 * One scaled-lasso regression (Section 2.1, Eq. (2); Algorithm 1): the joint
 * minimiser over (beta, sigma > 0) of
 *     ||y - X beta||^2 / (2 n sigma) + sigma / 2 + lambda0 ||beta||_1,
 * with the predictors standardised when opts->standardize (the weighted
 * penalty lambda0 sqrt(s_kk) |beta_k| of Proposition 1; beta and sigma are
 * returned in the original scale), by cyclic coordinate descent with the
 * alternating sigma update of Eq. (14).  It is one column problem of SPMESL:
 * the Gram of [X y] is built (spmesl_gram, so SPMESL_MIXED uses the
 * tensor-core Gram) and column p is solved.
 *   X        n x p predictors, row-major (ld p), device, element type per
 *            opts->precision (double for SPMESL_FP64, float otherwise).
 *   y        n responses, device, same type.
 *   lambda0  penalty level; with opts->lambda_rule != GIVEN the rule is
 *            applied with (n, p) and lambda0 is ignored.
 *   beta     p doubles (device), written on SPMESL_OK / NOT_CONVERGED /
 *            EDEGENERATE; sigma: one double (device).
 *   stats    optional host pointer; non-NULL synchronises `stream` and
 *            fills the counters of the one column solve (nnz_B = nonzero
 *            beta, ms_total = whole call).
 *   workspace  spmesl_scaled_lasso_workspace_bytes(n, p, precision) bytes,
 *            256-byte aligned, owned by the caller.
 * opts: precision, standardize, center, lambda_rule, heavy_heat and
 * heavy_min_p are used; the inner rule is the per-column one and the gradient
 * SPMESL_GRADIENT_AUTO (the column solved as in a whole fit).
 * Errors: EINVAL (NULL pointers, n < 1, p < 1, p + 1 above spmesl_max_p,
 * tol <= 0, maxit < 1, short or misaligned workspace, no usable lambda0),
 * ENONFINITE (non-finite data), ECUDA.
 */
size_t spmesl_scaled_lasso_workspace_bytes(int n, int p, int precision);
spmesl_status spmesl_scaled_lasso(const void* X, const void* y, int n, int p, double lambda0,
                                  double tol, int maxit, const spmesl_opts* opts, double* beta,
                                  double* sigma, spmesl_stats* stats, void* workspace,
                                  size_t ws_bytes, void* stream);

/*
 * Support-recovery and estimation-error measures of an estimate against the
 * true precision matrix, as defined in Section 4.2 (the estimation study):
 * over the pairs j < k an entry is an edge when it is not exactly zero;
 *   SEN = TP/(TP+FN), SPE = TN/(TN+FP), FDR = FP/(TP+FP),
 *   MISR = (FP+FN)/(p(p-1)/2),
 *   MCC = (TP TN - FP FN)/sqrt((TP+FP)(TP+FN)(TN+FP)(TN+FN)),
 * and the Frobenius norm of Theta_hat - Theta_true over all entries.  A ratio
 * with a zero denominator is NaN.  The paper has no GPU counterpart: this is
 * the evaluation of its estimates.
 *   Theta_hat, Theta_true  p x p FP64, row-major, device.
 *   out        host pointer; the call synchronises `stream`.
 *   workspace  spmesl_metrics_workspace_bytes() bytes, 256-byte aligned.
 * The sums are formed in a fixed order (deterministic).
 * Errors: EINVAL (NULL pointers, p < 2, short or misaligned workspace), ECUDA.
 */
typedef struct {
    int64_t tp, fp, tn, fn;
    int64_t n_edges_hat;        /* TP + FP */
    int64_t n_edges_true;       /* TP + FN */
    double frobenius;           /* ||Theta_hat - Theta_true||_F */
    double sen, spe, fdr, misr, mcc;
} spmesl_metrics;

size_t spmesl_metrics_workspace_bytes(void);
spmesl_status spmesl_support_metrics(const double* Theta_hat, const double* Theta_true, int p,
                                     spmesl_metrics* out, void* workspace, size_t ws_bytes,
                                     void* stream);

/*
 * End-to-end solve from HOST data (Section 2.2 and Algorithm 2): copies X_host
 * to the device, builds S
 * (spmesl_gram), fits (spmesl_fit), copies Theta and sigma back to the host
 * buffers and synchronises `stream`.
 *   X_host      n x p row-major host buffer (FP64 for SPMESL_FP64, else FP32);
 *               pinned memory gives the fastest copies.
 *   Theta_host  p x p FP64 host output; sigma_host p FP64 host output.
 *   workspace   device scratch of spmesl_solve_workspace_bytes(n, p, precision).
 * Returns the fit's status (errors as spmesl_gram and spmesl_fit).
 */
size_t spmesl_solve_workspace_bytes(int n, int p, int precision);
spmesl_status spmesl_solve(const void* X_host, int n, int p, double lambda0, double tol,
                           int maxit, const spmesl_opts* opts, double* Theta_host,
                           double* sigma_host, spmesl_stats* stats, void* workspace,
                           size_t ws_bytes, void* stream);

/*
 * Batched fits: many independent SPMESL problems of different p and n solved
 * together (Algorithm 2 for each; the columns of all fits share one
 * coordinate-descent launch, Section 3.3's observation that the p column
 * problems are independent extended across problems).
 *
 * spmesl_problem describes one fit; all pointers are device pointers owned by
 * the caller and must stay valid while the batch runs:
 *   X        n x p data (row-major, ld p) from which S = X'X/n is built, or
 *            NULL to use S directly.  Element type per opts->precision.
 *   S        p x p covariance (used when X is NULL).
 *   lambda0  penalty level; <= 0 means "apply opts->lambda_rule with n, p".
 *   Theta    p x p FP64 output; sigma p FP64 output (as spmesl_fit).
 */
typedef struct {
    const void* X;
    const void* S;
    int32_t n;
    int32_t p;
    double lambda0;
    double* Theta;
    double* sigma;
} spmesl_problem;

typedef struct spmesl_batch spmesl_batch;

/* Plan a batch of Algorithm 2 fits (host only: sizes, ordering, workspace
 * layout).  The problems
 * are copied; tol and maxit apply to every fit.  opts: precision FP64, FP32 or
 * MIXED (FP32 data; the Gram of every fit given as X runs as split-BF16
 * products on the tensor cores in one launch for the whole batch, the rest as
 * in the single-fit mixed path, so each fit equals spmesl_gram + spmesl_fit
 * with SPMESL_MIXED), inner_rule must be SPMESL_INNER_COLUMN,
 * standardize / center / lambda_rule /
 * warps_per_block / use_graph as documented in spmesl_opts.
 * Errors: EINVAL (no problems, p < 2 or above spmesl_max_p, missing
 * pointers, no usable lambda0), ENOMEM (host allocation). */
spmesl_status spmesl_batch_create(const spmesl_problem* problems, int count, double tol,
                                  int maxit, const spmesl_opts* opts, spmesl_batch** batch);

/* Device workspace of a batch of Algorithm 2 fits (256-byte aligned when
 * passed). */
size_t spmesl_batch_workspace_bytes(const spmesl_batch* batch);

/* Enqueue the whole batch on `stream` (Section 2.2 and Algorithm 2 per fit):
 * descriptor upload, Gram (fits with X),
 * standardisation, coordinate descent, Theta.  Asynchronous.  With use_graph
 * the sequence is captured into a CUDA graph on the first run (per
 * workspace) and replayed afterwards.  The workspace must not be reused until
 * the run has completed. */
spmesl_status spmesl_batch_run(spmesl_batch* batch, void* workspace, size_t ws_bytes,
                               void* stream);

/* The batch's outcome (Algorithm 2 per fit): synchronise `stream`, write
 * each fit's status to statuses[i] (host array in
 * the caller's problem order, may be NULL) and aggregate counters to stats
 * (may be NULL).  Returns the most severe status. */
spmesl_status spmesl_batch_result(const spmesl_batch* batch, const void* workspace,
                                  int32_t* statuses, spmesl_stats* stats, void* stream);

/* A helper (no passage of the paper): the counters of fit i (caller's order)
 * from the last spmesl_batch_result:
 * status, sweeps, moves, nonzero coefficients, the block solver's columns, the
 * penalty level and, with opts.diagnostics, the fit's kkt_viol / dual_gap /
 * err_est (the aggregate of spmesl_batch_result gives their maxima).  Host
 * only.  EINVAL for a bad index, ENOTFOUND before the first result. */
spmesl_status spmesl_batch_fit_stats(const spmesl_batch* batch, int i, spmesl_stats* stats);

/* Autotune (not in the paper) warps per block of the batch's
 * coordinate-descent launch (Algorithm 1 per column) by timing
 * a few candidates on this workspace (runs the batch several times); the
 * choice is kept in the batch and written to *best_warps. */
spmesl_status spmesl_batch_tune(spmesl_batch* batch, void* workspace, size_t ws_bytes,
                                void* stream, int* best_warps);

/*
 * Launch choice of the batch tuner (not in the paper): warps per block of the
 * lazy launch, the lazy solver's hand-over support (opts.handover), the fit
 * size from which heavy columns are routed by heat (opts.heavy_min_p, -1 =
 * never) and the heat limit, with the step time measured for it.
 */
typedef struct {
    int32_t warps_per_block;
    int32_t handover;
    int32_t heavy_min_p;
    int32_t heavy_heat;
    float ms;                   /* measured time of one batch run with this choice, ms */
    int32_t from_cache;         /* 1: read from the cache file, nothing timed */
} spmesl_tune_choice;

/* Autotune with a persistent cache (not in the paper): with cache_path
 * non-NULL, a choice stored for this class of batch (spmesl_tune_key) by the
 * same library version is applied without timing; otherwise the batch is run
 * for every candidate (warps 4 or 8; hand-over support 32 or 64; heat routing
 * from p >= 4096, from p >= 1024 or never), the fastest is applied and, with
 * cache_path, stored.  Runs the batch several times on `workspace` when it
 * times.  out (host, may be NULL) receives the choice.  Errors: EINVAL, ECUDA. */
spmesl_status spmesl_batch_tune_cached(spmesl_batch* batch, void* workspace, size_t ws_bytes,
                                       void* stream, const char* cache_path,
                                       spmesl_tune_choice* out);

/* A helper (no passage of the paper): the tuning cache's key of a class of
 * batches: precision, standardisation, SM count and the power-of-two buckets
 * of the largest p, the mean n and the number of fits.  Writes at most len
 * bytes to key; returns its length, or -1. */
int spmesl_tune_key(int precision, int standardize, int sms, int count, int max_p, double mean_n,
                    char* key, size_t len);

/* A helper (no passage of the paper): the choice stored under key in the
 * JSON cache file at path by this library version (from_cache = 1), else
 * ENOTFOUND (no file, no entry, another version, or a malformed file). */
spmesl_status spmesl_tune_cache_lookup(const char* path, const char* key, spmesl_tune_choice* out);

/* A helper (no passage of the paper): store the choice under key in the cache
 * file at path (other entries kept; written to a temporary file and renamed).
 * EINVAL if the file cannot be written or the key holds a quote. */
spmesl_status spmesl_tune_cache_store(const char* path, const char* key,
                                      const spmesl_tune_choice* choice);

/* A helper (no passage of the paper): release the batch's host resources
 * (pinned staging, captured graph). */
void spmesl_batch_destroy(spmesl_batch* batch);

/*
 * Serving context: continuous batching of requests that arrive over time.
 * A worker thread admits queued requests in arrival order while the device
 * bytes of all admitted requests stay within `mem_budget_bytes` and at most
 * `max_slots` requests are admitted.  The requests of one admission round run
 * as one batch (as spmesl_batch_run) on one of the context's streams;
 * requests that arrive while earlier batches run are admitted into new
 * batches on other streams, so their work overlaps on the device.  A result
 * does not depend on what it was batched with.  The paper has no serving
 * system; each request is the fit of Algorithm 2.
 *
 * spmesl_ctx_create: tol / maxit apply to every request; opts: precision FP64,
 *   FP32 or MIXED (inner_rule COLUMN), other fields as for spmesl_batch_create.
 *   Uses the current device.  Errors: EINVAL, ENOMEM, ECUDA.
 * spmesl_submit: `request` (an spmesl_problem: device pointers that must stay
 *   valid until the request completes; lambda0 <= 0 applies opts->lambda_rule)
 *   is queued and *ticket receives its id.  EINVAL for a bad request, ENOMEM
 *   if the request alone exceeds the budget, EBUSY if the queue is full.
 * spmesl_poll: the request's status once it has completed (its Theta and
 *   sigma are then written, and stats gets ms_queue / ms_total / batch_size);
 *   EBUSY while it is queued or running; ENOTFOUND for an unknown ticket or
 *   one already reported.
 * spmesl_ctx_query: queued and admitted request counts and the device bytes
 *   admitted requests hold.
 * spmesl_ctx_destroy: waits for the batches in flight, then frees the
 *   context; requests still queued are dropped.
 */
typedef struct spmesl_ctx spmesl_ctx;
spmesl_status spmesl_ctx_create(spmesl_ctx** ctx, size_t mem_budget_bytes, int max_slots,
                                double tol, int maxit, const spmesl_opts* opts);
spmesl_status spmesl_submit(spmesl_ctx* ctx, const spmesl_problem* request, uint64_t* ticket);
spmesl_status spmesl_poll(spmesl_ctx* ctx, uint64_t ticket, spmesl_stats* stats);
spmesl_status spmesl_ctx_query(spmesl_ctx* ctx, int32_t* queued, int32_t* running,
                               size_t* bytes_in_use);
void spmesl_ctx_destroy(spmesl_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPMESL_H */
