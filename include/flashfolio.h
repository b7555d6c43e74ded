/*
 * flashfolio.h -- C ABI of the GB300 portfolio solver.
 *
 * The library solves the single-period portfolio model of Sec. 2.1 (Eqs. 1-3)
 *
 *     max_w  GMV alpha^T w - lambda1 GMV^2 w^T Sigma w
 *            - lambda2 GMV s^T |w - w0| - lambda3 GMV q^T |w - w0|^d
 *     s.t.   L <= A w <= U,   ||w||_1 <= 1,
 *
 * and the multi-period model of Sec. 2.2 (Eqs. 4-6), the same terms summed
 * over t = 1..T with risk on (w_t - w_T), costs on (w_t - w_{t-1}), w_0 and w_T
 * fixed and the constraints imposed for t = 1..T-1.  The risk matrix has the
 * factor form Sigma = F Omega F^T + diag(D) of Sec. 3.2 (F is the paper's beta,
 * Omega its Sigma_f).
 *
 * The paper gives no algorithm beyond "a first-order method that stops on a
 * fixed-point residual, started at w0" (Sec. 4.1).  This library runs a
 * restarted, reflected Halpern iteration of the Condat-Vu primal-dual
 * splitting on
 *     min f(x) + sum_t indicator(||x_t||_1 <= 1) + h_A(A x_t) + phi(Delta x + b)
 * (f = return + risk, h_A = indicator of [L, U], phi = spread + impact cost
 * on the trades) and stops on the relative KKT residual
 *     max(r_primal, r_dual, r_gap) <= tol
 * whose three parts are reported in ff_result.
 *
 * Conventions for every entry point:
 *   - Pointers inside ff_problem are DEVICE pointers owned by the caller;
 *     the library never frees or reallocates them and reads them only.
 *   - ws is a caller-owned device workspace of at least ff_workspace_size()
 *     bytes, 256-byte aligned.  Its contents are overwritten.
 *   - All calls are asynchronous on the CUDA stream passed as `stream`
 *     (a cudaStream_t; NULL = legacy default stream).  Device results are
 *     valid once the stream reaches the point of the call.
 *   - Return value: FF_OK or an FF_ERR_* code.  Argument errors are detected
 *     on the host before anything is enqueued.  Nothing aborts, traps or
 *     prints.  Per-instance solver outcomes are written to ff_result.status.
 */
#ifndef FLASHFOLIO_H
#define FLASHFOLIO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------- */
#define FF_OK                  0
#define FF_ERR_INVALID_ARG     1   /* a size, pointer, bound or option is invalid */
#define FF_ERR_CUDA            2   /* a CUDA runtime call failed */
#define FF_ERR_WORKSPACE       3   /* ws too small or misaligned */
#define FF_ERR_UNSUPPORTED     4   /* shape exceeds what the kernels support */
#define FF_ERR_DEVICE          5   /* device-side error flag (bounded wait expired) */

/* ff_result.status (per instance) */
#define FF_CONVERGED           0   /* relative KKT <= tol */
#define FF_MAX_ITER            1   /* iteration limit reached */
#define FF_TIME_LIMIT          2   /* device clock passed options.time_limit */
#define FF_NUMERICAL           3   /* NaN/Inf met in the iteration */
#define FF_STALLED             4   /* a bounded wait for a panel tile copy expired */
#define FF_PRECISION           5   /* FP32/BF16 modes: the relative KKT residual stopped halving
                                      (options.stall_checks checks): the mode's rounding floor was
                                      reached above tol; solve again with FF_PREC_F64 */

/* element types */
#define FF_F64                 0
#define FF_F32                 1

/* precision modes of the solver */
#define FF_PREC_F64            0   /* panels, products, iterates and reductions in FP64 */
#define FF_PREC_F32            1   /* FP32 panels and products; FP64 iterate state updated by
                                      FP32 increments; FP64 reductions and KKT */
#define FF_PREC_BF16           2   /* BF16 F and A panels, FP32 products; otherwise as FP32 */

/* One problem instance in the paper's notation and units (Eqs. 1-6).
 * Single period: T = 0; D, alpha, s, q hold n entries.
 * Multi-period:  T >= 2; D, alpha, s, q hold T x n entries (row t-1 is period
 *   t = 1..T; the row for t = T of alpha and D only enters a constant); wT
 *   holds n entries.
 * F is n x k row-major (asset-major), A is m x n row-major, Omega is k x k
 * row-major (or its diagonal when omega_diag = 1).  L and U have m entries
 * (+-INFINITY allowed, L <= U).  All arrays have element type `dtype`. */
typedef struct ff_problem {
    int32_t n, k, m;
    int32_t T;
    int32_t dtype;          /* FF_F64 or FF_F32 */
    int32_t omega_diag;     /* 1: Omega points to k diagonal entries */
    const void* F;
    const void* Omega;
    const void* D;
    const void* alpha;
    const void* s;
    const void* q;
    const void* w0;
    const void* wT;         /* multi-period only, else NULL */
    const void* A;          /* may be NULL when m = 0 */
    const void* L;
    const void* U;
    double GMV, lambda1, lambda2, lambda3, d;   /* GMV > 0, lambda1 > 0, lambda2,3 >= 0, 1 < d <= 2 */
} ff_problem;

typedef struct ff_options {
    double  tol;                /* relative KKT tolerance, default 1e-6 */
    int64_t max_iter;           /* default 400000 */
    double  time_limit;         /* seconds of device time, default 360 (Sec. 4.1) */
    int32_t precision;          /* FF_PREC_*, default FF_PREC_F32 */
    int32_t check_every;        /* iterations between KKT/restart checks, default 64 */
    double  reflection;         /* Halpern reflection rho, default 1/3; must satisfy
                                   rho <= (2 beta - 1) / (2 beta) so that the reflected
                                   operator stays nonexpansive */
    double  restart_sufficient; /* default 0.2 */
    double  restart_necessary;  /* default 0.8 */
    double  step_fraction;      /* primal step tau = step_fraction * 2 / L_f, default 0.4 */
    int32_t cluster_size;       /* CTAs per instance: 0 = automatic (see cta_work), else 1, 2, 4,
                                   8 or 16 for every instance */
    int32_t max_teams;          /* batch: concurrent instance teams, 0 = as many as fit */
    double  beta;               /* dual steps sigma_i ||K_i||^2 sum to 1/tau - beta L_f, so the
                                   smooth part is (beta)-cocoercive in the step metric; beta > 1/2,
                                   default 0.75 */
    int32_t reuse_workspace;    /* 0 (default): copy the instance table to ws, repack, solve.
                                   1: ws already holds the table and the repacked data of exactly
                                   these problems from an earlier call with the same ws (same
                                   arrays, same values): only the solver runs.
                                   2: ws already holds the table (same problems, same pointers)
                                   but the arrays may hold new values: repack and solve, with no
                                   host-to-device copy (the call is then capturable in a CUDA
                                   graph once a mode-0 call has run outside the capture). */
    double  cta_work;           /* batch scheduling: asset-periods per CTA that decide each
                                   instance's cluster size (smallest power of two G <= 16 with
                                   n * P / G <= cta_work; while the batch would fill fewer than
                                   half the SMs, the instance with the most work per CTA is
                                   split further); default 8192.  Instances of equal G and kind
                                   (single- or multi-period) form one persistent launch; the
                                   launches run concurrently on library-owned streams forked
                                   from `stream`. */
    double  restart_artificial; /* also restart once the iterations since the last restart
                                   reach this share of all iterations so far (0 = off);
                                   default 0.36 */
    int32_t stall_checks;       /* FP32/BF16 modes: end an instance with FF_PRECISION once its
                                   relative KKT residual has not halved over this many checks;
                                   0 = never; default 48 */
    int32_t round_panels_bf16;  /* FF_PREC_F64 only: round F and A to bfloat16 (nearest even) in
                                   the repack, so that an FP64 solve sees exactly the data of an
                                   FF_PREC_BF16 solve of the same arrays; default 0 */
    int32_t warm_start;         /* 0 (default): start every instance at w0 (single) or on the
                                   straight line from w0 to w_T (multi), with zero multipliers.
                                   1: start from the values the output buffers hold when the call
                                   runs (w_out; yA_out and yD_out where given, else zero): warm start
                                   from the solution of a neighbouring problem (another date or
                                   lambda).  The outputs are overwritten with the result as usual. */
    int32_t panel_l2_keep;      /* 1 (default): the copies of the panel tiles ask the L2 to keep
                                   their lines (evict_last policy); every iteration reads an
                                   instance's panel twice.  0: default L2 policy */
    int32_t primal_weight;      /* 0 (default): fixed steps.  1: adaptive primal weight: at every
                                   restart the ratio of the dual to the primal step moves halfway (in
                                   logarithm) toward the ratio of the distances the dual and the
                                   primal iterates travelled since the previous restart; the steps
                                   keep satisfying the Condat-Vu condition */
    int32_t test_expire_first_wait; /* testing aid, default 0.  1: the first wait of each
                                   instance for a panel-tile copy counts as expired (the copy
                                   itself is valid and is let land before the team moves on),
                                   so the instance ends with FF_STALLED; this exercises the
                                   bounded-wait path without a faulty copy */
} ff_options;

/* Per-instance outcome, written to DEVICE memory by the solve calls. */
typedef struct ff_result {
    int32_t status;             /* FF_CONVERGED, FF_MAX_ITER, FF_TIME_LIMIT, FF_NUMERICAL, FF_STALLED,
                                   FF_PRECISION */
    int32_t restarts;
    int64_t iterations;
    double  rel_kkt;            /* max(r_primal, r_dual, r_gap) at the returned point */
    double  r_primal, r_dual, r_gap;   /* r_primal = ||Ax - clip(Ax)|| / (||Ax|| + ||clip(Ax)||);
                                   r_dual = ||x - Proj(x - grad f - K^T y)|| /
                                   (||x|| + ||grad f|| + ||K^T y||); r_gap = |P - D| / (|P| + |D|) */
    double  primal_obj;         /* scaled minimisation objective P(x) = -(Eq. 1)/GMV (+ constant, multi) */
    double  dual_obj;           /* the matching dual bound */
    double  paper_obj;          /* Eq. 1 / Eq. 4 in the paper's units (maximised) */
    double  fixed_point_res;    /* ||z - T(z)|| in the step-size metric at the last check */
    double  seconds;            /* device time of this instance's solve */
    double  lipschitz;          /* 2 lambda1 GMV lambda_max(Sigma) estimate used for the step */
    int64_t threshold_rounds;   /* rounds of the l1-threshold search over the whole solve */
    double  phase_seconds[6];   /* device time by phase (rank 0 of the team): setup,
                                   expand pass, l1 thresholds, elementwise prox,
                                   reduce pass + team sums, KKT checks */
    double  term_scale;         /* Phi = sum |alpha_i x_i| + risk + trading cost at the returned
                                   point (scaled units): the magnitude of the objective's terms,
                                   against which |P - D| can also be read */
} ff_result;

/* Fill *o with the defaults listed above. */
void ff_default_options(ff_options* o);

/* Bytes of device workspace for `count` instances (host only, no CUDA call).
 * Returns 0 if an argument is invalid. */
size_t ff_workspace_size(const ff_problem* probs, int count, const ff_options* o);

/* Solve one single-period instance (p->T == 0).
 *   result_dev : device pointer to one ff_result.
 *   w_out      : device, n entries of p->dtype: the post-trade portfolio w.
 *   yA_out     : device, m entries of p->dtype or NULL: exposure-row multipliers.
 *   yD_out     : device, n entries of p->dtype or NULL: trade multipliers. */
int ff_solve_single(const ff_problem* p, const ff_options* o, void* ws, size_t ws_bytes,
                    ff_result* result_dev, void* w_out, void* yA_out, void* yD_out, void* stream);

/* Solve one multi-period instance (p->T >= 2).
 *   w_out  : device, (T-1) x n entries: w_1..w_{T-1}.
 *   yA_out : device, (T-1) x m entries or NULL.   yD_out : device, T x n entries or NULL. */
int ff_solve_multi(const ff_problem* p, const ff_options* o, void* ws, size_t ws_bytes,
                   ff_result* result_dev, void* w_out, void* yA_out, void* yD_out, void* stream);

/* Solve `count` independent instances (single- and multi-period mixed) in one
 * persistent launch.  probs is a HOST array of count problems (1 <= count <=
 * 65535); w_out is a HOST array of count DEVICE pointers (layout as above);
 * yA_out and yD_out are NULL or HOST arrays of count DEVICE pointers (entries
 * may be NULL) receiving the multipliers as in ff_solve_single/multi;
 * result_dev is a device array of count ff_result. */
int ff_solve_batch(const ff_problem* probs, int count, const ff_options* o, void* ws, size_t ws_bytes,
                   ff_result* result_dev, void* const* w_out, void* const* yA_out, void* const* yD_out,
                   void* stream);

/* Workspace bytes of ff_solve_joint_batch for these instances (host only; 0 if
 * an instance is not single-period or a size is invalid).  Per instance about
 * 8 n (k + m + 12) bytes: FP64 copies of F (transposed) and A, and the state. */
size_t ff_joint_workspace_size(const ff_problem* probs, int count);

/* The joint primal prox variant of the single-period solve (Eqs. 1-3): the
 * trading cost and the budget set of Eq. 3 form one primal prox,
 *   prox(v)_i = argmin_w 0.5 (w - v_i)^2 + tau phi_i(w - w0_i) + mu |w|,
 * with the budget multiplier mu found by a safeguarded Newton iteration, so the
 * only multiplier of the iteration is y_A; the steps, the reflected Halpern
 * scheme, the restarts and the relative KKT test are those of ff_solve_batch;
 * the KKT test's trade multiplier is the cost's slope phi'(w - w0), or on the
 * cost's kink (w = w0) the remainder of the prox's optimality condition.
 * FP64 throughout, one CTA per instance; o->precision must be FF_PREC_F64
 * (else FF_ERR_UNSUPPORTED; o = NULL gives the defaults with FF_PREC_F64),
 * every instance single-period (T = 0) with k <= 256
 * and m <= 256 (else FF_ERR_UNSUPPORTED).  warm_start, cluster_size, cta_work,
 * max_teams, stall_checks, round_panels_bf16, panel_l2_keep, primal_weight and
 * the test hook have no effect.  Arguments and outputs as ff_solve_batch
 * (yD_out receives the recovered trade multiplier); ff_result.threshold_rounds
 * counts the evaluations of ||w(mu)||_1.  ws: ff_joint_workspace_size bytes,
 * 256-byte aligned.  Asynchronous on `stream` (one launch after a host-to-device
 * copy of the instance table); FF_OK or an FF_ERR_* code. */
int ff_solve_joint_batch(const ff_problem* probs, int count, const ff_options* o, void* ws, size_t ws_bytes,
                         ff_result* result_dev, void* const* w_out, void* const* yA_out, void* const* yD_out,
                         void* stream);

/* Size of the library-owned workspace used by ff_solve_single_static (32 MiB). */
#define FF_STATIC_WORKSPACE_BYTES (32u * 1024u * 1024u)

/* ff_solve_single_static: ff_solve_single without a caller workspace and
 * without any allocation.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory at solve time, for
 * example a host application or plugin framework that has reserved all
 * device memory up front and hands out only fixed buffers, or a
 * latency-critical loop where the implicit device synchronisation of
 * cudaMalloc / cudaFree is not acceptable.
 *
 * Arguments, layouts and results are those of ff_solve_single (the caller
 * still passes the problem arrays, result_dev and the outputs as device
 * pointers); the cluster size is chosen as there.  options.reuse_workspace
 * has no effect: every call writes the instance record and repacks the
 * problem into the array.  The workspace is a file-scope device array of
 * FF_STATIC_WORKSPACE_BYTES inside this library, which every GPU that loads
 * the library holds until the process exits.  The call makes no cudaMalloc,
 * cudaFree or other allocating call on the host or the device.
 *
 * - Problems whose workspace (ff_workspace_size for this one instance plus a
 *   few hundred bytes of instance record) exceeds FF_STATIC_WORKSPACE_BYTES
 *   are rejected with FF_ERR_WORKSPACE before anything is enqueued;
 *   ff_last_error() then states the bytes needed.
 * - The first call on each device looks up the array's device address with
 *   cudaGetSymbolAddress (with that device current) and caches it.
 * - Every call on a device shares the one array, and it keeps the previous
 *   call's contents (nothing in it needs to start at zero: each solve writes
 *   every region before reading it).  Calls that overlap on the GPU (other
 *   streams, or other host threads) race on it: serialise them.
 * Returns FF_OK or an FF_ERR_* code, like ff_solve_single. */
int ff_solve_single_static(const ff_problem* p, const ff_options* o, ff_result* result_dev,
                           void* w_out, void* yA_out, void* yD_out, void* stream);

/* Host-only schedule of ff_solve_batch for these problems and options (no
 * device work; it reads the SM count of the current device when one is
 * present): cluster_out (HOST, count entries, may be NULL) receives each
 * instance's CTAs per instance, launches_out (may be NULL) the number of
 * persistent solver launches (one per distinct cluster size and kind,
 * single- or multi-period).  A cluster
 * size that cannot be resident on the device is halved at solve time. */
int ff_batch_plan(const ff_problem* probs, int count, const ff_options* o, int32_t* cluster_out,
                  int32_t* launches_out);

/* Message for an FF_* return code (static storage). */
const char* ff_status_string(int code);

/* Gradient outputs of the adjoint calls: DEVICE pointers with the layout and
 * element type of the matching ff_problem arrays (single period: alpha, D, s,
 * q, w0 hold n entries; multi-period: alpha, D, s, q hold T x n and w0, wT n;
 * F: n x k row-major).  Any may be NULL (not computed).  wT is used by
 * multi-period instances only. */
typedef struct ff_grads {
    void* alpha;
    void* F;
    void* D;
    void* s;
    void* q;
    void* w0;
    void* wT;
} ff_grads;

/* Workspace bytes of ff_backward for this problem (host only; 0 if p is
 * invalid): the single-period adjoint for T == 0, the multi-period one
 * (ff_backward_multi_workspace_size of this one instance) for T >= 2. */
size_t ff_backward_workspace_size(const ff_problem* p);

/* Vector-Jacobian product of the single-period solve (Sec. 2.1, Eqs. 1-3):
 * with L = <grad_w, w*>, writes dL/dalpha, dL/dF, dL/dD, dL/ds, dL/dq and
 * dL/dw0 (paper units: alpha, F, D, s, q, w0 as passed in p) to `out`.
 * Implicit differentiation of the optimality conditions at w*: the active
 * structure is read from the forward results (zero holdings: w_i == 0; dead
 * trades: |yD_i| < lambda2 s_i; active exposure rows: |yA_j| > 1e-12 max|yA|;
 * active budget: ||w||_1 >= 1 - 1e-10 for FP64 data, 1 - 1e-6 for FP32), and
 * the reduced KKT system is solved
 * in FP64 on the GPU (Woodbury through the k x k factor block, Schur
 * complement on the active constraints).  A is treated as independent data
 * (no derivative through A).  At a point where a piece is exactly on its
 * kink boundary the result is the one-sided derivative of the identified
 * active set.
 *   w, yA, yD  : device, the forward outputs of ff_solve_single (n, m, n
 *                entries of p->dtype; yA may be NULL when m = 0).
 *   grad_w     : device, n entries of p->dtype.
 *   status_dev : device int32 or NULL: 0 ok, 1 / 2 a factorisation met a
 *                non-positive pivot (degenerate active set).
 * Asynchronous on `stream`; FF_OK or an FF_ERR_* code. */
int ff_backward_single(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                       const ff_grads* out, void* ws, size_t ws_bytes, int32_t* status_dev, void* stream);

/* The adjoint entry point for any instance (implicit differentiation of the
 * solve): a single-period instance (p->T == 0, Eqs. 1-3) goes to
 * ff_backward_single, a multi-period one (p->T >= 2, Eqs. 4-6) to
 * ff_backward_multi_batch with count 1; arguments, layouts, statuses and
 * workspace as there (ff_backward_workspace_size covers both).  Invalid
 * arguments return FF_ERR_INVALID_ARG before anything is enqueued. */
int ff_backward(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                const ff_grads* out, void* ws, size_t ws_bytes, int32_t* status_dev, void* stream);

/* Workspace bytes of ff_backward_multi_batch for these instances (host only;
 * 0 if an instance is not multi-period or a size is invalid).  Per instance it
 * is about 333 (T-1) n + 16 ((T-1)(m+1))^2 bytes: the second term holds the
 * matrix of the active constraint rows and its inverse. */
size_t ff_backward_multi_workspace_size(const ff_problem* probs, int count);

/* Vector-Jacobian products of the multi-period solve (Sec. 2.2, Eqs. 4-6) for
 * `count` instances (all with T >= 2): with L = <grad_w, x*> summed over the
 * T-1 free periods, writes dL/dalpha, dL/dD, dL/ds, dL/dq (T x n each; the
 * rows t = T of alpha and D receive 0, they enter only a constant), dL/dF
 * (n x k), dL/dw0 and dL/dwT (n each) to out[t] (paper units, as passed).
 * The active structure is read from the forward results of ff_solve_multi /
 * ff_solve_batch: dead trades |yD_{r,i}| < lambda2 s_{r,i} (they tie
 * neighbouring periods, or a period to w0 / w_T), zero holdings w == 0, the
 * budget of period t when ||w_t||_1 >= 1 - 1e-10 (FP64 data; 1 - 1e-6 for
 * FP32), exposure rows with |yA| > 1e-12 max|yA|.  The reduced KKT system is
 * solved in FP64 on the GPU by projected conjugate gradients (per-asset
 * tridiagonal preconditioner; constraint rows through the explicit inverse of
 * E M^-1 E^T, with linearly dependent rows dropped); A is treated as
 * independent data (no derivative through A).
 *   probs, w, yA, yD, grad_w, out : HOST arrays of count entries; the pointers
 *       inside are DEVICE pointers: w (T-1) x n, yA (T-1) x m (NULL allowed when
 *       m = 0), yD T x n, grad_w (T-1) x n, all of the problem's dtype.
 *   status_dev : device array of count int32 or NULL: 0 ok, 3 the conjugate
 *       gradients reached their iteration limit (600), 4 a non-positive or
 *       non-finite curvature / residual was met (degenerate active set), 5 a
 *       bounded wait at a grid barrier expired (outputs undefined).
 *   ws : device workspace of ff_backward_multi_workspace_size bytes, 256-byte
 *       aligned; its contents are overwritten.
 * Asynchronous on `stream`: one cooperative kernel launch (the phases of the
 * computation are separated by grid barriers; every wait at a barrier is
 * bounded, and a wait that expires ends every instance with status 5) after
 * a host-to-device copy of the instance table and a memset of the barrier
 * state; no host synchronisation.  FF_ERR_UNSUPPORTED if the device has no
 * cooperative launch; FF_OK or an FF_ERR_* code. */
int ff_backward_multi_batch(const ff_problem* probs, int count, const void* const* w, const void* const* yA,
                            const void* const* yD, const void* const* grad_w, const ff_grads* out, void* ws,
                            size_t ws_bytes, int32_t* status_dev, void* stream);

/* ff_backward_single for `count` single-period instances in one launch (one
 * CTA per instance).  probs, w, yA, yD, grad_w and out are HOST arrays of
 * count entries (pointers inside are DEVICE pointers as in
 * ff_backward_single; yA may be NULL when every m = 0); status_dev is NULL
 * or a device array of count int32.  Workspace: ff_backward_batch_workspace_size. */
size_t ff_backward_batch_workspace_size(const ff_problem* probs, int count);
int ff_backward_batch(const ff_problem* probs, int count, const void* const* w, const void* const* yA,
                      const void* const* yD, const void* const* grad_w, const ff_grads* out, void* ws,
                      size_t ws_bytes, int32_t* status_dev, void* stream);

/* ---- risk-model estimation (Sec. 3.2) ---------------------------------
 * For `count` estimation windows of T days (one per date; the paper uses the
 * previous 504 business days), with p factor returns and n stock returns per
 * day, estimate the factor model Sigma = beta Sigma_f beta^T + D of Sec. 3.2:
 *   Sigma_f = (F - 1 1^T F / T)^T (F - 1 1^T F / T) / (T - 1),
 *   beta_i  = least-squares coefficients of r_i ~ F beta_i (no intercept) over
 *             the days on which stock i has a return,
 *   D_ii    = sample variance (mean removed, divisor days - 1) of the residuals
 *             theta_{k,i} = r_{k,i} - beta_i^T f_k over those days.
 * A stock's returns start on its first day in the window (NaN before: a
 * listing inside the window); a NaN after that makes it irregular.  Stocks with
 * fewer than min_obs days (the paper: two months of history), irregular
 * stocks, and stocks whose Gram matrix is not positive definite are not
 * estimated: beta = 0, D = NaN.
 *   F       : device, count x T x p float32, row k = f_k.
 *   R       : device, count x T x n float32 (row-major: day-major), NaN = no return.
 *   beta    : device, count x n x p float64 (output).
 *   sigma_f : device, count x p x p float64 (output).
 *   D       : device, count x n float64 (output).
 *   nobs    : device, count x n int32 or NULL: days with a return, -1 irregular,
 *             -2 singular Gram matrix (output).
 *   ws      : device workspace of ff_risk_workspace_size bytes, 256-byte aligned.
 * 1 <= p <= 8, 2 <= T <= 4096, n >= 1, 1 <= count <= 65535, min_obs >= 2;
 * otherwise FF_ERR_INVALID_ARG (0 from ff_risk_workspace_size), before
 * anything is enqueued.  Asynchronous on `stream`: four launches (the suffix
 * Gram tables and Sigma_f of every window, the inverse Gram matrix of every
 * first day, one pass over R, the per-stock solve and variance). */
size_t ff_risk_workspace_size(int count, int T, int n, int p);
int ff_risk_estimate(int count, int T, int n, int p, const float* F, const float* R, int min_obs, double* beta,
                     double* sigma_f, double* D, int32_t* nobs, void* ws, size_t ws_bytes, void* stream);
/* Description of the CUDA call behind the last FF_ERR_CUDA of ff_risk_estimate
 * on the calling host thread ("" if none). */
const char* ff_risk_last_error(void);

/* Description of the CUDA runtime call that made the last FF_ERR_CUDA return
 * on the calling host thread ("" if none); static thread-local storage. */
const char* ff_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int ff_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FLASHFOLIO_H */
