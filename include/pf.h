/*
 * pf.h - C ABI of the GB300 polynomial-filtered subspace extraction library
 * (libpf.so).
 *
 * The library computes, on one GPU, the hot path of the polynomial-filtered
 * proximal-gradient / ADMM framework of "Low-rank Matrix Optimization Using
 * Polynomial-filtered Subspace Extraction": a warm-started Chebyshev filter on
 * an n x p block (Sec. 2.1, Eqs. (cheb), (cheb-linear-map),
 * (subspace-update)), CholQR2 orthonormalisation, the Rayleigh-Ritz
 * projection with a p x p eigensolve (Sec. 2.2, Eq. (RR)), and the low-rank
 * prox reconstruction of PFPG (Eqs. (pfpg1)-(pfpg2)) and PFAM
 * (Eqs. (PFAM1)-(PFAM2)).
 *
 * Conventions shared by every call:
 *  - All array pointers are DEVICE pointers owned by the caller, unless a
 *    parameter says "host".  The library never frees caller memory.
 *  - A context owns only its workspace, allocated by pf_create; no call
 *    allocates device memory afterwards (pf_solve's CUDA graph is the one
 *    exception: it is instantiated once per context and problem shape).
 *  - Calls are asynchronous and ordered on the stream given to pf_create.
 *    Calls that return host values (pf_prox_step with a non-NULL info,
 *    pf_solve, pf_problem_init) synchronise that stream.
 *  - Dense blocks are row-major: element (i, j) of an n x p block U with
 *    leading dimension ldu >= p is U[i*ldu + j].  A dense symmetric n x n
 *    matrix A is row-major with lda >= n.
 *  - Errors are returned as pf_status and never abort.  A CUDA error is
 *    reported as PF_ERR_CUDA; the context must then be destroyed.  The text
 *    of the last error is available from pf_last_error.
 *  - p (the block width) is fixed per context, 1 <= p <= PF_MAX_P, and every
 *    call needs p <= n.
 *  - Symbols are plain C; no CUDA, C++ or PyTorch types appear here.  The
 *    stream is passed as an opaque pointer (a cudaStream_t value; NULL means
 *    the legacy default stream).
 */
#ifndef PF_H
#define PF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF_MAX_P 64
#define PF_MAX_ACCEL 6   /* largest extrapolation window l (Sec. 4.3) */

typedef struct pf_ctx pf_ctx;

typedef enum {
  PF_OK = 0,
  PF_ERR_INVALID_ARG = 1,      /* a size, pointer or option is out of range      */
  PF_ERR_OOM = 2,              /* workspace allocation failed in pf_create        */
  PF_ERR_CUDA = 3,             /* a CUDA call or kernel failed (context unusable) */
  PF_ERR_CHOL_BREAKDOWN = 4,   /* CholQR2 failed even with the shifted pass       */
  PF_ERR_NAN = 5,              /* a non-finite value reached the Ritz values      */
  PF_ERR_NOT_CONVERGED = 6,    /* pf_solve hit max_iter above its tolerance       */
  PF_ERR_DEVICE_TIMEOUT = 7,   /* a bounded device wait ran out                   */
  PF_ERR_UNSUPPORTED = 8       /* valid request this build does not implement     */
} pf_status;

/* Iteration-matrix kinds accepted by pf_filter / pf_rayleigh_ritz. */
typedef enum {
  PF_OP_DENSE = 0,           /* op(X) = A X, A dense symmetric FP64 n x n             */
  PF_OP_LOWRANK_SPARSE = 1   /* op(X) = Uf diag(lam) Uf^T X + sparse_scale S X + shift X */
} pf_op_kind;

typedef enum { PF_PREC_FP64 = 0, PF_PREC_TF32 = 1, PF_PREC_BF16 = 2 } pf_precision;

/* Arithmetic of the FP64 dense product A X (PF_OP_DENSE on the FP64 path). */
typedef enum {
  PF_DENSE_SLICED = 0,  /* error-free 8-bit digit planes of A (stored as bytes) and X
                         * (fp16), fp16 MMAs on the tensor cores (tcgen05), level
                         * sums exact in fp32, folded in int64: an
                         * FP64-accurate product (per entry within a few units of
                         * 2^-53 max|A_i.| max|X_.j| per term of the sum) -- default */
  PF_DENSE_FP64 = 1     /* FP64 fused multiply-adds on the CUDA cores            */
} pf_dense_product;

typedef enum {
  PF_PROBLEM_MAXCUT = 0,       /* max-cut SDP by PFAM (Sec. 2.3)                          */
  PF_PROBLEM_COMPLETION = 1,   /* PSD matrix completion by PFPG (Sec. 2.2)                */
  PF_PROBLEM_NCE = 2,          /* nearest correlation estimation, PFPG on the dual (Sec. 5.1) */
  PF_PROBLEM_SVT = 3,          /* nuclear-norm matrix completion, PFSVT (Sec. 5.2.1)        */
  PF_PROBLEM_NNLS = 4          /* nuclear-norm regularised least squares, PFNNLS (Sec. 5.2.2) */
} pf_problem_kind;

/* Solver options (Sec. 2.2-2.3 and Sec. 4: degree d, q, eta, block width p). */
typedef struct {
  int32_t p;            /* block width, 1..PF_MAX_P                                  */
  int32_t degree;       /* Chebyshev degree d >= 1 (Eq. (cheb))                       */
  int32_t degree_max;   /* upper degree for the adaptive low-precision ladder         */
  int32_t q;            /* filter applications before orth (q = 1 is the only value   */
                        /* this build accepts; Eqs. (pfpg2)/(PFAM2) allow 1..3)       */
  double eta;           /* interval parameter of Sec. 4.1 (0 < eta < 1), e.g. 0.1    */
  int32_t precision;    /* pf_precision of the filter products                       */
  int32_t adaptive;     /* nonzero: raise precision, then degree, when the KKT stalls  */
  /* Block width rule (Sec. 4.2), FP64 contexts: with adapt_guard > 0, after
   * every adapt_every-th step of a problem its active width becomes
   * min(p, max(p_min, r_+ + adapt_guard)) rounded up to a multiple of 8,
   * r_+ the positive Ritz count of that step (p above is the maximum and
   * sizes the workspace).  Shrinking drops trailing Ritz columns (their
   * Ritz values are <= 0); growing takes the problem's guard columns of the
   * same index.  0 disables the rule.                                       */
  int32_t p_min;
  int32_t adapt_guard;
  int32_t adapt_every;
  /* pf_dense_product of the FP64 dense products.  The sliced product keeps
   * digit planes of A (7 byte planes, 7 bytes per entry of an
   * n_max x n_max matrix) in device memory allocated by the context on the
   * first dense call outside a stream capture, and freed by pf_destroy.  */
  int32_t dense_product;
} pf_options;

/*
 * Iteration matrix descriptor (all pointers device, caller-owned, read only).
 * PF_OP_DENSE:          A (n x n, row-major, lda), symmetric.  Optional
 *                       low-precision shadow A_lp (bf16 or fp32 per the
 *                       context precision) holding A / lp_scale, lda_lp.
 * PF_OP_LOWRANK_SPARSE: op(X) = Uf diag(lam) Uf^T X + sparse_scale * S X
 *                       + shift * X, with Uf n x r (row-major, lduf), lam r
 *                       values (r <= PF_MAX_P), and S a symmetric CSR matrix
 *                       (rowptr n+1 int32, colind nnz int32 sorted per row,
 *                       vals nnz FP64).
 */
typedef struct {
  int32_t kind;
  int64_t n;
  const double *A; int64_t lda;
  const void *A_lp; int64_t lda_lp; double lp_scale;
  const double *Uf; int64_t lduf; const double *lam; int32_t r;
  const int32_t *rowptr; const int32_t *colind; const double *vals; int64_t nnz;
  double sparse_scale; double shift;
} pf_operator;

/*
 * Problem state for pf_prox_step / pf_solve.  Data (read only):
 *  MAXCUT:      C = -L/4 as a symmetric CSR with its diagonal (vals_f64).
 *  COMPLETION:  the sampled entries of M on Omega as a symmetric CSR
 *               (vals_f32); mu > 0; t the step size.
 * Resident state (read and written by every step; device, caller-owned):
 *  U     n x p block (ldu), the warm start of the filter (after each step
 *        the Ritz basis V, the output U <- QV of the commented CheSE
 *        algorithm of Sec. 2.1).  On entry to
 *        pf_problem_init it holds the start block (any full-rank n x p).
 *  V     n x p Ritz vectors of the last Rayleigh-Ritz step (ldv); with theta
 *        they hold the low-rank iterate X = V diag(max(theta,0)) V^T.
 *  theta p Ritz values of the last step, descending.
 *  Z     MAXCUT only: dense FP64 n x n iteration matrix (ldz).  NULL selects
 *        the structured operator Z = X~ - tC - Diag(lam), applied without
 *        forming Z (C must then store every diagonal entry, zeros included).
 *  Z_lp  MAXCUT with a bf16 / tf32 context: the dense low-precision shadow
 *        Z / s (n x n, ldz_lp elements, 16-byte aligned row pitch) that the
 *        tensor-core filter reads; the Rayleigh-Ritz step then uses the
 *        structured FP64 operator, so Z may be NULL.
 *  Z_tf32  MAXCUT with a bf16 context (optional): an fp32 n x n buffer
 *        (ldz_tf32 elements, 16-byte aligned row pitch).  When given,
 *        pf_solve's adaptive ladder (options.adaptive) has three rungs: the
 *        bf16 filter, raised in degree up to degree_max while the KKT
 *        residual stalls; then the tf32 filter on the fp32 shadow Z / s kept
 *        in this buffer; then the FP64 structured filter.  Without it the
 *        ladder goes from bf16 to FP64.
 *  lam   MAXCUT only: n-vector lambda of the last DRS update.
 *  S     nnz FP64 workspace: COMPLETION P_Omega(X - M); structured MAXCUT
 *        the sparse part -tC - Diag(lam).
 * NCE (min 1/2||G - X||^2 s.t. diag X = 1, X psd, solved on its dual
 *  F(x) = 1/2||P_+(G + Diag x)||^2 - 1^T x by the filtered gradient method):
 *  Z holds G (dense FP64, ldz) on entry to pf_problem_init and G + Diag(x)
 *  afterwards; lam is the dual vector x (n); no CSR data; t is the gradient
 *  step (t <= 0 selects 1); the report's kkt is ||grad F(x_k)|| /
 *  ||grad F(x_0)|| and obj is F(x_k).
 *  Extrapolation (Sec. 4.3, regularized nonlinear acceleration): with
 *  1 <= accel_l <= PF_MAX_ACCEL and hist an (accel_l + 2) x n FP64 device
 *  buffer (row i holds iterate x_i of the current window, caller-owned,
 *  contents managed by the library), every accel_l + 1 steps the window
 *  x_0..x_{l+1} is replaced by x = sum_i c_i x_i, c = (D^T D + lam I)^{-1} 1
 *  normalised to sum 1, D = [x_1 - x_0, ..., x_{l+1} - x_l], lam =
 *  accel_lam * tr(D^T D) (accel_lam <= 0 selects 1e-10), and the iteration
 *  continues from x.  accel_l = 0 (or hist NULL) disables it.  If the small
 *  system has a non-positive pivot the window restarts from the current
 *  iterate instead.  Ignored by the other kinds.
 * SVT (min ||X||_* + 1/(2 mu)||X||_F^2 s.t. P_Omega(X) = P_Omega(M), by the
 *  SVT iteration W = shrink_mu(A*(x)), x <- x + t (b - A(W)) with the
 *  singular pairs of Y = A*(x) from a subspace filtered on Y^T Y):
 *  rowptr/colind/vals_f64 hold M on Omega (row-major CSR of the n x n
 *  matrix), t_rowptr/t_colind/t_perm the CSR of the transposed pattern and
 *  the map from its entries to the row-major ones; t is the step, mu the
 *  threshold; S (nnz) holds the dual x, set to t P_Omega(M) by
 *  pf_problem_init (the first iteration from x = 0); theta holds the Ritz
 *  values of Y^T Y (sigma^2) and V the right singular vectors.  The report's
 *  kkt is ||P_Omega(W - M)||_F / ||P_Omega(M)||_F, obj the dual F(x), r_plus
 *  the number of singular values above mu, pinf ||P_Omega(W - M)||_F.
 * NNLS (min mu ||X||_* + 1/2 ||P_Omega(X) - P_Omega(M)||_F^2 by accelerated
 *  proximal gradient with continuation mu_{k+1} = max(0.7 mu_k, mu_bar); the
 *  singular pairs of G = (1+beta) X^k - beta X^{k-1} - A*(A(Y) - b) come from
 *  a subspace filtered on G^T G): the data fields as for SVT; t = mu_0
 *  (t <= 0 selects 0.1 sqrt(||P_Omega M||_1 ||P_Omega M||_inf)); mu is
 *  mu_bar / mu_0; S (nnz) holds the residual A(Y) - b; fac (n x 4p, ldfac >=
 *  4p) holds [L | Lp | R | Rp], the orthonormal factors of X^k = L diag(s)
 *  R^T and of X^{k-1}; fsv (2p) holds [s | sp]; at most rank_cap pairs are
 *  kept (0 selects p - 8); p <= 32.  The report's kkt is
 *  ||X^{k+1} - X^k||_F / max(1, ||X^{k+1}||_F) once mu has reached mu_bar
 *  (at least 1 before), obj is mu ||X^k||_* + 1/2 ||A(X^k) - b||^2, r_plus
 *  the rank of X^{k+1}, dinf the step's mu.
 * COMPLETION, optional t_perm (nnz int32, device): for a symmetric sampling
 *  pattern (j in row i iff i in row j), the index of each entry's transposed
 *  entry.  The sampled residual S = P_Omega(X - M) is then formed on the
 *  entries with j >= i only and written to both places (X and M symmetric:
 *  half the dot products).  pf_problem_init checks the map on the device and
 *  returns PF_ERR_INVALID_ARG if some entry (i, j) does not map to (j, i).
 *  NULL forms every entry.
 * t: MAXCUT step; if t <= 0 on entry to pf_problem_init it is set to
 *    10 sqrt(n)/||C||_F.  COMPLETION step (t = 1 matches the Lipschitz
 *    constant of P_Omega).
 */
typedef struct {
  int32_t kind;
  int64_t n;
  const int32_t *rowptr; const int32_t *colind;
  const double *vals_f64; const float *vals_f32; int64_t nnz;
  double t; double mu;
  double *U; int64_t ldu;
  double *V; int64_t ldv;
  double *theta;
  double *Z; int64_t ldz;
  void *Z_lp; int64_t ldz_lp;
  double *lam;
  double *S;
  int64_t iter;          /* host-side counter, advanced by each step */
  int32_t accel_l;       /* NCE extrapolation window l (0 = off)     */
  double accel_lam;      /* NCE extrapolation regulariser (relative) */
  double *hist;          /* NCE (accel_l + 2) x n window of iterates  */
  int32_t p_active;      /* active block width; 0 on entry to pf_problem_init selects p;
                            maintained by the library under the width rule */
  const double *guard;   /* n x p random columns for width growth (ldg), read only */
  int64_t ldg;
  const int32_t *t_rowptr; const int32_t *t_colind; const int32_t *t_perm;  /* SVT, NNLS;
                            COMPLETION: t_perm optional, see below */
  double *fac; int64_t ldfac; double *fsv; int32_t rank_cap;                /* NNLS */
  void *Z_tf32; int64_t ldz_tf32;  /* MAXCUT, bf16 context, optional: fp32 shadow for the tf32 rung */
} pf_problem;

/* Per-step report (host struct).  MAXCUT: obj = <C, X~>, pinf/dinf/gap as in
 * the standard SDP report of Sec. 5.4; COMPLETION: obj = 1/2||P_Omega(X-M)||^2
 * + mu tr X and kkt the relative fixed-point residual; pinf/dinf/gap are 0. */
typedef struct {
  double a, b;               /* filter interval used by the step (Sec. 4.1) */
  double obj, kkt, pinf, dinf, gap;
  double theta_max, theta_min;
  int32_t r_plus;            /* number of positive Ritz values               */
  int32_t flags;             /* bit 0: shifted CholQR pass used; bit 1: Cholesky
                                breakdown; bit 2: non-finite Ritz value; bit 3:
                                a bounded device wait ran out; bit 4: the block
                                is saturated, r_plus >= p - 2 on each of the
                                last 20 steps (p too small for the solution
                                rank, Sec. 4.2)                                 */
  int32_t degree;            /* degree used by the step                      */
  int32_t precision;         /* precision used by the step                   */
  int32_t jacobi_sweeps;     /* sweeps of the p x p eigensolve of the step   */
  int32_t reserved;
} pf_iter_info;

typedef struct {
  int64_t iters;
  double kkt, obj;
  pf_iter_info last;
} pf_result;

/* Create a context for problems of size n <= n_max with the given options.
 * Allocates all workspace.  stream: cudaStream_t (opaque).  out: host. */
pf_status pf_create(const pf_options *opt, int64_t n_max, void *stream, pf_ctx **out);

/* Release the context and its workspace (after synchronising its stream). */
pf_status pf_destroy(pf_ctx *ctx);

/* U <- orth(rho(op) U) with rho(t) = T_d((t - (a+b)/2)/((b-a)/2)),
 * Sec. 2.1 Eqs. (cheb), (cheb-linear-map), (subspace-update); orth is
 * CholQR2 (QR with positive diagonal R).  a < b host scalars, degree >= 1,
 * U n x p device (ldu >= p), overwritten in place. */
pf_status pf_filter(pf_ctx *ctx, const pf_operator *op, double a, double b, int32_t degree,
                    double *U, int64_t ldu);

/* Rayleigh-Ritz on span(Q), Sec. 2.2 Eq. (RR): H = Q^T op(Q), H = Y Theta Y^T,
 * V = Q Y.  Q n x p orthonormal (ldq), V n x p out (ldv), theta p out
 * (descending), resid p out (||op(v_i) - theta_i v_i||_2); resid may be NULL. */
pf_status pf_rayleigh_ritz(pf_ctx *ctx, const pf_operator *op, const double *Q, int64_t ldq,
                           double *V, int64_t ldv, double *theta, double *resid);

/* Y = op(X): one product of the iteration matrix with an n x p block, the
 * building block of the Chebyshev recurrence of Sec. 2.1 (Eq. (cheb)).
 * X, Y device n x p (ldx, ldy >= p), distinct.  Asynchronous. */
pf_status pf_apply(pf_ctx *ctx, const pf_operator *op, const double *X, int64_t ldx, double *Y,
                   int64_t ldy);

/* Prepare the resident state of a problem: MAXCUT sets Z = Z^1 = I - t offdiag(C)
 * (the DRS image of Z^0 = 0), lam = -t diag(C) - 1, theta = 0; COMPLETION sets
 * theta = 0 (X^0 = 0).  Computes t for MAXCUT when t <= 0.  Synchronises. */
pf_status pf_problem_init(pf_ctx *ctx, pf_problem *prob);

/* One PFAM (MAXCUT, Eqs. (PFAM1)-(PFAM2)) or PFPG (COMPLETION,
 * Eqs. (pfpg1)-(pfpg2)) iteration: interval, filter, CholQR2, Rayleigh-Ritz,
 * prox/DRS update, KKT.  info (host) may be NULL; when given, the call
 * synchronises and fills it. */
pf_status pf_prox_step(pf_ctx *ctx, pf_problem *prob, pf_iter_info *info);

/* Iterate pf_prox_step until kkt <= tol (checked every check_every steps,
 * tol <= 0 disables the test) or max_iter steps.  The step is captured once
 * in a CUDA graph and replayed.  An adaptive context feeds every check to
 * the ladder (pf_ladder_update).  out (host) receives the final report.
 * Returns PF_ERR_NOT_CONVERGED if tol > 0 was not reached. */
pf_status pf_solve(pf_ctx *ctx, pf_problem *prob, int64_t max_iter, double tol,
                   int32_t check_every, pf_result *out);

/* Copy the report of the most recent step to host (synchronises). */
pf_status pf_get_info(pf_ctx *ctx, pf_iter_info *info);

/* Enqueue n_steps iterations of pf_prox_step (replays of the step's CUDA
 * graph when the stream is not the legacy default stream) and return without
 * synchronising.  The adaptive ladder is applied only through
 * pf_ladder_update.  Used by request loops that keep several solves in
 * flight on different streams. */
pf_status pf_enqueue_steps(pf_ctx *ctx, pf_problem *prob, int64_t n_steps);

/* Feed the KKT residual of a check (e.g. from a pf_report_async report) to
 * the adaptive ladder of an adaptive context (options.adaptive != 0; a no-op
 * otherwise), as pf_solve does at each of its checks.  The ladder has
 * stalled when the best of the last 5 checks is not 5% below the best of the
 * 5 checks before; a stall moves a low-precision filter up one precision
 * (bf16 -> tf32 when the problem carries Z_tf32 -> FP64), and in FP64 raises
 * the degree by one up to degree_max.  The ladder's state belongs to the
 * context and restarts at pf_problem_init.  May enqueue the tf32 shadow's
 * fill on the context's stream. */
pf_status pf_ladder_update(pf_ctx *ctx, pf_problem *prob, double kkt);

/* Enqueue a copy of the latest step report into `info` (host memory owned
 * by the caller; page-locked memory keeps the copy asynchronous).  The
 * report is valid once the context's stream has reached this point (e.g.
 * after an event recorded behind it has completed). */
pf_status pf_report_async(pf_ctx *ctx, pf_iter_info *info);

/* Y = A X for a dense symmetric FP64 A (n x n, row-major, lda >= n) and an
 * n x p block X (ldx >= p, 1 <= p <= PF_MAX_P), written to Y (ldy >= p,
 * distinct from X), enqueued on `stream` (a cudaStream_t; NULL = legacy
 * default stream).  No counterpart in the paper: it is pf_apply's dense FP64
 * product for callers that cannot allocate device memory -- code that has no
 * pf_ctx to own a workspace, or that runs under a memory manager which owns
 * all device memory, or on a path that must not pay for cudaMalloc (which
 * may synchronise the device).  It allocates nothing: the split-K partial
 * sums live in one fixed device array inside the library of
 * 2 Mi doubles (16 MiB), which every GPU that loads the library keeps until
 * the process exits; calls need n * p <= 2,097,152 (PF_ERR_INVALID_ARG
 * otherwise).  Every call looks up that array's device address for the
 * current device (so the address stays right after cudaDeviceReset); the
 * first call on each device may load the library's device code and should
 * come before any stream capture.  All calls share the array: calls whose
 * kernels can overlap on a GPU (different streams without ordering) race and
 * must be serialised by the caller.  Nothing in the array needs to start at
 * zero (every partial sum a call reads it has written itself).  A CUDA error
 * already pending when the call starts is left in place and reported as
 * PF_ERR_CUDA with nothing launched.  Errors: PF_ERR_INVALID_ARG,
 * PF_ERR_CUDA, PF_ERR_UNSUPPORTED (device index >= 64). */
pf_status pf_apply_dense_noalloc(const double *A, int64_t lda, const double *X, int64_t ldx,
                                 double *Y, int64_t ldy, int64_t n, int32_t p, void *stream);

/* Phases of a step, in the paper's terms: the interval [a, b] (Sec. 4.1),
 * the Chebyshev filter products (Sec. 2.1, Eq. (cheb)), orth by CholQR2
 * (Eq. (subspace-update)), the Rayleigh-Ritz product and projected matrix
 * (Sec. 2.2, Eq. (RR)), the p x p eigensolve with the Ritz vectors, and the
 * update (prox / DRS step, reconstruction and KKT report; for completion also
 * the sampled residual that starts a step). */
#define PF_NUM_PHASES 6
typedef enum {
  PF_PHASE_INTERVAL = 0,
  PF_PHASE_FILTER = 1,
  PF_PHASE_ORTH = 2,
  PF_PHASE_RR = 3,
  PF_PHASE_EIG = 4,
  PF_PHASE_UPDATE = 5
} pf_phase;

/* Phase tracing (instrumentation with no counterpart in the paper).  Every
 * call that enqueues a step, a filter or a Rayleigh-Ritz projection opens an
 * NVTX range named "pf:<phase>" per phase (host-side, always on; visible to
 * Nsight tools).  With tracing on (on != 0; creates CUDA events, allocates no
 * device memory), such calls enqueued outside a stream capture also record an
 * event at each phase boundary; pf_phase_times then waits for the most recent
 * traced call and writes the device time of each phase to ms (host,
 * PF_NUM_PHASES doubles, milliseconds; zeros when nothing was traced).  Steps
 * replayed from pf_solve's CUDA graph are not traced. */
pf_status pf_set_tracing(pf_ctx *ctx, int32_t on);
pf_status pf_phase_times(pf_ctx *ctx, double *ms);

/* Limit, in nanoseconds of the GPU's global timer, of each bounded wait in
 * the tensor-core pipelines (TMA and MMA stages); 2 s by default.  A wait that
 * runs out makes its kernel stop its pipeline, let the copies and MMAs it has
 * already issued land (with a separate fixed limit), free its tensor memory,
 * and set flags bit 3 of the step report, which pf_prox_step / pf_solve
 * return as PF_ERR_DEVICE_TIMEOUT; the results of that step are then invalid
 * but the context stays usable.  0 gives up on the first wait that is not
 * already satisfied (for tests of that path).  Applies to the current device,
 * is synchronous, and must not be called while this library's kernels run
 * or during a stream capture.  No counterpart in the paper. */
pf_status pf_set_wait_limit(uint64_t ns);

/* Number of kernels this library has enqueued in this process (host-side
 * count; a replayed CUDA graph adds nothing).  Instrumentation with no
 * counterpart in the paper: it lets a caller count the GPU launches of a
 * step by differencing around a non-graph call. */
int64_t pf_kernel_launch_count(void);

const char *pf_status_string(pf_status s);
const char *pf_last_error(const pf_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
