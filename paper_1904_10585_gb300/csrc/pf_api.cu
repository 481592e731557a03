// C ABI of libpf: context and workspace management, the filter and
// Rayleigh-Ritz entry points, the PFAM / PFPG steps and the graph-captured
// solve loop.  Every step of the path is a kernel launched on the context's
// stream; the host only validates arguments, enqueues and (where a call
// returns host values) synchronises.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "pf_internal.cuh"

using namespace pf;

namespace pf {
std::atomic<int64_t> g_launches{0};
}

// phase boundaries kept per traced call (a step marks at most about 8)
constexpr int kTraceMarks = 32;

struct pf_ctx {
  pf_options opt;
  int64_t n_max;
  int p;
  cudaStream_t stream;
  Workspace ws;
  void *base;
  size_t bytes;
  char err[512];
  // graph of one step, cached per problem description and ladder state
  cudaGraphExec_t gexec;
  pf_problem gkey;
  int gdegree;
  int gprec;
  int gp;
  bool have_graph;
  // adaptive ladder state: degree and filter precision (pf_precision)
  // currently used
  int cur_degree;
  int cur_prec;
  // KKT residuals at the last (up to kLadderWin) checks of the ladder; kept
  // across calls so that a solve run in pieces climbs the same ladder
  double ladder_hist[10];
  int ladder_n;
  // digit planes of the sliced dense product (allocated on first use) and
  // the matrix (pointer, n) they currently hold, nullptr when unknown
  void *oz_base;
  const void *oz_owner;
  int64_t oz_owner_n;
  // the sliced dense max-cut problem (its lam) whose interval row bounds the
  // interval slot holds, nullptr when unknown: each step of that problem
  // leaves them for the next step
  const void *ivl_owner;
  // phase tracing (pf_set_tracing): an event at each phase boundary of the
  // most recent call enqueued outside a stream capture
  bool trace;
  bool nvtx_open;
  int nmarks;
  int tmark[kTraceMarks];
  cudaEvent_t tev[kTraceMarks + 1];
};

namespace {

bool width_rule_on(const pf_ctx *ctx) { return ctx->opt.adapt_guard > 0; }

// The filter currently runs on a low-precision shadow (bf16 or tf32).
bool cur_lp(const pf_ctx *ctx) { return ctx->cur_prec != PF_PREC_FP64; }

// Active block width of a problem (validated by check_problem).
int active_width(const pf_ctx *ctx, const pf_problem *pr) {
  return pr->p_active > 0 ? pr->p_active : ctx->p;
}

// The FP64 dense product of this operator runs on the tensor cores as bf16
// digit planes (pf_oz.cu).
bool sliced(const pf_ctx *ctx, const Op &op) {
  return op.kind == PF_OP_DENSE && op.A != nullptr &&
         ctx->opt.dense_product == PF_DENSE_SLICED;
}

// Dense max-cut whose update runs on the tensor cores and leaves the digit
// planes of the new Z for the next step.
bool sliced_maxcut(const pf_ctx *ctx, const pf_problem *pr) {
  return pr->kind == PF_PROBLEM_MAXCUT && pr->Z != nullptr &&
         ctx->opt.precision == PF_PREC_FP64 && ctx->opt.dense_product == PF_DENSE_SLICED;
}

// Problems whose digit planes stay with the problem between steps: the
// sliced dense max-cut (its expansion writes the planes of the next Z) and
// the sliced NCE (its steps change only the diagonal of Z, whose chunks each
// step slices again).
bool planes_kept(const pf_ctx *ctx, const pf_problem *pr) {
  return sliced_maxcut(ctx, pr) ||
         (pr->kind == PF_PROBLEM_NCE && ctx->opt.dense_product == PF_DENSE_SLICED &&
          ctx->opt.precision == PF_PREC_FP64);
}

// Problems whose steps apply a dense FP64 iteration matrix.
bool dense_f64_problem(const pf_ctx *ctx, const pf_problem *pr) {
  return pr->kind == PF_PROBLEM_NCE ||
         (pr->kind == PF_PROBLEM_MAXCUT && pr->Z != nullptr &&
          ctx->opt.precision == PF_PREC_FP64);
}

pf_status set_err(pf_ctx *ctx, pf_status s, const char *fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

#define PF_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return set_err(ctx, PF_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                     __LINE__);                                                                  \
  } while (0)

#define PF_TRY(expr)                  \
  do {                                \
    pf_status s_ = (expr);            \
    if (s_ != PF_OK) return s_;       \
  } while (0)

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------------------
// Phase tracing: an NVTX range per phase of a call (always), and, when
// tracing is on and the stream is not being captured, a timing event at each
// phase boundary (pf_phase_times turns them into milliseconds per phase).
// ---------------------------------------------------------------------------
const char *const kPhaseName[PF_NUM_PHASES] = {"pf:interval", "pf:filter", "pf:orth",
                                               "pf:rayleigh_ritz", "pf:eigensolve", "pf:update"};

bool capturing(const pf_ctx *ctx) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &st) != cudaSuccess) return true;
  return st != cudaStreamCaptureStatusNone;
}

void trace_begin(pf_ctx *ctx) {
  if (ctx->nvtx_open) {
    nvtxRangePop();
    ctx->nvtx_open = false;
  }
  if (ctx->trace && !capturing(ctx)) ctx->nmarks = 0;
}

void phase(pf_ctx *ctx, int ph) {
  if (ctx->nvtx_open) nvtxRangePop();
  nvtxRangePushA(kPhaseName[ph]);
  ctx->nvtx_open = true;
  if (ctx->trace && ctx->nmarks < kTraceMarks && !capturing(ctx)) {
    if (cudaEventRecord(ctx->tev[ctx->nmarks], ctx->stream) == cudaSuccess)
      ctx->tmark[ctx->nmarks++] = ph;
  }
}

void trace_end(pf_ctx *ctx) {
  if (ctx->nvtx_open) {
    nvtxRangePop();
    ctx->nvtx_open = false;
  }
  if (ctx->trace && ctx->nmarks > 0 && !capturing(ctx) &&
      cudaEventRecord(ctx->tev[ctx->nmarks], ctx->stream) != cudaSuccess)
    ctx->nmarks = 0;
}


// Digit-plane buffers of the sliced dense product, sized for n_max and the
// context's p; allocated once, outside any stream capture.
pf_status ensure_oz(pf_ctx *ctx) {
  if (ctx->oz_base != nullptr || ctx->opt.dense_product != PF_DENSE_SLICED) return PF_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  PF_CUDA(cudaStreamIsCapturing(ctx->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone)
    return set_err(ctx, PF_ERR_UNSUPPORTED,
                   "the sliced dense product allocates its digit planes on the first dense call, "
                   "which must not be inside a stream capture");
  const int64_t nz = ((ctx->n_max + 127) / 128) * 128;
  const int64_t chunks = nz / 128;
  int smax = kOzMaxSplits;
  const int need = (int)((chunks + kOzMaxChunks - 1) / kOzMaxChunks);
  if (need > smax) smax = need;
  const size_t sizes[] = {(size_t)kOzSlices * nz * nz,                     // zs (one byte a digit)
                          (size_t)nz * chunks * sizeof(int),               // ez
                          (size_t)kOzSlices * kMaxP * nz * 2,              // xs[0]
                          (size_t)kOzSlices * kMaxP * nz * 2,              // xs[1]
                          (size_t)chunks * kMaxP * sizeof(int),            // ex[0]
                          (size_t)chunks * kMaxP * sizeof(int),            // ex[1]
                          (size_t)smax * ctx->n_max * ctx->p * sizeof(double),  // part
                          (size_t)chunks * 2 * sizeof(int),                // cnt
                          (size_t)kOzSlices * nz * 64 * 2,                 // wp
                          (size_t)kOzSlices * nz * 64 * 2,                 // vp
                          (size_t)nz * sizeof(int),                        // ew
                          (size_t)nz * sizeof(int),                        // ev
                          (size_t)nz * sizeof(double),                     // xdiag
                          (size_t)chunks * sizeof(double),                 // mchunk
                          (size_t)nz * sizeof(double),                     // cdiag
                          (size_t)nz * sizeof(double)};                    // crsum
  constexpr int nbuf = 16;
  size_t off[nbuf], tot = 0;
  for (int i = 0; i < nbuf; ++i) {
    off[i] = tot;
    tot += align_up(sizes[i]);
  }
  void *base = nullptr;
  if (cudaMalloc(&base, tot) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, PF_ERR_OOM, "digit planes of the sliced dense product (%zu bytes)", tot);
  }
  if (cudaMemsetAsync(base, 0, tot, ctx->stream) != cudaSuccess) {
    cudaFree(base);
    return set_err(ctx, PF_ERR_CUDA, "clearing the digit planes failed");
  }
  char *b = (char *)base;
  OzBuffers &oz = ctx->ws.oz;
  oz.zs = b + off[0];
  oz.ez = (int *)(b + off[1]);
  oz.xs[0] = b + off[2];
  oz.xs[1] = b + off[3];
  oz.ex[0] = (int *)(b + off[4]);
  oz.ex[1] = (int *)(b + off[5]);
  oz.part = (double *)(b + off[6]);
  oz.cnt = (int *)(b + off[7]);
  oz.wp = b + off[8];
  oz.vp = b + off[9];
  oz.ew = (int *)(b + off[10]);
  oz.ev = (int *)(b + off[11]);
  oz.xdiag = (double *)(b + off[12]);
  oz.mchunk = (double *)(b + off[13]);
  oz.cdiag = (double *)(b + off[14]);
  oz.crsum = (double *)(b + off[15]);
  oz.ldk = nz;
  oz.slice_rows = nz;
  ctx->oz_base = base;
  return PF_OK;
}

// Before steps of a problem: the digit-plane buffers, and for a sliced dense
// max-cut or NCE the planes of its current Z (sliced here, outside any
// capture, unless they already hold it).
pf_status oz_prepare_problem(pf_ctx *ctx, const pf_problem *pr) {
  const bool ivl_kept = sliced_maxcut(ctx, pr) && pr->Z != nullptr;
  if (!ivl_kept) ctx->ivl_owner = nullptr;
  if (!dense_f64_problem(ctx, pr)) return PF_OK;
  PF_TRY(ensure_oz(ctx));
  if (planes_kept(ctx, pr) && (ctx->oz_owner != pr->Z || ctx->oz_owner_n != pr->n)) {
    PF_CUDA(launch_oz_zslice(ctx->stream, ctx->ws, pr->Z, pr->ldz, (int)pr->n));
    ctx->oz_owner = pr->Z;
    ctx->oz_owner_n = pr->n;
  }
  if (ivl_kept && ctx->ivl_owner != pr->lam) {
    // C's diagonal and row sums, and the first step's interval row bounds;
    // from then on every step leaves the next step's bounds
    PF_CUDA(launch_maxcut_cdata(ctx->stream, ctx->ws, pr->rowptr, pr->colind, pr->vals_f64,
                                (int)pr->n));
    PF_CUDA(launch_interval_rows(ctx->stream, ctx->ws, pr->rowptr, pr->colind, pr->vals_f64,
                                 (int)pr->n, pr->lam));
    ctx->ivl_owner = pr->lam;
  }
  return PF_OK;
}

// After steps: the planes hold the problem's Z only for the sliced max-cut
// and NCE.
void oz_after_steps(pf_ctx *ctx, const pf_problem *pr) {
  if (!dense_f64_problem(ctx, pr)) return;
  if (planes_kept(ctx, pr)) {
    ctx->oz_owner = pr->Z;
    ctx->oz_owner_n = pr->n;
  } else {
    ctx->oz_owner = nullptr;
  }
}

pf_status make_op(pf_ctx *ctx, const pf_operator *op, Op *out) {
  if (!op) return set_err(ctx, PF_ERR_INVALID_ARG, "operator is NULL");
  if (op->n < ctx->p || op->n > ctx->n_max)
    return set_err(ctx, PF_ERR_INVALID_ARG, "operator n=%lld outside [p=%d, n_max=%lld]",
                   (long long)op->n, ctx->p, (long long)ctx->n_max);
  Op o = {};
  o.kind = op->kind;
  o.n = (int)op->n;
  if (op->kind == PF_OP_DENSE) {
    const bool lp = ctx->opt.precision != PF_PREC_FP64;
    if (!lp && (!op->A || op->lda < op->n))
      return set_err(ctx, PF_ERR_INVALID_ARG, "dense operator needs A and lda >= n");
    if (lp) {
      const int esz = ctx->opt.precision == PF_PREC_TF32 ? 4 : 2;
      if (!op->A_lp || op->lda_lp < op->n || (op->lda_lp * esz) % 16 != 0 ||
          ((uintptr_t)op->A_lp & 15) != 0 || !(op->lp_scale > 0.0))
        return set_err(ctx, PF_ERR_INVALID_ARG,
                       "low-precision dense operator needs A_lp 16-byte aligned, lda_lp >= n with "
                       "a 16-byte row pitch, and lp_scale > 0");
    }
    o.A = op->A;
    o.lda = op->lda;
    o.A_lp = op->A_lp;
    o.lda_lp = op->lda_lp;
    o.lp_scale = op->lp_scale;
  } else if (op->kind == PF_OP_LOWRANK_SPARSE) {
    if (op->r < 0 || op->r > kMaxP)
      return set_err(ctx, PF_ERR_INVALID_ARG, "low-rank width r=%d outside [0, %d]", op->r, kMaxP);
    if (op->r > 0 && (!op->Uf || !op->lam || op->lduf < op->r))
      return set_err(ctx, PF_ERR_INVALID_ARG, "low-rank part needs Uf, lam and lduf >= r");
    if (op->nnz > 0 && (!op->rowptr || !op->colind || !op->vals))
      return set_err(ctx, PF_ERR_INVALID_ARG, "sparse part needs rowptr, colind and vals");
    if (op->nnz < 0 || op->nnz > INT32_MAX)
      return set_err(ctx, PF_ERR_INVALID_ARG, "nnz out of range");
    o.Uf = op->Uf;
    o.lduf = op->lduf;
    o.lam = op->lam;
    o.r = op->r;
    o.clamp = 0;
    o.rowptr = op->rowptr;
    o.colind = op->colind;
    o.vals = op->nnz > 0 ? op->vals : nullptr;
    o.sscale = op->sparse_scale;
    o.shift = op->shift;
    if (op->nnz == 0 && op->rowptr == nullptr) {
      o.vals = nullptr;  // pure low-rank + shift operator
    }
  } else {
    return set_err(ctx, PF_ERR_INVALID_ARG, "unknown operator kind %d", op->kind);
  }
  *out = o;
  return PF_OK;
}

pf_status apply(pf_ctx *ctx, const Op &op, const double *X, int64_t ldx, const double *Yprev,
                int64_t ldp, double *Ynext, int64_t ldn, int mode) {
  if (op.kind == PF_OP_DENSE)
    PF_CUDA(launch_dense_apply(ctx->stream, ctx->ws, op, X, ldx, Yprev, ldp, Ynext, ldn, mode));
  else
    PF_CUDA(launch_lowrank_sparse_apply(ctx->stream, ctx->ws, op, X, ldx, Yprev, ldp, Ynext, ldn,
                                        mode));
  return PF_OK;
}

// Q = orth(Y) by CholQR2 (a third pass follows a shifted first pass).
pf_status cholqr2(pf_ctx *ctx, const double *Y, int64_t ldy, double *U, int64_t ldu, int n) {
  phase(ctx, PF_PHASE_ORTH);
  const int p = ctx->ws.p;  // active width
  cudaStream_t s = ctx->stream;
  const Workspace &ws = ctx->ws;
  int nb = 0;
  // symmetric Grams: the Cholesky factorisation reads the upper triangle only
  PF_CUDA(launch_gram(s, ws, Y, ldy, Y, ldy, n, p, p, 0, &nb, true));
  PF_CUDA(launch_chol_inv(s, ws, nb, n, p, 0));
  PF_CUDA(launch_apply_right(s, ws, Y, ldy, U, ldu, n, p, ws.Rinv, 1, 0));
  for (int pass = 1; pass <= 2; ++pass) {
    const int cond = pass == 2 ? 1 : 0;
    PF_CUDA(launch_gram(s, ws, U, ldu, U, ldu, n, p, p, cond, &nb, true));
    PF_CUDA(launch_chol_inv(s, ws, nb, n, p, pass));
    PF_CUDA(launch_apply_right(s, ws, U, ldu, U, ldu, n, p, ws.Rinv, 1, cond));
  }
  return PF_OK;
}

// Low-precision filter (tensor cores): fp32 recurrence, bf16/tf32 operands,
// then CholQR2 in FP64.
pf_status filter_core_lp(pf_ctx *ctx, const Op &op, double *U, int64_t ldu, int degree,
                         bool tf32) {
  const int p = ctx->ws.p;  // active width
  cudaStream_t s = ctx->stream;
  const Workspace &ws = ctx->ws;
  if (op.lp_scale > 0.0) PF_CUDA(launch_set_scale(s, ws.prm, op.lp_scale));
  PF_CUDA(launch_prep_lp(s, ws, tf32, U, ldu, op.n, ws.U32, ws.Xt[0]));
  for (int j = 0; j < degree; ++j) {
    const float *cur = j == 0 ? ws.U32 : ws.Y32[(j - 1) & 1];
    const float *prev = j == 1 ? ws.U32 : ws.Y32[j & 1];
    float *next = ws.Y32[j & 1];
    void *xt_next = (j + 1 < degree) ? ws.Xt[(j + 1) & 1] : nullptr;
    PF_CUDA(launch_tc_product(s, ws, tf32, op.A_lp, op.lda_lp, op.n, ws.Xt[j & 1], cur, prev,
                              next, xt_next, j == 0 ? MODE_FIRST : MODE_RECUR));
  }
  PF_CUDA(launch_f32_to_f64(s, ws, ws.Y32[(degree - 1) & 1], (int64_t)op.n * p, ws.Y[0]));
  return cholqr2(ctx, ws.Y[0], p, U, ldu, op.n);
}

// Low-precision context, low-rank + sparse operator: fp32 products on the
// CUDA cores, fp32 recurrence, then CholQR2 in FP64.
pf_status filter_core_lp_sparse(pf_ctx *ctx, const Op &op, double *U, int64_t ldu, int degree) {
  const int p = ctx->ws.p;  // active width
  cudaStream_t s = ctx->stream;
  const Workspace &ws = ctx->ws;
  const float *Uf32 = nullptr;
  if (op.r > 0 && op.Uf != nullptr) {
    PF_CUDA(launch_to_f32(s, ws, op.Uf, op.lduf, op.n, op.r, ws.Wf));
    Uf32 = ws.Wf;
  }
  PF_CUDA(launch_to_f32(s, ws, U, ldu, op.n, p, ws.U32));
  for (int j = 0; j < degree; ++j) {
    const float *cur = j == 0 ? ws.U32 : ws.Y32[(j - 1) & 1];
    const float *prev = j == 1 ? ws.U32 : ws.Y32[j & 1];
    float *next = ws.Y32[j & 1];
    PF_CUDA(launch_lowrank_sparse_apply32(s, ws, op, Uf32, cur, prev, next,
                                          j == 0 ? MODE_FIRST : MODE_RECUR));
  }
  PF_CUDA(launch_f32_to_f64(s, ws, ws.Y32[(degree - 1) & 1], (int64_t)op.n * p, ws.Y[0]));
  return cholqr2(ctx, ws.Y[0], p, U, ldu, op.n);
}

// U <- orth(rho(op) U) with the interval already in the device parameters.
pf_status filter_core(pf_ctx *ctx, const Op &op, double *U, int64_t ldu, int degree) {
  phase(ctx, PF_PHASE_FILTER);
  const int p = ctx->ws.p;  // active width
  if (op.kind == PF_OP_LOWRANK_SPARSE && cur_lp(ctx))
    return filter_core_lp_sparse(ctx, op, U, ldu, degree);
  if (op.kind == PF_OP_DENSE && op.A_lp != nullptr && ctx->opt.precision != PF_PREC_FP64)
    return filter_core_lp(ctx, op, U, ldu, degree, ctx->opt.precision == PF_PREC_TF32);
  double *const *Y = ctx->ws.Y;
  if (sliced(ctx, op)) {
    // digit planes of A (unless current), of U, then one tensor-core product
    // per degree, each cutting its output into the planes of the next
    cudaStream_t s = ctx->stream;
    const Workspace &ws = ctx->ws;
    if (!op.zs_ready) PF_CUDA(launch_oz_zslice(s, ws, op.A, op.lda, op.n));
    PF_CUDA(launch_oz_xslice(s, ws, U, ldu, op.n, 0));
    for (int j = 0; j < degree; ++j) {
      const double *cur = j == 0 ? U : Y[(j - 1) & 1];
      const int64_t ldc = j == 0 ? ldu : p;
      const double *prev = j == 0 ? nullptr : (j == 1 ? U : Y[j & 1]);
      const int64_t ldprev = j == 1 ? ldu : p;
      PF_CUDA(launch_oz_product(s, ws, op.n, j & 1, cur, ldc, prev, ldprev, Y[j & 1], p,
                                j + 1 < degree ? ((j + 1) & 1) : -1,
                                j == 0 ? MODE_FIRST : MODE_RECUR));
    }
    return cholqr2(ctx, Y[(degree - 1) & 1], p, U, ldu, op.n);
  }
  PF_TRY(apply(ctx, op, U, ldu, nullptr, 0, Y[0], p, MODE_FIRST));
  for (int j = 1; j < degree; ++j) {
    const double *cur = Y[(j - 1) & 1];
    const double *prev = (j == 1) ? U : Y[j & 1];
    const int64_t ldprev = (j == 1) ? ldu : p;
    PF_TRY(apply(ctx, op, cur, p, prev, ldprev, Y[j & 1], p, MODE_RECUR));
  }
  return cholqr2(ctx, Y[(degree - 1) & 1], p, U, ldu, op.n);
}

pf_status rr_core(pf_ctx *ctx, const Op &op, const double *Q, int64_t ldq, double *V, int64_t ldv,
                  double *theta, double *resid) {
  phase(ctx, PF_PHASE_RR);
  const int p = ctx->ws.p;  // active width
  cudaStream_t s = ctx->stream;
  const Workspace &ws = ctx->ws;
  if (sliced(ctx, op)) {
    if (!op.zs_ready) PF_CUDA(launch_oz_zslice(s, ws, op.A, op.lda, op.n));
    PF_CUDA(launch_oz_xslice(s, ws, Q, ldq, op.n, 0));
    PF_CUDA(launch_oz_product(s, ws, op.n, 0, Q, ldq, nullptr, 0, ws.W, p, -1, MODE_PLAIN));
  } else {
    PF_TRY(apply(ctx, op, Q, ldq, nullptr, 0, ws.W, p, MODE_PLAIN));
  }
  int nb = 0;
  PF_CUDA(launch_gram(s, ws, Q, ldq, ws.W, p, op.n, p, p, 0, &nb));
  // launch_gram leaves the reduced H = Q^T W in the first Gram slot
  phase(ctx, PF_PHASE_EIG);
  PF_CUDA(launch_jacobi(s, ws, ws.gpart, p, theta));
  if (resid != nullptr)
    PF_CUDA(launch_rotate_resid(s, ws, Q, ldq, ws.W, p, op.n, p, theta, V, ldv, resid));
  else  // Ritz vectors only (the solver steps do not use the residual norms)
    PF_CUDA(launch_apply_right(s, ws, Q, ldq, V, ldv, op.n, p, ws.Yeig, 0, 0));
  return PF_OK;
}

pf_status check_problem(pf_ctx *ctx, const pf_problem *pr) {
  if (!pr) return set_err(ctx, PF_ERR_INVALID_ARG, "problem is NULL");
  const int p = ctx->p;
  if (pr->n < p || pr->n > ctx->n_max)
    return set_err(ctx, PF_ERR_INVALID_ARG, "problem n=%lld outside [p=%d, n_max=%lld]",
                   (long long)pr->n, p, (long long)ctx->n_max);
  if (pr->p_active < 0 || pr->p_active > p)
    return set_err(ctx, PF_ERR_INVALID_ARG, "p_active=%d outside [0, p=%d]", pr->p_active, p);
  if (width_rule_on(ctx)) {
    if (ctx->opt.precision != PF_PREC_FP64)
      return set_err(ctx, PF_ERR_UNSUPPORTED, "the block width rule runs in an FP64 context");
    if (ctx->opt.p_min < 1 || ctx->opt.p_min > p || ctx->opt.adapt_every < 1)
      return set_err(ctx, PF_ERR_INVALID_ARG, "width rule needs 1 <= p_min <= p, adapt_every >= 1");
    if (!pr->guard || pr->ldg < p)
      return set_err(ctx, PF_ERR_INVALID_ARG, "width rule needs guard columns (ldg >= p)");
  }
  if (pr->kind != PF_PROBLEM_NCE &&
      (!pr->rowptr || !pr->colind || pr->nnz < 0 || pr->nnz > INT32_MAX))
    return set_err(ctx, PF_ERR_INVALID_ARG, "problem needs a CSR matrix (rowptr, colind, nnz)");
  if (!pr->U || pr->ldu < p || !pr->V || pr->ldv < p || !pr->theta)
    return set_err(ctx, PF_ERR_INVALID_ARG, "problem needs U, V (ld >= p) and theta");
  if (pr->kind == PF_PROBLEM_MAXCUT) {
    if (!pr->vals_f64) return set_err(ctx, PF_ERR_INVALID_ARG, "max-cut needs vals_f64 (C)");
    if (!pr->lam) return set_err(ctx, PF_ERR_INVALID_ARG, "max-cut needs lam");
    const bool lp = ctx->opt.precision != PF_PREC_FP64;
    if (lp) {
      const int esz = ctx->opt.precision == PF_PREC_TF32 ? 4 : 2;
      if (!pr->Z_lp || pr->ldz_lp < pr->n || (pr->ldz_lp * esz) % 16 != 0 ||
          ((uintptr_t)pr->Z_lp & 15) != 0)
        return set_err(ctx, PF_ERR_INVALID_ARG,
                       "low-precision max-cut needs Z_lp (16-byte aligned, ldz_lp >= n, 16-byte "
                       "row pitch)");
    }
    if (pr->Z_tf32 != nullptr &&
        (ctx->opt.precision != PF_PREC_BF16 || pr->ldz_tf32 < pr->n ||
         (pr->ldz_tf32 * 4) % 16 != 0 || ((uintptr_t)pr->Z_tf32 & 15) != 0))
      return set_err(ctx, PF_ERR_INVALID_ARG,
                     "Z_tf32 (the tf32 rung's shadow) needs a bf16 context, 16-byte alignment, "
                     "ldz_tf32 >= n and a 16-byte row pitch");
    if (pr->Z != nullptr && pr->ldz < pr->n)
      return set_err(ctx, PF_ERR_INVALID_ARG, "max-cut Z needs ldz >= n");
    if ((lp || pr->Z == nullptr) && !pr->S)
      return set_err(ctx, PF_ERR_INVALID_ARG, "structured max-cut needs the S workspace (nnz)");
  } else if (pr->kind == PF_PROBLEM_NCE) {
    if (!pr->Z || pr->ldz < pr->n || !pr->lam)
      return set_err(ctx, PF_ERR_INVALID_ARG, "NCE needs Z (G, ldz >= n) and lam (x)");
    if (ctx->opt.precision != PF_PREC_FP64)
      return set_err(ctx, PF_ERR_UNSUPPORTED, "NCE runs in an FP64 context");
    if (pr->accel_l < 0 || pr->accel_l > PF_MAX_ACCEL || (pr->accel_l > 0 && !pr->hist))
      return set_err(ctx, PF_ERR_INVALID_ARG,
                     "NCE extrapolation needs 0 <= accel_l <= %d and hist ((l+2) x n)",
                     PF_MAX_ACCEL);
  } else if (pr->kind == PF_PROBLEM_NNLS) {
    if (!pr->vals_f64 || !pr->S || !pr->t_rowptr || !pr->t_colind || !pr->t_perm || !pr->fac ||
        pr->ldfac < 4 * p || !pr->fsv)
      return set_err(ctx, PF_ERR_INVALID_ARG,
                     "NNLS needs vals_f64, S, the transposed pattern, fac (ldfac >= 4p) and fsv");
    if (!(pr->mu > 0.0) || !(pr->mu <= 1.0) || pr->rank_cap < 0 || pr->rank_cap > p)
      return set_err(ctx, PF_ERR_INVALID_ARG, "NNLS needs 0 < mu <= 1 and 0 <= rank_cap <= p");
    if (p > kMaxP / 2)
      return set_err(ctx, PF_ERR_UNSUPPORTED, "NNLS runs with p <= %d", kMaxP / 2);
    if (ctx->opt.precision != PF_PREC_FP64 || width_rule_on(ctx))
      return set_err(ctx, PF_ERR_UNSUPPORTED, "NNLS runs in an FP64 context without the width rule");
  } else if (pr->kind == PF_PROBLEM_SVT) {
    if (!pr->vals_f64 || !pr->S || !pr->t_rowptr || !pr->t_colind || !pr->t_perm)
      return set_err(ctx, PF_ERR_INVALID_ARG,
                     "SVT needs vals_f64 (M on Omega), S (x) and the transposed pattern");
    if (!(pr->t > 0.0) || !(pr->mu > 0.0))
      return set_err(ctx, PF_ERR_INVALID_ARG, "SVT needs t > 0 and mu > 0");
    if (ctx->opt.precision != PF_PREC_FP64)
      return set_err(ctx, PF_ERR_UNSUPPORTED, "SVT runs in an FP64 context");
  } else if (pr->kind == PF_PROBLEM_COMPLETION) {
    if (!pr->vals_f32 || !pr->S)
      return set_err(ctx, PF_ERR_INVALID_ARG, "completion needs vals_f32 (M on Omega) and S");
    if (pr->t_perm != nullptr && (pr->nnz <= 0 || pr->nnz > INT32_MAX))
      return set_err(ctx, PF_ERR_INVALID_ARG, "completion with a mirror map needs 0 < nnz < 2^31");
    if (!(pr->t > 0.0) || !(pr->mu >= 0.0))
      return set_err(ctx, PF_ERR_INVALID_ARG, "completion needs t > 0 and mu >= 0");
  } else {
    return set_err(ctx, PF_ERR_INVALID_ARG, "unknown problem kind %d", pr->kind);
  }
  return PF_OK;
}

pf_status step_body(pf_ctx *ctx, const pf_problem *pr);

// One step of the problem's method, enqueued only (graph-capturable), then
// the saturation count of the block.
pf_status step_core(pf_ctx *ctx, const pf_problem *pr) {
  trace_begin(ctx);
  PF_TRY(step_body(ctx, pr));
  PF_CUDA(launch_step_end(ctx->stream, ctx->ws));
  trace_end(ctx);
  return PF_OK;
}

pf_status step_body(pf_ctx *ctx, const pf_problem *pr) {
  const int p = ctx->ws.p;  // active width
  const int n = (int)pr->n;
  cudaStream_t s = ctx->stream;
  const Workspace &ws = ctx->ws;
  const int degree = ctx->cur_degree;
  const bool lp = cur_lp(ctx);
  // the tf32 rung of a bf16 context's ladder reads the problem's fp32 shadow
  const bool tf32_now = ctx->cur_prec == PF_PREC_TF32;
  void *const zlp_now = (tf32_now && ctx->opt.precision == PF_PREC_BF16) ? pr->Z_tf32 : pr->Z_lp;
  const int64_t ldzlp_now =
      (tf32_now && ctx->opt.precision == PF_PREC_BF16) ? pr->ldz_tf32 : pr->ldz_lp;
  if (pr->kind == PF_PROBLEM_NNLS) {
    // G = (1+beta) X - beta Xp - A*(r): coefficients, residual r (in S), interval
    phase(ctx, PF_PHASE_UPDATE);
    PF_CUDA(launch_nnls_residual(s, ws, pr->rowptr, pr->colind, pr->t_rowptr, pr->t_perm,
                                 pr->vals_f64, n, pr->fac, pr->ldfac, pr->fsv, pr->S, pr->theta));
    Op og = {};  // G Z = [L | Lp] diag(coef) [R | Rp]^T Z - R_sp Z
    og.kind = PF_OP_LOWRANK_SPARSE;
    og.n = n;
    og.Uf = pr->fac;
    og.lduf = pr->ldfac;
    og.Vf = pr->fac + 2 * p;
    og.ldvf = pr->ldfac;
    og.lam = ws.resid;
    og.r = 2 * p;
    og.rowptr = pr->rowptr;
    og.colind = pr->colind;
    og.vals = pr->S;
    og.sscale = -1.0;
    Op ot = og;  // G^T Z = [R | Rp] diag(coef) [L | Lp]^T Z - R_sp^T Z
    ot.Uf = pr->fac + 2 * p;
    ot.Vf = pr->fac;
    ot.rowptr = pr->t_rowptr;
    ot.colind = pr->t_colind;
    ot.perm = pr->t_perm;
    double *const *Yb = ws.Y;
    phase(ctx, PF_PHASE_FILTER);
    for (int j = 0; j < degree; ++j) {
      const double *cur = j == 0 ? pr->U : Yb[(j - 1) & 1];
      const int64_t ldc = j == 0 ? pr->ldu : p;
      const double *prev = j == 1 ? pr->U : Yb[j & 1];
      const int64_t ldprev = j == 1 ? pr->ldu : p;
      PF_CUDA(launch_lowrank_sparse_apply(s, ws, og, cur, ldc, nullptr, 0, ws.W, p, MODE_PLAIN));
      PF_CUDA(launch_lowrank_sparse_apply(s, ws, ot, ws.W, p, j == 0 ? nullptr : prev, ldprev,
                                          Yb[j & 1], p, j == 0 ? MODE_FIRST : MODE_RECUR, cur,
                                          ldc));
    }
    PF_TRY(cholqr2(ctx, Yb[(degree - 1) & 1], p, pr->U, pr->ldu, n));
    phase(ctx, PF_PHASE_RR);
    PF_CUDA(launch_lowrank_sparse_apply(s, ws, og, pr->U, pr->ldu, nullptr, 0, ws.W, p,
                                        MODE_PLAIN));
    int nb = 0;
    PF_CUDA(launch_gram(s, ws, ws.W, p, ws.W, p, n, p, p, 0, &nb));
    phase(ctx, PF_PHASE_EIG);
    PF_CUDA(launch_jacobi(s, ws, ws.gpart, p, pr->theta));
    PF_CUDA(launch_apply_right(s, ws, pr->U, pr->ldu, pr->V, pr->ldv, n, p, ws.Yeig, 0, 0));
    PF_CUDA(launch_apply_right(s, ws, ws.W, p, Yb[0], p, n, p, ws.Yeig, 0, 0));
    phase(ctx, PF_PHASE_UPDATE);
    const int cap = pr->rank_cap > 0 ? pr->rank_cap : (p > 8 ? p - 8 : 1);
    PF_CUDA(launch_nnls_update(s, ws, n, pr->fac, pr->ldfac, pr->fsv, Yb[0], pr->V, pr->ldv,
                               pr->theta, cap));
    PF_CUDA(launch_copy_block(s, ws, pr->V, pr->ldv, n, p, pr->U, pr->ldu));
    return PF_OK;
  }
  if (pr->kind == PF_PROBLEM_SVT) {
    // interval on Y^T Y, Y = A*(x) (values x in S)
    phase(ctx, PF_PHASE_INTERVAL);
    PF_CUDA(launch_svt_interval(s, ws, pr->rowptr, pr->t_rowptr, pr->t_perm, pr->S, n,
                                pr->theta));
    // filter: each product Y^T (Y X) is two SpMMs, the recurrence in the second;
    // Y X is the plain CSR product of the low-rank + sparse kernel (r = 0)
    Op oy = {};
    oy.kind = PF_OP_LOWRANK_SPARSE;
    oy.n = n;
    oy.rowptr = pr->rowptr;
    oy.colind = pr->colind;
    oy.vals = pr->S;
    oy.sscale = 1.0;
    oy.shift = 0.0;
    double *const *Yb = ws.Y;
    phase(ctx, PF_PHASE_FILTER);
    for (int j = 0; j < degree; ++j) {
      const double *cur = j == 0 ? pr->U : Yb[(j - 1) & 1];
      const int64_t ldc = j == 0 ? pr->ldu : p;
      const double *prev = j == 1 ? pr->U : Yb[j & 1];
      const int64_t ldprev = j == 1 ? pr->ldu : p;
      PF_CUDA(launch_lowrank_sparse_apply(s, ws, oy, cur, ldc, nullptr, 0, ws.W, p, MODE_PLAIN));
      PF_CUDA(launch_svt_spmm(s, ws, pr->t_rowptr, pr->t_colind, pr->S, pr->t_perm, n, ws.W, p,
                              cur, ldc, j == 0 ? nullptr : prev, ldprev, Yb[j & 1], p,
                              j == 0 ? MODE_FIRST : MODE_RECUR));
    }
    PF_TRY(cholqr2(ctx, Yb[(degree - 1) & 1], p, pr->U, pr->ldu, n));
    // Rayleigh-Ritz on the projected Gram matrix: B = Y Q, B^T B = Wr theta Wr^T
    phase(ctx, PF_PHASE_RR);
    PF_CUDA(launch_lowrank_sparse_apply(s, ws, oy, pr->U, pr->ldu, nullptr, 0, ws.W, p,
                                        MODE_PLAIN));
    int nb = 0;
    PF_CUDA(launch_gram(s, ws, ws.W, p, ws.W, p, n, p, p, 0, &nb));
    phase(ctx, PF_PHASE_EIG);
    PF_CUDA(launch_jacobi(s, ws, ws.gpart, p, pr->theta));
    PF_CUDA(launch_apply_right(s, ws, pr->U, pr->ldu, pr->V, pr->ldv, n, p, ws.Yeig, 0, 0));
    PF_CUDA(launch_apply_right(s, ws, ws.W, p, Yb[0], p, n, p, ws.Yeig, 0, 0));
    phase(ctx, PF_PHASE_UPDATE);
    // shrink, sampled residual, dual update and report
    PF_CUDA(launch_svt_update(s, ws, pr->rowptr, pr->colind, pr->vals_f64, n, Yb[0], p, pr->V,
                              pr->ldv, pr->theta, pr->mu, pr->t, pr->S));
    PF_CUDA(launch_copy_block(s, ws, pr->V, pr->ldv, n, p, pr->U, pr->ldu));
    return PF_OK;
  }
  if (pr->kind == PF_PROBLEM_NCE) {
    phase(ctx, PF_PHASE_INTERVAL);
    PF_CUDA(launch_nce_interval(s, ws, pr->Z, pr->ldz, n, pr->theta, p));
    Op op = {};
    op.kind = PF_OP_DENSE;
    op.n = n;
    op.A = pr->Z;
    op.lda = pr->ldz;
    if (sliced(ctx, op)) {
      // one set of digit planes serves the filter and Rayleigh-Ritz; they
      // hold Z as sliced before the steps (oz_prepare_problem) or by the
      // previous step, which changed only the diagonal of Z: the chunks
      // holding a diagonal entry are sliced again
      PF_CUDA(launch_oz_zslice_diag(s, ws, pr->Z, pr->ldz, n));
      op.zs_ready = 1;
    }
    PF_TRY(filter_core(ctx, op, pr->U, pr->ldu, degree));
    PF_TRY(rr_core(ctx, op, pr->U, pr->ldu, pr->V, pr->ldv, pr->theta, nullptr));
    phase(ctx, PF_PHASE_UPDATE);
    PF_CUDA(launch_copy_block(s, ws, pr->V, pr->ldv, n, p, pr->U, pr->ldu));
    PF_CUDA(launch_nce_update(s, ws, pr->Z, pr->ldz, n, p, pr->V, pr->ldv, pr->theta, pr->lam,
                              pr->t > 0.0 ? pr->t : 1.0, pr->hist, pr->accel_l, pr->accel_lam));
    return PF_OK;
  }
  // a low-precision context keeps no FP64 dense Z up to date, so it always
  // uses the structured operator (also after the ladder has dropped to FP64)
  const bool structured = ctx->opt.precision != PF_PREC_FP64 || pr->Z == nullptr;
  if (pr->kind == PF_PROBLEM_MAXCUT && structured) {
    // structured Z = X~prev - tC - Diag(lam) for the Rayleigh-Ritz step (and
    // for the filter unless a low-precision dense shadow is used)
    phase(ctx, PF_PHASE_INTERVAL);
    PF_CUDA(launch_save_prev(s, ws, pr->V, pr->ldv, pr->theta, n, p));
    PF_CUDA(launch_maxcut_sparse_part(s, ws, pr->rowptr, pr->colind, pr->vals_f64, n, pr->lam,
                                      pr->S));
    PF_CUDA(launch_interval(s, ws, PF_PROBLEM_MAXCUT, pr->rowptr, pr->colind, pr->vals_f64, n,
                            pr->lam, ws.thprev, p));
    Op op = {};
    op.kind = PF_OP_LOWRANK_SPARSE;
    op.n = n;
    op.Uf = ws.Vprev;
    op.lduf = p;
    op.lam = ws.thprev;
    op.r = p;
    op.clamp = 1;
    op.rowptr = pr->rowptr;
    op.colind = pr->colind;
    op.vals = pr->S;
    op.sscale = 1.0;
    op.shift = 0.0;
    if (lp) {
      Op dop = {};
      dop.kind = PF_OP_DENSE;
      dop.n = n;
      dop.A_lp = zlp_now;
      dop.lda_lp = ldzlp_now;
      dop.lp_scale = 0.0;  // the scale the shadow was written with is on the device
      PF_TRY(filter_core_lp(ctx, dop, pr->U, pr->ldu, degree, tf32_now));
    } else {
      PF_TRY(filter_core(ctx, op, pr->U, pr->ldu, degree));
    }
    PF_TRY(rr_core(ctx, op, pr->U, pr->ldu, pr->V, pr->ldv, pr->theta, nullptr));
    phase(ctx, PF_PHASE_UPDATE);
    PF_CUDA(launch_copy_block(s, ws, pr->V, pr->ldv, n, p, pr->U, pr->ldu));
    PF_CUDA(launch_maxcut_struct_update(s, ws, pr->rowptr, pr->colind, pr->vals_f64, n, p, pr->V,
                                        pr->ldv, pr->theta, pr->lam));
    if (lp)
      PF_CUDA(launch_maxcut_lp_shadow(s, ws, tf32_now, pr->rowptr, pr->colind, pr->vals_f64, n,
                                      p, pr->V, pr->ldv, pr->theta, pr->lam, zlp_now, ldzlp_now));
  } else if (pr->kind == PF_PROBLEM_MAXCUT) {
    phase(ctx, PF_PHASE_INTERVAL);
    if (ctx->opt.dense_product == PF_DENSE_SLICED) {
      // the sliced update takes the dual residual from the factors of the
      // previous and the new X~: keep the previous Ritz pairs.  The row
      // bounds of the interval were left by the previous step's update (or
      // by oz_prepare_problem); the chunk maxima of the expansion's bound
      // start at zero
      PF_CUDA(launch_save_prev(s, ws, pr->V, pr->ldv, pr->theta, n, p));
      PF_CUDA(launch_interval_final(s, ws, n, pr->theta, p, ws.oz.mchunk, (n + 127) / 128));
    } else {
      PF_CUDA(launch_interval(s, ws, PF_PROBLEM_MAXCUT, pr->rowptr, pr->colind, pr->vals_f64, n,
                              pr->lam, pr->theta, p));
    }
    Op op = {};
    op.kind = PF_OP_DENSE;
    op.n = n;
    op.A = pr->Z;
    op.lda = pr->ldz;
    // the digit planes of Z are current: written by the previous step's
    // update, or by the host before the first step (pf_prox_step / pf_solve)
    op.zs_ready = sliced(ctx, op) ? 1 : 0;
    PF_TRY(filter_core(ctx, op, pr->U, pr->ldu, degree));
    PF_TRY(rr_core(ctx, op, pr->U, pr->ldu, pr->V, pr->ldv, pr->theta, nullptr));
    phase(ctx, PF_PHASE_UPDATE);
    PF_CUDA(launch_copy_block(s, ws, pr->V, pr->ldv, n, p, pr->U, pr->ldu));
    PF_CUDA(launch_maxcut_update(s, ws, pr->rowptr, pr->colind, pr->vals_f64, n, p, pr->V, pr->ldv,
                                 pr->theta, pr->Z, pr->ldz, pr->lam, sliced(ctx, op)));
  } else {
    phase(ctx, PF_PHASE_UPDATE);  // the sampled residual: the gradient of the prox step
    PF_CUDA(launch_save_prev(s, ws, pr->V, pr->ldv, pr->theta, n, p));
    PF_CUDA(launch_completion_residual(s, ws, pr->rowptr, pr->colind, pr->vals_f32, n, p, ws.Vprev,
                                       p, ws.thprev, pr->S, pr->t_perm, pr->nnz));
    // the residual kernel left the Gershgorin row bounds of -tS - t mu I
    phase(ctx, PF_PHASE_INTERVAL);
    PF_CUDA(launch_interval_final(s, ws, n, ws.thprev, p, nullptr, 0));
    Op op = {};
    op.kind = PF_OP_LOWRANK_SPARSE;
    op.n = n;
    op.Uf = ws.Vprev;
    op.lduf = p;
    op.lam = ws.thprev;
    op.r = p;
    op.clamp = 1;
    op.rowptr = pr->rowptr;
    op.colind = pr->colind;
    op.vals = pr->S;
    op.sscale = -pr->t;
    op.shift = -pr->t * pr->mu;
    PF_TRY(filter_core(ctx, op, pr->U, pr->ldu, degree));
    PF_TRY(rr_core(ctx, op, pr->U, pr->ldu, pr->V, pr->ldv, pr->theta, nullptr));
    phase(ctx, PF_PHASE_UPDATE);
    PF_CUDA(launch_copy_block(s, ws, pr->V, pr->ldv, n, p, pr->U, pr->ldu));
    PF_CUDA(launch_completion_kkt(s, ws, pr->V, pr->ldv, pr->theta, n, p));
  }
  return PF_OK;
}

void params_to_info(const Params &h, pf_iter_info *info, const pf_ctx *ctx = nullptr) {
  info->a = h.a;
  info->b = h.b;
  info->obj = h.obj;
  info->kkt = h.kkt;
  info->pinf = h.pinf;
  info->dinf = h.dinf;
  info->gap = h.gap;
  info->theta_max = h.theta_max;
  info->theta_min = h.theta_min;
  info->r_plus = h.r_plus;
  info->flags = h.flags;
  info->jacobi_sweeps = h.sweeps;
  info->reserved = 0;
  info->degree = ctx ? ctx->cur_degree : h.degree;
  info->precision = ctx ? ctx->cur_prec : h.precision;
}

pf_status read_params(pf_ctx *ctx, Params *h) {
  PF_CUDA(cudaMemcpyAsync(h, ctx->ws.prm, sizeof(Params), cudaMemcpyDeviceToHost, ctx->stream));
  PF_CUDA(cudaStreamSynchronize(ctx->stream));
  return PF_OK;
}

bool same_problem(const pf_problem &a, const pf_problem &b) {
  return a.kind == b.kind && a.n == b.n && a.rowptr == b.rowptr && a.colind == b.colind &&
         a.vals_f64 == b.vals_f64 && a.vals_f32 == b.vals_f32 && a.nnz == b.nnz && a.t == b.t &&
         a.mu == b.mu && a.U == b.U && a.ldu == b.ldu && a.V == b.V && a.ldv == b.ldv &&
         a.theta == b.theta && a.Z == b.Z && a.ldz == b.ldz && a.lam == b.lam && a.S == b.S &&
         a.Z_lp == b.Z_lp && a.ldz_lp == b.ldz_lp && a.accel_l == b.accel_l &&
         a.accel_lam == b.accel_lam && a.hist == b.hist && a.p_active == b.p_active &&
         a.guard == b.guard && a.ldg == b.ldg && a.t_rowptr == b.t_rowptr &&
         a.t_colind == b.t_colind && a.t_perm == b.t_perm && a.fac == b.fac &&
         a.ldfac == b.ldfac && a.fsv == b.fsv && a.rank_cap == b.rank_cap &&
         a.Z_tf32 == b.Z_tf32 && a.ldz_tf32 == b.ldz_tf32;
}

bool graph_matches(const pf_ctx *ctx, const pf_problem &pr) {
  return ctx->have_graph && same_problem(ctx->gkey, pr) && ctx->gdegree == ctx->cur_degree &&
         ctx->gprec == ctx->cur_prec && ctx->gp == ctx->ws.p;
}



// The adaptive ladder (spec precision pattern; readings in the design
// notes): a KKT residual read at a check joins the history; the solve has
// stalled when the best of the last 5 checks is not 5% below the best of the
// 5 checks before (the KKT residual of DRS is not monotone, and comparing
// single checks fires on its plateaus).  A stall moves a low-precision filter
// up one precision (bf16 -> tf32 when the problem carries the fp32 shadow ->
// FP64): a filter's precision sets a floor on the KKT residual that a higher
// degree does not remove.  In FP64 a stall raises the degree by one, up to
// degree_max.  Each move clears the history.
pf_status ladder_feed(pf_ctx *ctx, const pf_problem *pr, double kkt) {
  constexpr int W = 5;
  double *hist = ctx->ladder_hist;
  int &nh = ctx->ladder_n;
  if (nh == 2 * W) {
    for (int i = 0; i < 2 * W - 1; ++i) hist[i] = hist[i + 1];
    nh = 2 * W - 1;
  }
  hist[nh++] = kkt;
  if (nh < 2 * W) return PF_OK;
  double before = hist[0], recent = hist[W];
  for (int i = 1; i < W; ++i) {
    before = fmin(before, hist[i]);
    recent = fmin(recent, hist[W + i]);
  }
  if (recent < 0.95 * before) return PF_OK;
  const int dmax = ctx->opt.degree_max > ctx->opt.degree ? ctx->opt.degree_max : ctx->opt.degree;
  if (ctx->cur_prec == PF_PREC_BF16 && pr->kind == PF_PROBLEM_MAXCUT && pr->Z_tf32 != nullptr) {
    // tf32 rung: the fp32 shadow of the current iteration matrix, written
    // now from the state the bf16 steps left
    ctx->cur_prec = PF_PREC_TF32;
    PF_CUDA(launch_maxcut_lp_shadow(ctx->stream, ctx->ws, true, pr->rowptr, pr->colind,
                                    pr->vals_f64, (int)pr->n, ctx->ws.p, pr->V, pr->ldv,
                                    pr->theta, pr->lam, pr->Z_tf32, pr->ldz_tf32));
  } else if (cur_lp(ctx)) {
    ctx->cur_prec = PF_PREC_FP64;
  } else if (ctx->cur_degree < dmax) {
    ctx->cur_degree += 1;
  } else {
    return PF_OK;
  }
  nh = 0;
  return PF_OK;
}

}  // namespace

extern "C" {

static pf_status capture_step(pf_ctx *ctx, pf_problem *pr);
// Width rule of Sec. 4.2 after the step that advanced pr->iter to a multiple
// of adapt_every: r_+ of that step plus the guard vectors, rounded up to a
// multiple of 8, clamped to [p_min, p].  Synchronises the stream (r_+ is
// read on the host).
static pf_status apply_width_rule(pf_ctx *ctx, pf_problem *pr);

pf_status pf_create(const pf_options *opt, int64_t n_max, void *stream, pf_ctx **out) {
  if (!out) return PF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!opt) return PF_ERR_INVALID_ARG;
  if (opt->p < 1 || opt->p > kMaxP || opt->degree < 1 || opt->degree > 64 || opt->q != 1 ||
      !(opt->eta > 0.0 && opt->eta < 1.0) || n_max < opt->p || n_max > (int64_t)INT32_MAX / 2)
    return PF_ERR_INVALID_ARG;
  if (opt->precision != PF_PREC_FP64 && opt->precision != PF_PREC_BF16 &&
      opt->precision != PF_PREC_TF32)
    return PF_ERR_INVALID_ARG;
  if (opt->dense_product != PF_DENSE_SLICED && opt->dense_product != PF_DENSE_FP64)
    return PF_ERR_INVALID_ARG;
  const bool oz = opt->dense_product == PF_DENSE_SLICED;
  const bool lp = opt->precision != PF_PREC_FP64;
  pf_ctx *ctx = new (std::nothrow) pf_ctx();
  if (!ctx) return PF_ERR_OOM;
  ctx->opt = *opt;
  ctx->n_max = n_max;
  ctx->p = opt->p;
  ctx->stream = (cudaStream_t)stream;
  ctx->cur_degree = opt->degree;
  ctx->cur_prec = opt->precision;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = configure_skinny();
  if (e == cudaSuccess) e = configure_sparse();
  if (e == cudaSuccess) e = configure_jacobi();
  if (e == cudaSuccess && (lp || oz)) e = configure_tc();
  if (e == cudaSuccess && oz) e = configure_oz();
  if (e != cudaSuccess) {
    delete ctx;
    return PF_ERR_CUDA;
  }
  const int p = opt->p;
  const size_t np = (size_t)n_max * p;
  // largest split-K partial buffer over all n <= n_max
  // (beyond 2^20 rows every split count is 1: a single split already has
  // more row blocks than 8 per SM)
  size_t part = np;
  const int64_t n_scan = n_max < ((int64_t)1 << 20) ? n_max : ((int64_t)1 << 20);
  for (int n = p; n <= n_scan; ++n) {
    int kc = 0;
    const size_t v = (size_t)dense_splits(n, sms, &kc) * n * p;
    if (v > part) part = v;
  }
  const size_t sq = (size_t)kMaxP * kMaxP;
  size_t off[20];
  size_t tot = 0;
  const size_t sizes[] = {np, np, np, np, part, (size_t)kMaxGramBlocks * sq,
                          (size_t)kRedSlots * kMaxRedBlocks * kRedWidth, sq, sq, sq, kMaxP, kMaxP,
                          (size_t)n_max, (size_t)n_max, (size_t)(kLanczos + 2) * n_max,
                          np + (size_t)n_max /* Xs: n_max x (p rounded up to even)
                                                float pairs, 8 bytes each */};
  const int nsz = sizeof(sizes) / sizeof(sizes[0]);
  for (int i = 0; i < nsz; ++i) {
    off[i] = tot;
    tot += align_up(sizes[i] * sizeof(double));
  }
  const size_t prm_off = tot;
  tot += align_up(sizeof(Params));
  const size_t info_off = tot;
  tot += align_up(sizeof(pf_iter_info));
  // low-precision buffers: Y32[2], U32 (fp32 n x p); Xt[2] (p x ldxt, 4-byte elements)
  const int64_t ldxt = ((n_max + 63) / 64) * 64;
  size_t lp_off[7] = {0, 0, 0, 0, 0, 0, 0};
  if (lp) {
    for (int i = 0; i < 3; ++i) {
      lp_off[i] = tot;
      tot += align_up(np * sizeof(float));
    }
    for (int i = 3; i < 5; ++i) {
      lp_off[i] = tot;
      tot += align_up((size_t)p * ldxt * sizeof(float));
    }
    for (int i = 5; i < 7; ++i) {
      lp_off[i] = tot;
      tot += align_up((size_t)n_max * 64 * sizeof(float));
    }
  }
  void *base = nullptr;
  if (cudaMalloc(&base, tot) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return PF_ERR_OOM;
  }
  char *b = (char *)base;
  Workspace &ws = ctx->ws;
  ws.n_max = (int)n_max;
  ws.p = p;
  ws.num_sms = sms;
  ws.Y[0] = (double *)(b + off[0]);
  ws.Y[1] = (double *)(b + off[1]);
  ws.W = (double *)(b + off[2]);
  ws.Vprev = (double *)(b + off[3]);
  ws.part = (double *)(b + off[4]);
  ws.gpart = (double *)(b + off[5]);
  ws.red = (double *)(b + off[6]);
  ws.Rinv = (double *)(b + off[7]);
  ws.Yeig = (double *)(b + off[8]);
  ws.T = (double *)(b + off[9]);
  ws.thprev = (double *)(b + off[10]);
  ws.resid = (double *)(b + off[11]);
  ws.gdiag = (double *)(b + off[12]);
  ws.rsum = (double *)(b + off[13]);
  ws.lz = (double *)(b + off[14]);
  ws.Xs = (float2 *)(b + off[15]);
  ws.prm = (Params *)(b + prm_off);
  ws.info = (pf_iter_info *)(b + info_off);
  ws.ldxt = ldxt;
  if (lp) {
    ws.Y32[0] = (float *)(b + lp_off[0]);
    ws.Y32[1] = (float *)(b + lp_off[1]);
    ws.U32 = (float *)(b + lp_off[2]);
    ws.Xt[0] = (void *)(b + lp_off[3]);
    ws.Xt[1] = (void *)(b + lp_off[4]);
    ws.Wf = (float *)(b + lp_off[5]);
    ws.Vf = (float *)(b + lp_off[6]);
  }
  ctx->base = base;
  ctx->bytes = tot;
  if (cudaMemsetAsync(base, 0, tot, ctx->stream) != cudaSuccess ||
      launch_params_init(ctx->stream, ws.prm, opt->eta, 0.0, 0.0, opt->degree, opt->precision) !=
          cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaFree(base);
    delete ctx;
    return PF_ERR_CUDA;
  }
  *out = ctx;
  return PF_OK;
}

pf_status pf_destroy(pf_ctx *ctx) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->have_graph) cudaGraphExecDestroy(ctx->gexec);
  cudaFree(ctx->base);
  if (ctx->oz_base) cudaFree(ctx->oz_base);
  if (ctx->trace)
    for (int i = 0; i <= kTraceMarks; ++i) cudaEventDestroy(ctx->tev[i]);
  delete ctx;
  return PF_OK;
}

pf_status pf_set_tracing(pf_ctx *ctx, int32_t on) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  if (on && !ctx->trace) {
    for (int i = 0; i <= kTraceMarks; ++i) {
      if (cudaEventCreate(&ctx->tev[i]) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->tev[j]);
        return set_err(ctx, PF_ERR_CUDA, "cudaEventCreate failed");
      }
    }
    ctx->trace = true;
    ctx->nmarks = 0;
  } else if (!on && ctx->trace) {
    PF_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i <= kTraceMarks; ++i) cudaEventDestroy(ctx->tev[i]);
    ctx->trace = false;
    ctx->nmarks = 0;
  }
  return PF_OK;
}

pf_status pf_phase_times(pf_ctx *ctx, double *ms) {
  if (!ctx || !ms) return PF_ERR_INVALID_ARG;
  for (int k = 0; k < PF_NUM_PHASES; ++k) ms[k] = 0.0;
  if (!ctx->trace || ctx->nmarks == 0) return PF_OK;
  PF_CUDA(cudaEventSynchronize(ctx->tev[ctx->nmarks]));
  for (int i = 0; i < ctx->nmarks; ++i) {
    float t = 0.0f;
    PF_CUDA(cudaEventElapsedTime(&t, ctx->tev[i], ctx->tev[i + 1]));
    ms[ctx->tmark[i]] += (double)t;
  }
  return PF_OK;
}

pf_status pf_ladder_update(pf_ctx *ctx, pf_problem *pr, double kkt) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  PF_TRY(check_problem(ctx, pr));
  if (ctx->opt.adaptive == 0) return PF_OK;
  if (!std::isfinite(kkt)) return set_err(ctx, PF_ERR_INVALID_ARG, "kkt must be finite");
  return ladder_feed(ctx, pr, kkt);
}

pf_status pf_set_wait_limit(uint64_t ns) {
  if (set_wait_limit_oz(ns) != cudaSuccess || set_wait_limit_tc(ns) != cudaSuccess)
    return PF_ERR_CUDA;
  return PF_OK;
}

pf_status pf_filter(pf_ctx *ctx, const pf_operator *op, double a, double b, int32_t degree,
                    double *U, int64_t ldu) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  ctx->ws.p = ctx->p;
  Op o;
  PF_TRY(make_op(ctx, op, &o));
  if (!(a < b) || !std::isfinite(a) || !std::isfinite(b))
    return set_err(ctx, PF_ERR_INVALID_ARG, "interval needs finite a < b");
  if (degree < 1 || degree > 64) return set_err(ctx, PF_ERR_INVALID_ARG, "degree must be 1..64");
  if (!U || ldu < ctx->p) return set_err(ctx, PF_ERR_INVALID_ARG, "U needs ldu >= p");
  if (sliced(ctx, o)) PF_TRY(ensure_oz(ctx));
  PF_CUDA(launch_set_interval(ctx->stream, ctx->ws.prm, a, b));
  if (sliced(ctx, o)) ctx->oz_owner = nullptr;
  trace_begin(ctx);
  PF_TRY(filter_core(ctx, o, U, ldu, degree));
  trace_end(ctx);
  if (sliced(ctx, o)) {
    ctx->oz_owner = o.A;
    ctx->oz_owner_n = o.n;
  }
  return PF_OK;
}

pf_status pf_rayleigh_ritz(pf_ctx *ctx, const pf_operator *op, const double *Q, int64_t ldq,
                           double *V, int64_t ldv, double *theta, double *resid) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  ctx->ws.p = ctx->p;
  Op o;
  PF_TRY(make_op(ctx, op, &o));
  if (!Q || ldq < ctx->p || !V || ldv < ctx->p || !theta)
    return set_err(ctx, PF_ERR_INVALID_ARG, "rayleigh_ritz needs Q, V (ld >= p) and theta");
  if (sliced(ctx, o)) {
    PF_TRY(ensure_oz(ctx));
    ctx->oz_owner = nullptr;
  }
  trace_begin(ctx);
  PF_TRY(rr_core(ctx, o, Q, ldq, V, ldv, theta, resid));
  trace_end(ctx);
  if (sliced(ctx, o)) {
    ctx->oz_owner = o.A;
    ctx->oz_owner_n = o.n;
  }
  return PF_OK;
}

pf_status pf_apply(pf_ctx *ctx, const pf_operator *op, const double *X, int64_t ldx, double *Y,
                   int64_t ldy) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  ctx->ws.p = ctx->p;
  Op o;
  PF_TRY(make_op(ctx, op, &o));
  if (!X || !Y || X == Y || ldx < ctx->p || ldy < ctx->p)
    return set_err(ctx, PF_ERR_INVALID_ARG, "apply needs distinct X, Y with ld >= p");
  if (o.kind == PF_OP_DENSE && o.A_lp != nullptr && ctx->opt.precision != PF_PREC_FP64) {
    const bool tf32 = ctx->opt.precision == PF_PREC_TF32;
    const Workspace &ws = ctx->ws;
    PF_CUDA(launch_set_scale(ctx->stream, ws.prm, o.lp_scale));
    PF_CUDA(launch_prep_lp(ctx->stream, ws, tf32, X, ldx, o.n, ws.U32, ws.Xt[0]));
    PF_CUDA(launch_tc_product(ctx->stream, ws, tf32, o.A_lp, o.lda_lp, o.n, ws.Xt[0], ws.U32,
                              nullptr, ws.Y32[0], nullptr, MODE_PLAIN));
    if (ldy == ctx->p)
      PF_CUDA(launch_f32_to_f64(ctx->stream, ws, ws.Y32[0], (int64_t)o.n * ctx->p, Y));
    else
      return set_err(ctx, PF_ERR_INVALID_ARG, "low-precision apply needs ldy == p");
    return PF_OK;
  }
  if (sliced(ctx, o)) {
    PF_TRY(ensure_oz(ctx));
    const Workspace &ws = ctx->ws;
    ctx->oz_owner = nullptr;
    PF_CUDA(launch_oz_zslice(ctx->stream, ws, o.A, o.lda, o.n));
    ctx->oz_owner = o.A;
    ctx->oz_owner_n = o.n;
    PF_CUDA(launch_oz_xslice(ctx->stream, ws, X, ldx, o.n, 0));
    PF_CUDA(launch_oz_product(ctx->stream, ws, o.n, 0, X, ldx, nullptr, 0, Y, ldy, -1,
                              MODE_PLAIN));
    return PF_OK;
  }
  return apply(ctx, o, X, ldx, nullptr, 0, Y, ldy, MODE_PLAIN);
}

int64_t pf_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

pf_status pf_problem_init(pf_ctx *ctx, pf_problem *pr) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  PF_TRY(check_problem(ctx, pr));
  if (dense_f64_problem(ctx, pr)) {
    PF_TRY(ensure_oz(ctx));
    ctx->oz_owner = nullptr;  // Z is set anew below
  }
  ctx->ivl_owner = nullptr;  // so is lam
  if (pr->p_active == 0) pr->p_active = ctx->p;
  ctx->ws.p = ctx->p;  // the fills below cover every column
  const int n = (int)pr->n, p = ctx->p;
  cudaStream_t s = ctx->stream;
  const Workspace &ws = ctx->ws;
  double t = pr->t;
  PF_CUDA(launch_params_init(s, ws.prm, ctx->opt.eta, t, pr->mu, ctx->opt.degree,
                             ctx->opt.precision));
  PF_CUDA(launch_fill(s, pr->V, n, p, pr->ldv, 0.0));
  PF_CUDA(launch_fill(s, pr->theta, 1, p, p, 0.0));
  if (pr->kind == PF_PROBLEM_SVT) {
    PF_CUDA(launch_params_init(s, ws.prm, ctx->opt.eta, pr->t, pr->mu, ctx->opt.degree,
                               ctx->opt.precision));
    PF_CUDA(launch_svt_init(s, ws, pr->vals_f64, pr->nnz, pr->t, pr->S));
  }
  if (pr->kind == PF_PROBLEM_NNLS) {
    PF_CUDA(launch_fill(s, pr->fac, n, 4 * p, pr->ldfac, 0.0));
    PF_CUDA(launch_nnls_init(s, ws, pr->rowptr, pr->t_rowptr, pr->t_perm, pr->vals_f64, n, pr->t,
                             pr->mu, pr->fsv));
  }
  if (pr->kind == PF_PROBLEM_NCE) {
    if (!(pr->t > 0.0)) pr->t = 1.0;
    PF_CUDA(launch_params_init(s, ws.prm, ctx->opt.eta, pr->t, 0.0, ctx->opt.degree,
                               ctx->opt.precision));
    PF_CUDA(launch_nce_init(s, ws, pr->Z, pr->ldz, n, pr->lam,
                            pr->accel_l > 0 ? pr->hist : nullptr));
  }
  if (pr->kind == PF_PROBLEM_MAXCUT) {
    PF_CUDA(launch_cnorm(s, ws, pr->vals_f64, pr->nnz));
    Params h;
    PF_TRY(read_params(ctx, &h));
    if (!(h.Cnorm > 0.0) || !std::isfinite(h.Cnorm))
      return set_err(ctx, PF_ERR_INVALID_ARG, "max-cut cost matrix has zero or non-finite norm");
    if (!(t > 0.0)) t = 10.0 * std::sqrt((double)n) / h.Cnorm;
    pr->t = t;
    PF_CUDA(launch_params_init(s, ws.prm, ctx->opt.eta, t, 0.0, ctx->opt.degree,
                               ctx->opt.precision));
    PF_CUDA(launch_cnorm(s, ws, pr->vals_f64, pr->nnz));
    if (pr->Z != nullptr)
      PF_CUDA(launch_maxcut_init(s, ws, pr->rowptr, pr->colind, pr->vals_f64, n, t, pr->Z,
                                 pr->ldz, pr->lam));
    else
      PF_CUDA(launch_maxcut_init_lam(s, ws, pr->rowptr, pr->colind, pr->vals_f64, n, t, pr->lam));
    if (ctx->opt.precision != PF_PREC_FP64)
      PF_CUDA(launch_maxcut_lp_shadow(s, ws, ctx->opt.precision == PF_PREC_TF32, pr->rowptr,
                                      pr->colind, pr->vals_f64, n, p, pr->V, pr->ldv, pr->theta,
                                      pr->lam, pr->Z_lp, pr->ldz_lp));
  }
  if (pr->kind == PF_PROBLEM_COMPLETION && pr->t_perm != nullptr) {
    // the mirror map must send (i, j) to (j, i): checked once per problem
    int *bad = reinterpret_cast<int *>(ws.red + (int64_t)SLOT_MISC * kMaxRedBlocks * kRedWidth);
    PF_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    PF_CUDA(launch_mirror_check(s, ws, pr->rowptr, pr->colind, pr->t_perm, n, pr->nnz, bad));
    int hbad = 0;
    PF_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    if (hbad)
      return set_err(ctx, PF_ERR_INVALID_ARG,
                     "t_perm is not the mirror map of a symmetric sampling pattern");
  }
  PF_CUDA(cudaStreamSynchronize(s));
  PF_CUDA(cudaGetLastError());
  pr->iter = 0;
  ctx->ws.p = pr->p_active;
  ctx->cur_degree = ctx->opt.degree;
  ctx->cur_prec = ctx->opt.precision;
  ctx->ladder_n = 0;
  return PF_OK;
}

pf_status pf_prox_step(pf_ctx *ctx, pf_problem *pr, pf_iter_info *info) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  PF_TRY(check_problem(ctx, pr));
  PF_TRY(oz_prepare_problem(ctx, pr));
  ctx->ws.p = active_width(ctx, pr);
  ctx->oz_owner = nullptr;
  PF_TRY(step_core(ctx, pr));
  oz_after_steps(ctx, pr);
  pr->iter += 1;
  if (info) {
    Params h;
    PF_TRY(read_params(ctx, &h));
    params_to_info(h, info, ctx);
    if (h.flags & 8) return set_err(ctx, PF_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
    if (h.flags & 4) return set_err(ctx, PF_ERR_NAN, "non-finite Ritz value");
    if (h.flags & 2) return set_err(ctx, PF_ERR_CHOL_BREAKDOWN, "CholQR2 broke down");
  }
  if (width_rule_on(ctx) && pr->iter % ctx->opt.adapt_every == 0)
    PF_TRY(apply_width_rule(ctx, pr));
  return PF_OK;
}

static pf_status apply_width_rule(pf_ctx *ctx, pf_problem *pr) {
  Params h;
  PF_TRY(read_params(ctx, &h));
  const int p_old = active_width(ctx, pr);
  int want = h.r_plus + ctx->opt.adapt_guard;
  want = ((want + 7) / 8) * 8;
  if (want < ctx->opt.p_min) want = ctx->opt.p_min;
  if (want > ctx->p) want = ctx->p;
  if (want > p_old)
    PF_CUDA(launch_grow_block(ctx->stream, ctx->ws, pr->U, pr->ldu, pr->V, pr->ldv, pr->theta,
                              (int)pr->n, p_old, want, pr->guard, pr->ldg));
  pr->p_active = want;
  ctx->ws.p = want;
  return PF_OK;
}

pf_status pf_get_info(pf_ctx *ctx, pf_iter_info *info) {
  if (!ctx || !info) return PF_ERR_INVALID_ARG;
  Params h;
  PF_TRY(read_params(ctx, &h));
  params_to_info(h, info, ctx);
  return PF_OK;
}

pf_status pf_enqueue_steps(pf_ctx *ctx, pf_problem *pr, int64_t n_steps) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  PF_TRY(check_problem(ctx, pr));
  if (n_steps < 0) return set_err(ctx, PF_ERR_INVALID_ARG, "n_steps must be >= 0");
  PF_TRY(oz_prepare_problem(ctx, pr));
  if (width_rule_on(ctx))
    return set_err(ctx, PF_ERR_UNSUPPORTED, "the block width rule needs host decisions "
                                            "(pf_prox_step / pf_solve)");
  ctx->ws.p = active_width(ctx, pr);
  ctx->oz_owner = nullptr;
  const bool use_graph = ctx->stream != nullptr;
  for (int64_t k = 0; k < n_steps; ++k) {
    if (use_graph) {
      if (!graph_matches(ctx, *pr))
        PF_TRY(capture_step(ctx, pr));
      PF_CUDA(cudaGraphLaunch(ctx->gexec, ctx->stream));
    } else {
      PF_TRY(step_core(ctx, pr));
    }
    pr->iter += 1;
  }
  oz_after_steps(ctx, pr);
  return PF_OK;
}

pf_status pf_report_async(pf_ctx *ctx, pf_iter_info *info) {
  if (!ctx || !info) return PF_ERR_INVALID_ARG;
  PF_CUDA(launch_export_info(ctx->stream, ctx->ws, ctx->cur_degree,
                             ctx->cur_prec));
  PF_CUDA(cudaMemcpyAsync(info, ctx->ws.info, sizeof(pf_iter_info), cudaMemcpyDeviceToHost,
                          ctx->stream));
  return PF_OK;
}

static pf_status capture_step(pf_ctx *ctx, pf_problem *pr) {
  if (ctx->have_graph) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->have_graph = false;
  }
  cudaGraph_t g = nullptr;
  PF_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  pf_status st = step_core(ctx, pr);
  cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
  if (st != PF_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  PF_CUDA(ce);
  cudaGraphExec_t ge = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  PF_CUDA(ie);
  ctx->gexec = ge;
  ctx->gkey = *pr;
  ctx->gdegree = ctx->cur_degree;
  ctx->gprec = ctx->cur_prec;
  ctx->gp = ctx->ws.p;
  ctx->have_graph = true;
  return PF_OK;
}

pf_status pf_solve(pf_ctx *ctx, pf_problem *pr, int64_t max_iter, double tol, int32_t check_every,
                   pf_result *out) {
  if (!ctx) return PF_ERR_INVALID_ARG;
  PF_TRY(check_problem(ctx, pr));
  PF_TRY(oz_prepare_problem(ctx, pr));
  if (max_iter < 0) return set_err(ctx, PF_ERR_INVALID_ARG, "max_iter must be >= 0");
  if (check_every < 1) check_every = 1;
  const bool use_graph = ctx->stream != nullptr;
  // adaptive ladder (ladder_feed) at every check
  const bool adaptive = ctx->opt.adaptive != 0;
  const bool check = tol > 0.0 || adaptive;
  Params h = {};
  int64_t it = 0;
  bool converged = false;
  ctx->ws.p = active_width(ctx, pr);
  ctx->oz_owner = nullptr;  // until the steps below have been enqueued without error
  for (; it < max_iter;) {
    if (use_graph) {
      if (!graph_matches(ctx, *pr))
        PF_TRY(capture_step(ctx, pr));
      PF_CUDA(cudaGraphLaunch(ctx->gexec, ctx->stream));
    } else {
      PF_TRY(step_core(ctx, pr));
    }
    ++it;
    pr->iter += 1;
    const bool rule_now = width_rule_on(ctx) && pr->iter % ctx->opt.adapt_every == 0;
    if (check && (it % check_every == 0 || it == max_iter || rule_now)) {
      PF_TRY(read_params(ctx, &h));
      if (tol > 0.0 && h.kkt <= tol) {
        converged = true;
        break;
      }
      if (adaptive) PF_TRY(ladder_feed(ctx, pr, h.kkt));
    }
    if (rule_now) PF_TRY(apply_width_rule(ctx, pr));
  }
  oz_after_steps(ctx, pr);
  PF_TRY(read_params(ctx, &h));
  if (out) {
    out->iters = it;
    out->kkt = h.kkt;
    out->obj = h.obj;
    params_to_info(h, &out->last, ctx);
  }
  if (h.flags & 8) return set_err(ctx, PF_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
  if (h.flags & 4) return set_err(ctx, PF_ERR_NAN, "non-finite Ritz value");
  if (h.flags & 2) return set_err(ctx, PF_ERR_CHOL_BREAKDOWN, "CholQR2 broke down");
  if (tol > 0.0 && !converged && max_iter > 0)
    return set_err(ctx, PF_ERR_NOT_CONVERGED, "kkt %.3e above tol %.3e after %lld steps", h.kkt,
                   tol, (long long)it);
  return PF_OK;
}

const char *pf_status_string(pf_status s) {
  switch (s) {
    case PF_OK: return "ok";
    case PF_ERR_INVALID_ARG: return "invalid argument";
    case PF_ERR_OOM: return "out of device memory";
    case PF_ERR_CUDA: return "CUDA error";
    case PF_ERR_CHOL_BREAKDOWN: return "CholQR2 breakdown";
    case PF_ERR_NAN: return "non-finite value";
    case PF_ERR_NOT_CONVERGED: return "not converged";
    case PF_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case PF_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *pf_last_error(const pf_ctx *ctx) { return ctx ? ctx->err : "no context"; }

}  // extern "C"
