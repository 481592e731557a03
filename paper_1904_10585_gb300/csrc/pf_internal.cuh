// Internal declarations shared by the CUDA translation units of libpf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "pf.h"

namespace pf {

constexpr int kMaxP = PF_MAX_P;
constexpr int kRedSlots = 6;        // independent reduction slots per step
constexpr int kRedWidth = 4;        // doubles per block in a reduction slot
constexpr int kMaxRedBlocks = 1024; // max blocks of a row reduction
constexpr int kMaxGramBlocks = 1024; // max blocks of a Gram (X^T Y) reduction (several per SM: the Dot2 chains need the warps)
constexpr int kMaxSplitK = 16;      // max K-splits of the dense FP64 product
// sliced tensor-core product (pf_oz.cu)
constexpr int kOzSlices = 7;        // 8-bit digit planes per FP64 operand
constexpr int kOzExpBad = 4096;     // exponent marking a row / chunk with Inf or NaN
constexpr int kOzMaxChunks = 32;    // 128-wide K chunks per split (int64 headroom)
constexpr int kOzMaxSplits = 8;     // K splits when the row blocks leave SMs idle

enum RedSlot { SLOT_INTERVAL = 0, SLOT_LAMBDA = 1, SLOT_EXPAND = 2, SLOT_SDDMM = 3, SLOT_RESID = 4,
               SLOT_MISC = 5 };

// Filter epilogue modes: Ynext = alpha (op(Ycur) - c Ycur) - beta Yprev.
enum CombineMode { MODE_PLAIN = 0, MODE_FIRST = 1, MODE_RECUR = 2 };

// Device-resident scalars of one context.  Written and read by kernels only
// (stream ordered), copied to host by pf_get_info.
struct Params {
  double a, b, c, e;      // filter interval [a, b], centre c, half-width e
  double ub;              // Gershgorin upper bound of the iteration matrix
  double eta;
  double t, mu;           // step size, completion weight
  double Cnorm;           // ||C||_F (max-cut)
  double lp_scale;        // s of the low-precision shadow A_lp = A / s
  double g0;              // NCE: ||grad F(x_0)||
  double obj, kkt, pinf, dinf, gap;
  double theta_max, theta_min;
  int have_prev;          // a previous Rayleigh-Ritz step exists
  int flags;              // bit0 shifted CholQR pass, bit1 breakdown, bit2 non-finite
  int r_plus;
  int degree;
  int precision;
  int sweeps;             // sweeps of the last p x p eigensolve
  int sat_run;            // consecutive steps with r_plus >= p - 2
  int acc_count;          // NCE extrapolation: iterates held in the window
  int acc_go;             // NCE extrapolation: the combination below is due
  double acc_c[PF_MAX_ACCEL + 1];  // its coefficients c_0..c_l
  // NCE: Lanczos estimate of the smallest eigenvalue (lower end of the interval)
  double lz_alpha[16], lz_beta[16];
  double a_lz;            // theta_min - residual bound
  int lz_m;               // Lanczos steps taken (fewer than kLanczos on breakdown)
  // NNLS (accelerated proximal gradient): momentum scalars and continuation
  double nn_t, nn_tp, nn_beta, nn_mu, nn_mubar;
};

// Lanczos steps of the NCE interval estimate (Sec. 4.1)
constexpr int kLanczos = 12;

// Internal iteration-matrix description.
struct Op {
  int kind;               // PF_OP_DENSE / PF_OP_LOWRANK_SPARSE
  int n;
  const double *A; int64_t lda;
  const void *A_lp; int64_t lda_lp; double lp_scale;   // low-precision shadow A / lp_scale
  const double *Uf; int64_t lduf; const double *lam; int r; int clamp;
  const int32_t *rowptr; const int32_t *colind; const double *vals;
  double sscale, shift;
  // non-symmetric low-rank part Uf diag(lam) Vf^T (Vf = nullptr: Vf = Uf), and
  // a sparse part read through a value permutation (vals[perm[e]], the
  // transposed pattern of a non-symmetric matrix); both optional
  const double *Vf; int64_t ldvf;
  const int32_t *perm;
  // dense, sliced product: the digit planes of A are already current
  int zs_ready;
};

// Digit planes of the sliced dense product (allocated on first use).
struct OzBuffers {
  void *zs;               // byte planes of A (digit + 128): kOzSlices x slice_rows x ldk
  int *ez;                // exponents of A per row and 128-column chunk, slice_rows x (slice_rows / 128)
  void *xs[2];            // fp16 planes of the block: kOzSlices x kMaxP x ldk each
  int *ex[2];             // chunk x column exponents, (slice_rows / 128) x kMaxP each
  double *part;           // split partials, max splits x n_max x p
  int *cnt;               // arrival tickets per row block and column half (zero between launches)
  int64_t ldk;            // row pitch of the planes (n_max rounded up to 128)
  int64_t slice_rows;     // rows per A plane (n_max rounded up to 128)
  // max-cut expansion on the tensor cores: digit planes of the rows of
  // W = V diag(theta+) and V (kOzSlices x slice_rows x 64 bf16 each), their
  // row exponents, diag(X~) and per 128-row chunk max sqrt(diag(X~))
  void *wp, *vp;
  int *ew, *ev;
  double *xdiag;
  double *mchunk;
  // max-cut: C_ii and the off-diagonal |C| row sums of the problem whose
  // steps run (for the update's next-interval bounds)
  double *cdiag, *crsum;
};

struct Workspace {
  int n_max, p, num_sms;
  OzBuffers oz;
  double *Y[2];           // filter recurrence buffers, n_max x p
  double *W;              // op(Q), n_max x p
  double *Vprev;          // previous Ritz vectors (completion), n_max x p
  float2 *Xs;             // a block as float pairs, n_max x (p rounded up to even)
  double *part;           // split-K partials, kMaxSplitK x n_max x p
  double *gpart;          // Gram partials, kMaxGramBlocks x p x p
  double *red;            // reduction partials, kRedSlots x kMaxRedBlocks x kRedWidth
  double *Rinv;           // p x p
  double *Yeig;           // p x p eigenvectors of H
  double *T;              // p x p low-rank coefficients diag(w) Uf^T X
  double *thprev;         // p
  double *resid;          // p
  Params *prm;
  pf_iter_info *info;     // device copy of the step report (pf_report_async)
  // low-precision filter (allocated only for a bf16 / tf32 context)
  float *Y32[2];          // fp32 recurrence buffers, n_max x p
  float *U32;             // fp32 copy of the start block
  void *Xt[2];            // transposed low-precision operands, p x ldxt
  float *Wf, *Vf;         // fp32 factors of the shadow expansion, n_max x 64
  double *gdiag, *rsum;   // NCE: diag(G) and off-diagonal |G| row sums, n_max each
  double *lz;             // NCE: Lanczos basis q_0..q_{k-1}, y, w: (kLanczos + 2) x n_max
  int64_t ldxt;
};

// Host-side count of kernels enqueued by this library (see pf_kernel_launch_count).
extern std::atomic<int64_t> g_launches;
#define PF_LAUNCHED() (::pf::g_launches.fetch_add(1, std::memory_order_relaxed))

// ---------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------
cudaError_t configure_skinny();
cudaError_t configure_tc();
cudaError_t configure_sparse();
cudaError_t configure_jacobi();
cudaError_t configure_oz();
// limits of the bounded tensor-core pipeline waits (per translation unit)
cudaError_t set_wait_limit_oz(uint64_t ns);
cudaError_t set_wait_limit_tc(uint64_t ns);
// K splits of the sliced product for size n and block width p
int oz_splits(int n, int p, int num_sms);
// K splits of the dense FP64 product for size n (returns S, sets the chunk).
int dense_splits(int n, int num_sms, int *kchunk);

// ---------------------------------------------------------------------------
// launchers (each returns the launch error, if any)
// ---------------------------------------------------------------------------
cudaError_t launch_set_interval(cudaStream_t s, Params *prm, double a, double b);
cudaError_t launch_set_scale(cudaStream_t s, Params *prm, double lp_scale);
cudaError_t launch_dense_apply(cudaStream_t s, const Workspace &ws, const Op &op, const double *X,
                               int64_t ldx, const double *Yprev, int64_t ldp, double *Ynext,
                               int64_t ldn, int mode);
cudaError_t launch_lowrank_sparse_apply(cudaStream_t s, const Workspace &ws, const Op &op,
                                        const double *X, int64_t ldx, const double *Yprev,
                                        int64_t ldp, double *Ynext, int64_t ldn, int mode,
                                        const double *Xr = nullptr, int64_t ldr = 0);
cudaError_t launch_gram(cudaStream_t s, const Workspace &ws, const double *X, int64_t ldx,
                        const double *Y, int64_t ldy, int n, int px, int py, int cond_flag,
                        int *nblocks_out, bool sym = false);
cudaError_t launch_chol_inv(cudaStream_t s, const Workspace &ws, int nparts, int n, int p, int pass);
cudaError_t launch_apply_right(cudaStream_t s, const Workspace &ws, const double *Y, int64_t ldy,
                               double *Q, int64_t ldq, int n, int p, const double *R, int upper,
                               int cond_flag);
cudaError_t launch_jacobi(cudaStream_t s, const Workspace &ws, const double *H, int p,
                          double *theta);
cudaError_t launch_rotate_resid(cudaStream_t s, const Workspace &ws, const double *Q, int64_t ldq,
                                const double *W, int64_t ldw, int n, int p, const double *theta,
                                double *V, int64_t ldv, double *resid_out);
cudaError_t launch_lowrank_coef(cudaStream_t s, const Workspace &ws, int nparts, const double *lam,
                                int r, int p, int clamp);

// FP64-accurate sliced dense product on the tensor cores (pf_oz.cu): the
// digit planes of A (once per A), of the block X into xs[which], and the
// product Ynext = alpha (A X - c X) - beta Yprev reading xs[which], writing
// the next block's planes into xs[next] unless next < 0
cudaError_t launch_oz_zslice(cudaStream_t s, const Workspace &ws, const double *A, int64_t lda,
                             int n);
cudaError_t launch_oz_zslice_diag(cudaStream_t s, const Workspace &ws, const double *A, int64_t lda,
                             int n);
cudaError_t launch_oz_xslice(cudaStream_t s, const Workspace &ws, const double *X, int64_t ldx,
                             int n, int which);
cudaError_t launch_oz_product(cudaStream_t s, const Workspace &ws, int n, int which,
                              const double *X, int64_t ldx, const double *Yprev, int64_t ldp,
                              double *Ynext, int64_t ldn, int next, int mode);

// tensor-core (tcgen05) low-precision filter product and its conversions
cudaError_t launch_tc_product(cudaStream_t s, const Workspace &ws, bool tf32, const void *A_lp,
                              int64_t lda_lp, int n, const void *Xt,
                              const float *Ycur, const float *Yprev, float *Ynext, void *Xt_next,
                              int mode);
cudaError_t launch_tc_expand(cudaStream_t s, const Workspace &ws, bool f32out, const int32_t *rowptr,
                             const int32_t *colind, const double *vals, int n, const double *V,
                             int64_t ldv, const double *theta, const double *lam, void *Zlp,
                             int64_t ldz);
cudaError_t launch_to_f32(cudaStream_t s, const Workspace &ws, const double *src, int64_t lds,
                          int n, int p, float *dst);
cudaError_t launch_lowrank_sparse_apply32(cudaStream_t s, const Workspace &ws, const Op &op,
                                          const float *Uf32, const float *X, const float *Yprev,
                                          float *Ynext, int mode);
cudaError_t launch_prep_lp(cudaStream_t s, const Workspace &ws, bool tf32, const double *U,
                           int64_t ldu, int n, float *U32, void *Xt);
cudaError_t launch_f32_to_f64(cudaStream_t s, const Workspace &ws, const float *src, int64_t total,
                              double *dst);

// problem-level kernels
// Gershgorin row bounds of the max-cut sparse part -tC - Diag(lam) into the
// interval slot (red_blocks(n) partials), and the interval of the step from
// them (choose_b of Sec. 4.1); the latter also zeroes `zero` (nzero doubles).
cudaError_t launch_interval_rows(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                 const int32_t *colind, const double *vals, int n,
                                 const double *lam);
cudaError_t launch_interval_final(cudaStream_t s, const Workspace &ws, int n, const double *theta,
                                  int p, double *zero, int nzero);
// C_ii and the off-diagonal |C| row sums into ws.oz.cdiag / crsum.
cudaError_t launch_maxcut_cdata(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                const int32_t *colind, const double *vals, int n);
// The sliced max-cut update's row pass (k_oz_maxcut_rows), nb blocks.
cudaError_t launch_oz_maxcut_rows(cudaStream_t s, const Workspace &ws, int n, int p,
                                  const double *V, int64_t ldv, const double *theta,
                                  const double *Z, int64_t ldz, double *lam, int nb,
                                  double *red_lam, double *red_ivl);
cudaError_t launch_interval(cudaStream_t s, const Workspace &ws, int kind, const int32_t *rowptr,
                            const int32_t *colind, const double *vals, int n, const double *lam,
                            const double *theta, int p);
cudaError_t launch_maxcut_init(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                               const int32_t *colind, const double *vals, int n, double t,
                               double *Z, int64_t ldz, double *lam);
cudaError_t launch_cnorm(cudaStream_t s, const Workspace &ws, const double *vals, int64_t nnz);
// sliced: the expansion runs on the tensor cores (pf_oz.cu) and also writes
// the digit planes of the new Z for the next step's products
cudaError_t launch_maxcut_update(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                 const int32_t *colind, const double *vals, int n, int p,
                                 const double *V, int64_t ldv, const double *theta, double *Z,
                                 int64_t ldz, double *lam, bool sliced = false);
cudaError_t launch_oz_expand(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                             const int32_t *colind, const double *vals, int n, int p,
                             const double *V, int64_t ldv, const double *theta, const double *lam,
                             double *Z, int64_t ldz, double *red, int *nblocks);
cudaError_t launch_completion_residual(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                       const int32_t *colind, const float *mvals, int n, int p,
                                       const double *V, int64_t ldv, const double *theta,
                                       double *S, const int32_t *mirror, int64_t nnz);
cudaError_t launch_mirror_check(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                const int32_t *colind, const int32_t *mirror, int n, int64_t nnz,
                                int *bad);
cudaError_t launch_completion_kkt(cudaStream_t s, const Workspace &ws, const double *V, int64_t ldv,
                                  const double *theta, int n, int p);
cudaError_t launch_save_prev(cudaStream_t s, const Workspace &ws, const double *V, int64_t ldv,
                             const double *theta, int n, int p);
cudaError_t launch_maxcut_sparse_part(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                      const int32_t *colind, const double *vals, int n,
                                      const double *lam, double *Sout);
cudaError_t launch_maxcut_struct_update(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                        const int32_t *colind, const double *vals, int n, int p,
                                        const double *V, int64_t ldv, const double *theta,
                                        double *lam);
cudaError_t launch_maxcut_init_lam(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                   const int32_t *colind, const double *vals, int n, double t,
                                   double *lam);
cudaError_t launch_maxcut_lp_shadow(cudaStream_t s, const Workspace &ws, bool f32out,
                                    const int32_t *rowptr, const int32_t *colind,
                                    const double *vals, int n, int p, const double *V, int64_t ldv,
                                    const double *theta, const double *lam, void *Zlp,
                                    int64_t ldz);
cudaError_t launch_copy_block(cudaStream_t s, const Workspace &ws, const double *src, int64_t lds,
                              int n, int p, double *dst, int64_t ldd);
cudaError_t launch_nce_init(cudaStream_t s, const Workspace &ws, double *Z, int64_t ldz, int n,
                            double *x, double *hist);
cudaError_t launch_nce_interval(cudaStream_t s, const Workspace &ws, const double *Z, int64_t ldz,
                                int n, const double *theta, int p);
cudaError_t launch_nce_update(cudaStream_t s, const Workspace &ws, double *Z, int64_t ldz, int n,
                              int p, const double *V, int64_t ldv, const double *theta, double *x,
                              double tau, double *hist, int accel_l, double accel_lam);
cudaError_t launch_fill(cudaStream_t s, double *x, int64_t rows, int64_t cols, int64_t ld, double v);
// PFSVT (pf_svt.cu)
cudaError_t launch_svt_spmm(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                            const int32_t *colind, const double *vals, const int32_t *perm, int n,
                            const double *X, int64_t ldx, const double *Xr, int64_t ldr,
                            const double *Yprev, int64_t ldp, double *Ynext, int64_t ldn,
                            int mode);
cudaError_t launch_svt_interval(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                const int32_t *t_rowptr, const int32_t *t_perm, const double *x,
                                int n, const double *theta);
cudaError_t launch_svt_update(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                              const int32_t *colind, const double *mvals, int n, const double *L,
                              int64_t ldl, const double *R, int64_t ldr, const double *theta,
                              double mu, double tau, double *x);
cudaError_t launch_svt_init(cudaStream_t s, const Workspace &ws, const double *mvals, int64_t nnz,
                            double tau, double *x);
// PFNNLS (pf_svt.cu); fac = [L | Lp | R | Rp] (n x 4p, ldfac), fsv = [s | sp]
cudaError_t launch_nnls_init(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                             const int32_t *t_rowptr, const int32_t *t_perm, const double *mvals,
                             int n, double mu0, double mubar_rel, double *fsv);
cudaError_t launch_nnls_residual(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                 const int32_t *colind, const int32_t *t_rowptr,
                                 const int32_t *t_perm, const double *mvals, int n,
                                 const double *fac, int64_t ldfac, const double *fsv, double *r,
                                 const double *theta);
cudaError_t launch_nnls_update(cudaStream_t s, const Workspace &ws, int n, double *fac,
                               int64_t ldfac, double *fsv, const double *BY, const double *V,
                               int64_t ldv, const double *theta, int cap);
cudaError_t launch_grow_block(cudaStream_t s, const Workspace &ws, double *U, int64_t ldu,
                              double *V, int64_t ldv, double *theta, int n, int p_old, int p_new,
                              const double *guard, int64_t ldg);
cudaError_t launch_export_info(cudaStream_t s, const Workspace &ws, int degree, int precision);
cudaError_t launch_step_end(cudaStream_t s, const Workspace &ws);
cudaError_t launch_params_init(cudaStream_t s, Params *prm, double eta, double t, double mu,
                               int degree, int precision);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Deterministic block reduction (fixed tree).  `sh` holds >= 32 doubles.
// op: 0 sum, 1 min, 2 max.  Result valid in all threads.
// 1/x for a positive, finite x by Newton-Raphson, y <- y + y (1 - x y),
// from a single-precision seed: the top 23 bits of the mantissa of x as a
// float in [1, 2), its hardware reciprocal (rcp.approx, relative error
// below 2^-22 with the truncation), and the exponent of x applied by integer
// arithmetic.  Each step squares the relative error (2^-44, then rounding),
// so the result takes four dependent FP64 operations after the seed (a
// Cholesky pivot chain, a Jacobi rotation).  Exponents near the ends of
// the range take the plain division.
__device__ __forceinline__ double rcp_newton(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex < 64 || ex > 1982) return 1.0 / x;
  const float m = __int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF));
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(m));  // in (0.5, 1]
  const long long rb = (long long)__float_as_uint(r);
  const long long de = ((rb >> 23) & 0xFF) - 127 + 1023 - (ex - 1023);
  double y = __longlong_as_double((de << 52) | ((rb & 0x7FFFFF) << 29));
  y = fma(y, fma(-x, y, 1.0), y);
  y = fma(y, fma(-x, y, 1.0), y);
  return y;
}

// ---------------------------------------------------------------------------
// FP64-accurate sums of products on the FP32 pipe (GB300 runs FP64 at 1/64
// of FP32).  A double x is carried as an unevaluated pair of floats
// x = x1 + x2 (+ at most 2^-49 |x|): x1 = fl32(x), x2 = fl32(x - x1).
// Products of pairs are accumulated by the Dot2 scheme of Ogita, Rump and
// Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005):
// TwoProduct of the leading parts (exact through an FMA), TwoSum of the
// running sum (Knuth), and the product errors with the first-order terms
// x1 y2 + x2 y1 summed in plain fp32.  The result is within a few units of
// m 2^-48 of sum |x_k y_k| for m terms (an FP64 dot product: m 2^-53);
// tests/test_pair_arithmetic.py checks the bound against exact arithmetic.
// ---------------------------------------------------------------------------
// The pair of x, with integer operations for 2^-60 <= |x| < 2^60 (the
// conversion instructions from FP64 run on the slow FP64 pipe).
// df_split outside float's comfortable exponent range (|x| < 2^-60 or
// |x| >= 2^60, and Inf / NaN) by FP64 conversions.  A separate, never-inlined
// function: inlined, the compiler evaluates this rare branch's FP64 pipe
// conversions on every call (if-conversion), which on GB300's 1/64-rate FP64
// pipe costs more than the whole integer split.
static __device__ __noinline__ float2 df_split_wide(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if ((b << 1) == 0ull) return make_float2(0.0f, 0.0f);  // +-0 (padding, zero entries)
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex < 1023 - 60 || ex >= 1023 + 60) return df_split_wide(x);
  // x = m 2^(ex - 1075), m of 53 bits; x1 keeps the top 24 bits (rounded to
  // nearest, ties to even), x2 = the rest (|rem| <= 2^28), rounded to 24 bits
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned hi = (unsigned)(m >> 29);
  int rem = (int)(m & 0x1FFFFFFFull);
  if (rem > (1 << 28) || (rem == (1 << 28) && (hi & 1u))) {
    hi += 1u;
    rem -= 1 << 29;
  }
  int e32 = ex - 896;  // float exponent field of hi 2^(ex - 1046), hi in [2^23, 2^24)
  if (hi == (1u << 24)) {
    hi >>= 1;
    e32 += 1;
  }
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const float x1 = __uint_as_float(sgn | ((unsigned)e32 << 23) | (hi & 0x7FFFFFu));
  float x2 = 0.0f;
  if (rem != 0) {
    const float r = __int2float_rn(rem);  // |rem| <= 2^28: rounded to 24 bits
    x2 = __uint_as_float((__float_as_uint(r) + ((unsigned)(ex - 1075) << 23)) ^ sgn);
  }
  return make_float2(x1, x2);
}
// Exact float -> double with integer operations only (zero, subnormals,
// Inf and NaN included: no FP64-pipe conversion, which the compiler would
// otherwise evaluate on every call).
__device__ __forceinline__ double df_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e8 = (u >> 23) & 0xFFu, man = u & 0x7FFFFFu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long d;
  if (e8 == 0xFFu) {
    d = sgn | (0x7FFull << 52) | ((unsigned long long)man << 29);
  } else if (e8 != 0u) {
    d = sgn | ((unsigned long long)(e8 + 896u) << 52) | ((unsigned long long)man << 29);
  } else if (man == 0u) {
    d = sgn;
  } else {
    // subnormal: man 2^-149 with its leading bit at msb (0..22)
    const int msb = 31 - __clz(man);
    d = sgn | ((unsigned long long)(msb + 874) << 52) |
        (((unsigned long long)man << (52 - msb)) & 0xFFFFFFFFFFFFFull);
  }
  return __longlong_as_double((long long)d);
}
// (a1, a2) += (b1, b2)
__device__ __forceinline__ void df_add(float b1, float b2, float &a1, float &a2) {
  const float t = __fadd_rn(a1, b1);
  const float bp = __fsub_rn(t, a1);
  const float te = __fadd_rn(__fsub_rn(a1, __fsub_rn(t, bp)), __fsub_rn(b1, bp));
  a1 = t;
  a2 = __fadd_rn(a2, __fadd_rn(te, b2));
}
// (a1, a2) += (s1 + s2)(x1 + x2)
__device__ __forceinline__ void df_fma(float s1, float s2, float x1, float x2, float &a1,
                                       float &a2) {
  const float pp = __fmul_rn(s1, x1);
  const float pe = __fmaf_rn(s1, x1, -pp);                        // s1 x1 = pp + pe
  const float q = __fmaf_rn(s1, x2, __fmaf_rn(s2, x1, pe));
  const float t = __fadd_rn(a1, pp);                              // a1 + pp = t + te
  const float bp = __fsub_rn(t, a1);
  const float te = __fadd_rn(__fsub_rn(a1, __fsub_rn(t, bp)), __fsub_rn(pp, bp));
  a1 = t;
  a2 = __fadd_rn(a2, __fadd_rn(te, q));
}

// a b for pairs whose product does not cancel: |error terms| << |a.h b.h|
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float ph = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -ph);
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));
  const float h = __fadd_rn(ph, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, ph)));
}

// Two pairs at once on the packed FP32 instructions of sm_100 and later
// (add/sub/mul/fma .f32x2: one instruction, two lanes).  A packed register
// holds lane 0 in its low half.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(f2x r, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
  f2x r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
  f2x r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// (a1, a2) += (v1 + v2)(x1 + x2) on two lanes of packed pairs: the Dot2
// step of df_fma (the same operations and roundings per lane), with the
// leading product's negative nv1 x1 formed first so that the product error
// comes out of one FMA.  v1, nv1 = -v1 and v2 are given packed.
__device__ __forceinline__ void df_fma2(f2x v1, f2x nv1, f2x v2, f2x x1, f2x x2, f2x &a1,
                                        f2x &a2) {
  const f2x ppn = mul2(nv1, x1);                    // -(v1 x1) rounded
  const f2x pe = fma2(v1, x1, ppn);                 // the product's error, exact
  const f2x q = fma2(v1, x2, fma2(v2, x1, pe));
  const f2x t = sub2(a1, ppn);                      // a1 + p
  const f2x bp = sub2(t, a1);
  const f2x te = sub2(sub2(a1, sub2(t, bp)), add2(ppn, bp));
  a1 = t;
  a2 = add2(a2, add2(te, q));
}
// (a1, a2) += (b1, b2) on two lanes of packed pairs (TwoSum of the leading
// parts, the low parts added to its error)
__device__ __forceinline__ void df_add2(f2x b1, f2x b2, f2x &a1, f2x &a2) {
  const f2x t = add2(a1, b1);
  const f2x bp = sub2(t, a1);
  const f2x te = add2(sub2(a1, sub2(t, bp)), sub2(b1, bp));
  a1 = t;
  a2 = add2(a2, add2(te, b2));
}
__device__ __forceinline__ f2x shfl_xor2(f2x v, int off) {
  float a, b;
  upk2(v, a, b);
  return pk2(__shfl_xor_sync(0xffffffffu, a, off), __shfl_xor_sync(0xffffffffu, b, off));
}

__device__ __forceinline__ double block_reduce(double v, double *sh, int op) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = op == 0 ? warp_sum(v) : (op == 1 ? warp_min(v) : warp_max(v));
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double init = op == 0 ? 0.0 : (op == 1 ? INFINITY : -INFINITY);
  double w = (threadIdx.x < nw) ? sh[threadIdx.x] : init;
  if (wid == 0) w = op == 0 ? warp_sum(w) : (op == 1 ? warp_min(w) : warp_max(w));
  if (threadIdx.x == 0) sh[0] = w;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}
#endif

}  // namespace pf
