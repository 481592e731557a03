// Skinny FP64 kernels of the subspace extraction:
//  * Gram partials X^T Y over row blocks (CholQR2's Y^T Y, Rayleigh-Ritz's
//    Q^T (A Q), the low-rank coefficient Uf^T X), reduced in a fixed order;
//  * one-block Cholesky of the Gram matrix with a triangular inverse, with the
//    shifted CholeskyQR fallback of Fukaya, Kannan, Nakatsukasa, Yamamoto and
//    Yanagisawa (SIAM J. Sci. Comput., 2020) when a pivot collapses;
//  * the right multiplication Q = Y R^{-1} (orth of Eq. (subspace-update),
//    realised as CholQR2 = QR with positive diagonal R in exact arithmetic);
//  * the Ritz rotation V = Q Y with residuals ||A v_i - theta_i v_i|| (Eq. (RR));
//    the p x p eigensolve itself is the double-float Jacobi of pf_jacobi.cu.
#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int NT = 256;
constexpr int RC = 32;  // rows staged per step

// SYM (X = Y, so X^T Y is symmetric): warps skip the column groups that lie
// entirely below the diagonal of their rows and leave zeros there; the
// consumers (the Cholesky factorisation) read the upper triangle only.
template <int PT, bool SYM>
__global__ void __launch_bounds__(NT) k_gram(const double *__restrict__ X, int64_t ldx,
                                             const double *__restrict__ Y, int64_t ldy, int n,
                                             int px, int py, int rows_per_block,
                                             double *__restrict__ gpart, const Params *prm,
                                             int cond_flag) {
  if (cond_flag && !(prm->flags & 1)) return;
  constexpr int TM = PT / 16, TN = PT / 16;
  // rows staged as float pairs (df_split); each staged chunk of RC rows is
  // summed on the FP32 pipe by the Dot2 scheme and added to FP64 accumulators
  __shared__ float2 Xs[RC][PT + 1];
  __shared__ float2 Ys[RC][PT + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(n, r0 + rows_per_block);
  for (int rb = r0; rb < r1; rb += RC) {
    for (int e = tid; e < RC * PT; e += NT) {
      const int r = e / PT, c = e % PT, gr = rb + r;
      Xs[r][c] = df_split((gr < r1 && c < px) ? X[(int64_t)gr * ldx + c] : 0.0);
      Ys[r][c] = df_split((gr < r1 && c < py) ? Y[(int64_t)gr * ldy + c] : 0.0);
    }
    __syncthreads();
    float s1[TM][TN], s2[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) s1[i][j] = s2[i][j] = 0.0f;
#pragma unroll 4
    for (int r = 0; r < RC; ++r) {
      float2 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = Xs[r][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Ys[r][tx + 16 * j];
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        // rows of this warp: [2 w TM, 2 w TM + 2 TM); columns of group j: [16 j, 16 j + 16)
        if (SYM && 2 * (tid >> 5) * TM > 16 * j + 15) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) df_fma(a[i].x, a[i].y, b[j].x, b[j].y, s1[i][j], s2[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] += df_widen(s1[i][j]) + df_widen(s2[i][j]);
    __syncthreads();
  }
  double *out = gpart + (int64_t)blockIdx.x * px * py;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int a = ty * TM + i;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int b = tx + 16 * j;
      if (a < px && b < py) out[a * py + b] = acc[i][j];
    }
  }
}

// In-place fixed-order reduction of the Gram partials into partial 0:
// out[idx] = sum_q part[q][idx].  A block covers 32 outputs with 8 threads
// each: thread q sums partials q, q + 8, q + 16, ... in order, then the 8
// sub-sums are added in a fixed tree (deterministic, 8x the parallelism of
// one thread per output).
constexpr int GR_OUT = 32, GR_SUB = 8;
__global__ void __launch_bounds__(GR_OUT * GR_SUB) k_gram_reduce(double *__restrict__ gpart,
                                                                 int nparts, int m) {
  __shared__ double sub[GR_SUB][GR_OUT];
  const int o = threadIdx.x & (GR_OUT - 1), q0 = threadIdx.x / GR_OUT;
  const int idx = blockIdx.x * GR_OUT + o;
  double s = 0.0;
  if (idx < m)
    for (int q = q0; q < nparts; q += GR_SUB) s += gpart[(int64_t)q * m + idx];
  sub[q0][o] = s;
  __syncthreads();
  if (q0 == 0 && idx < m) {
    const double a = (sub[0][o] + sub[1][o]) + (sub[2][o] + sub[3][o]);
    const double b = (sub[4][o] + sub[5][o]) + (sub[6][o] + sub[7][o]);
    gpart[idx] = a + b;
  }
}

// Sum Gram partials, Cholesky G = R^T R (upper R), write R^{-1}.
// pass 0: on a collapsed pivot retry once with the shift
//         s = 11 (n p + p (p+1)) u tr(G) and set flags bit 0;
// pass 1: plain; pass 2: only runs when flags bit 0 is set.
// A failure with no retry left sets flags bit 1 and writes R^{-1} = I.
// Only the upper triangle of G is read.  Right-looking factorisation with one
// barrier per column: in step k every thread scales row k of R by 1/r_kk and
// updates the trailing upper triangle from the unscaled row; thread 0 updates
// A[k+1][k+1] first and takes the next pivot (square root and reciprocal)
// while the other warps finish the update.  The inverse reuses the pivot
// reciprocals: four lanes per column share each back-substitution sum.
__global__ void __launch_bounds__(NT) k_chol_inv(const double *__restrict__ gpart, int nparts,
                                                 int n, int p, int pass, double *__restrict__ Rinv,
                                                 Params *prm) {
  if (pass == 2 && !(prm->flags & 1)) return;
  extern __shared__ double dyn[];
  // A: the Gram matrix, reduced in place to the pivots (upper triangle);
  // U: the strict upper part of the unit upper factor G = U^T D U,
  // overwritten by that of -U^{-1}
  double(*A)[kMaxP + 1] = reinterpret_cast<double(*)[kMaxP + 1]>(dyn);
  double(*U)[kMaxP + 1] = reinterpret_cast<double(*)[kMaxP + 1]>(dyn + kMaxP * (kMaxP + 1));
  __shared__ double dpiv[kMaxP], rpiv[kMaxP];
  __shared__ double diag0[kMaxP];
  __shared__ int fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;
  // the partials were reduced in place: nparts is 1 on every call path
  for (int idx = tid; idx < p * p; idx += NT) {
    const int a = idx / p, b = idx % p;
    if (a <= b) {
      double s = 0.0;
      for (int q = 0; q < nparts; ++q) s += gpart[(int64_t)q * p * p + idx];
      A[a][b] = s;
      if (a == b) diag0[a] = s;
    }
  }
  __syncthreads();
  // pivot k: accepted when it is finite and above 1e-13 of the (shifted)
  // diagonal; its reciprocal then comes from rcp_newton
  auto take_pivot = [&](int k, double sh) {
    const double piv = A[k][k];
    if (!(piv > 1e-13 * (diag0[k] + sh)) || !isfinite(piv)) {
      fail = 1;
    } else {
      dpiv[k] = piv;
      rpiv[k] = rcp_newton(piv);
    }
  };
  double sh = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      // shifted retry from the original Gram matrix
      for (int idx = tid; idx < p * p; idx += NT) {
        const int a = idx / p, b = idx % p;
        if (a <= b) {
          double g = 0.0;
          for (int q = 0; q < nparts; ++q) g += gpart[(int64_t)q * p * p + idx];
          A[a][b] = g + (a == b ? sh : 0.0);
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      fail = 0;
      take_pivot(0, sh);
    }
    __syncthreads();
    // G = U^T D U without square roots: row k of U is row k of the reduced
    // matrix times 1/d_k, and the trailing triangle loses A_ki A_kj / d_k.
    // The chain from one pivot to the next is one multiply, one FMA and
    // rcp_newton (no square root, no division).  (Spreading the trailing
    // triangle element by element over all warps measured slower: the step
    // is bound by that chain and the barrier, not by FP64 throughput.)
    for (int k = 0; k < p && !fail; ++k) {
      const double rk = rpiv[k];
      for (int j = k + 1 + tid; j < p; j += NT) U[k][j] = A[k][j] * rk;
      // trailing upper triangle; row k+1 first on warp 0 so that thread 0
      // can take the next pivot early
      for (int i = k + 1 + warp; i < p; i += NW) {
        const double aki = A[k][i] * rk;
        for (int j = i + lane; j < p; j += 32) A[i][j] = fma(-aki, A[k][j], A[i][j]);
        if (tid == 0 && i == k + 1) take_pivot(i, sh);
      }
      __syncthreads();
    }
    if (!fail) {
      ok = true;
      break;
    }
    if (pass != 0) break;
    __syncthreads();
    if (tid == 0) atomicOr(&prm->flags, 1);
    double tr = 0.0;
    for (int k = 0; k < p; ++k) tr += diag0[k];
    sh = 11.0 * ((double)n * p + (double)p * (p + 1)) * 1.1102230246251565e-16 * tr;
  }
  if (!ok) {
    if (tid == 0) atomicOr(&prm->flags, 2);
    for (int idx = tid; idx < p * p; idx += NT) Rinv[idx] = (idx / p == idx % p) ? 1.0 : 0.0;
    return;
  }
  // Y = -U^{-1} (strict upper part) in place, right-looking from the last
  // row: Y_mc = U_mc - sum_{m<j<c} U_mj Y_jc.  At the step for row j, row j
  // is final and column j still holds U; the step reads column j and row j
  // and writes only columns c > j of rows m < j, so it needs no barrier
  // inside
  for (int j = p - 2; j >= 1; --j) {
    const int w = p - 1 - j;
    for (int idx = tid; idx < j * w; idx += NT) {
      const int m = idx / w, c = j + 1 + idx % w;
      U[m][c] = fma(-U[m][j], U[j][c], U[m][c]);
    }
    __syncthreads();
  }
  // R = D^{1/2} U, so R^{-1} = U^{-1} D^{-1/2}: column b scaled by d_b^{-1/2}
  if (tid < p) rpiv[tid] = rsqrt(dpiv[tid]);
  __syncthreads();
  for (int idx = tid; idx < p * p; idx += NT) {
    const int a = idx / p, b = idx % p;
    Rinv[idx] = a < b ? -U[a][b] * rpiv[b] : (a == b ? rpiv[b] : 0.0);
  }
}

// Q = Y R (R p x p; `upper` skips the zero lower part).  In place allowed.
template <int PT>
__global__ void __launch_bounds__(NT) k_apply_right(const double *Y, int64_t ldy, double *Q,
                                                    int64_t ldq, int n, int p,
                                                    const double *__restrict__ R, int upper,
                                                    int rows_per_block, const Params *prm,
                                                    int cond_flag) {
  if (cond_flag && !(prm->flags & 1)) return;
  // R and the staged rows of Y as float pairs (df_split); each output is a
  // dot product of at most p terms summed by the Dot2 scheme on the FP32 pipe
  extern __shared__ double dyn[];
  float2(*Rs)[PT + 1] = reinterpret_cast<float2(*)[PT + 1]>(dyn);
  float2(*Ys)[PT + 1] = reinterpret_cast<float2(*)[PT + 1]>(dyn + PT * (PT + 1));
  const int tid = threadIdx.x;
  for (int idx = tid; idx < PT * PT; idx += NT) {
    const int a = idx / PT, b = idx % PT;
    Rs[a][b] = df_split((a < p && b < p) ? R[a * p + b] : 0.0);
  }
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(n, r0 + rows_per_block);
  for (int rb = r0; rb < r1; rb += RC) {
    __syncthreads();
    for (int e = tid; e < RC * PT; e += NT) {
      const int r = e / PT, c = e % PT, gr = rb + r;
      Ys[r][c] = df_split((gr < r1 && c < p) ? Y[(int64_t)gr * ldy + c] : 0.0);
    }
    __syncthreads();
    // warp w takes the CPW adjacent columns w CPW .. and lane l the column
    // w CPW + l mod CPW for rows l / CPW + RG u (U independent FMA chains
    // sharing each load of R).  With the upper-triangular R a warp's loop
    // ends at its own columns (k <= c), so the triangle halves the FP64 work
    // of the warps; a store instruction writes CPW adjacent entries of RG
    // rows (whole 32-byte sectors at CPW = 4)
    constexpr int NWARP = NT / 32, CPW = PT / NWARP, RG = 32 / CPW, U = RC / RG;
    static_assert(PT % NWARP == 0 && 32 % CPW == 0 && RC % RG == 0, "apply_right tiling");
    const int w = tid >> 5, lane = tid & 31;
    const int c = w * CPW + lane % CPW, rg = lane / CPW;
    const int kend = upper ? min(p, w * CPW + CPW) : p;  // the same for the whole warp
    if (w * CPW < p) {
      float a1[U], a2[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a1[u] = a2[u] = 0.0f;
      for (int k = 0; k < kend; ++k) {
        const float2 rk = Rs[k][c];  // zero below the diagonal and beyond p
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float2 y = Ys[rg + RG * u][k];
          df_fma(y.x, y.y, rk.x, rk.y, a1[u], a2[u]);
        }
      }
      if (c < p) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int gr = rb + rg + RG * u;
          if (gr < r1) Q[(int64_t)gr * ldq + c] = df_widen(a1[u]) + df_widen(a2[u]);
        }
      }
    }
  }
}

// V = Q Yeig and per-block column sums of (W Yeig - theta V)^2.
template <int PT>
__global__ void __launch_bounds__(NT) k_rotate_resid(const double *__restrict__ Q, int64_t ldq,
                                                     const double *__restrict__ W, int64_t ldw,
                                                     int n, int p, const double *__restrict__ Yeig,
                                                     const double *__restrict__ theta, double *V,
                                                     int64_t ldv, int rows_per_block,
                                                     double *__restrict__ rpart) {
  static_assert(NT % PT == 0, "thread count must be a multiple of the padded width");
  extern __shared__ double dyn[];
  double(*Ys)[PT + 1] = reinterpret_cast<double(*)[PT + 1]>(dyn);
  double(*Qs)[PT + 1] = reinterpret_cast<double(*)[PT + 1]>(dyn + PT * (PT + 1));
  double(*Ws)[PT + 1] = reinterpret_cast<double(*)[PT + 1]>(dyn + (PT + RC) * (PT + 1));
  double *red = dyn + (PT + 2 * RC) * (PT + 1);
  const int tid = threadIdx.x;
  const int c = tid % PT;
  for (int idx = tid; idx < PT * PT; idx += NT) {
    const int a = idx / PT, b = idx % PT;
    Ys[a][b] = (a < p && b < p) ? Yeig[a * p + b] : 0.0;
  }
  const double th = c < p ? theta[c] : 0.0;
  double racc = 0.0;
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(n, r0 + rows_per_block);
  for (int rb = r0; rb < r1; rb += RC) {
    __syncthreads();
    for (int e = tid; e < RC * PT; e += NT) {
      const int r = e / PT, cc = e % PT, gr = rb + r;
      const bool in = gr < r1 && cc < p;
      Qs[r][cc] = in ? Q[(int64_t)gr * ldq + cc] : 0.0;
      Ws[r][cc] = in ? W[(int64_t)gr * ldw + cc] : 0.0;
    }
    __syncthreads();
    for (int r = tid / PT; r < RC; r += NT / PT) {
      const int gr = rb + r;
      if (gr >= r1 || c >= p) continue;
      double v = 0.0, w = 0.0;
      for (int k = 0; k < p; ++k) {
        v = fma(Qs[r][k], Ys[k][c], v);
        w = fma(Ws[r][k], Ys[k][c], w);
      }
      V[(int64_t)gr * ldv + c] = v;
      const double d = w - th * v;
      racc = fma(d, d, racc);
    }
  }
  red[tid] = racc;
  __syncthreads();
  if (tid < PT) {
    double s = 0.0;
    for (int t = tid; t < NT; t += PT) s += red[t];
    if (tid < p) rpart[(int64_t)blockIdx.x * p + tid] = s;
  }
}

__global__ void k_resid_final(const double *__restrict__ rpart, int nparts, int p,
                              double *__restrict__ resid) {
  const int j = threadIdx.x;
  if (j >= p) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += rpart[(int64_t)q * p + j];
  resid[j] = sqrt(s);
}

// T[l][j] = w_l (Uf^T X)[l][j], w_l = lam_l (clamped at 0 when `clamp`).
__global__ void k_lowrank_coef(const double *__restrict__ gpart, int nparts, const double *lam,
                               int r, int p, int clamp, double *__restrict__ T) {
  for (int idx = threadIdx.x; idx < r * p; idx += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += gpart[(int64_t)q * r * p + idx];
    double w = lam[idx / p];
    if (clamp) w = w > 0.0 ? w : 0.0;
    T[idx] = w * s;
  }
}

constexpr size_t kSqBytes = 2 * kMaxP * (kMaxP + 1) * sizeof(double);
constexpr size_t apply_bytes(int PT) { return (size_t)(PT + RC) * (PT + 1) * sizeof(double); }
constexpr size_t rotate_bytes(int PT) {
  return ((size_t)(PT + 2 * RC) * (PT + 1) + NT) * sizeof(double);
}

}  // namespace

cudaError_t configure_skinny() {
  cudaError_t e;
#define PF_SET(fn, bytes)                                                                   \
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes)); \
  if (e != cudaSuccess) return e;
  PF_SET(k_chol_inv, kSqBytes)
  PF_SET(k_apply_right<16>, apply_bytes(16))
  PF_SET(k_apply_right<32>, apply_bytes(32))
  PF_SET(k_apply_right<64>, apply_bytes(64))
  PF_SET(k_rotate_resid<16>, rotate_bytes(16))
  PF_SET(k_rotate_resid<32>, rotate_bytes(32))
  PF_SET(k_rotate_resid<64>, rotate_bytes(64))
#undef PF_SET
  return cudaSuccess;
}

static void row_split(int n, int max_blocks, int min_rows, int *nb, int *rpb) {
  int b = (n + min_rows - 1) / min_rows;
  if (b > max_blocks) b = max_blocks;
  if (b < 1) b = 1;
  int r = (n + b - 1) / b;
  r = ((r + RC - 1) / RC) * RC;
  *rpb = r;
  *nb = (n + r - 1) / r;
  if (*nb < 1) *nb = 1;
}

cudaError_t launch_gram(cudaStream_t s, const Workspace &ws, const double *X, int64_t ldx,
                        const double *Y, int64_t ldy, int n, int px, int py, int cond_flag,
                        int *nblocks_out, bool sym) {
  int nb, rpb;
  row_split(n, kMaxGramBlocks, RC, &nb, &rpb);  // all SMs: the FP64 rate of one SM is small
  const int pm = px > py ? px : py;
  if (pm <= 16)
    {
      if (sym) k_gram<16, true><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      else k_gram<16, false><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      PF_LAUNCHED();
    }
  else if (pm <= 32)
    {
      if (sym) k_gram<32, true><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      else k_gram<32, false><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      PF_LAUNCHED();
    }
  else if (pm <= 48)
    {
      if (sym) k_gram<48, true><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      else k_gram<48, false><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      PF_LAUNCHED();
    }
  else
    {
      if (sym) k_gram<64, true><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      else k_gram<64, false><<<nb, NT, 0, s>>>(X, ldx, Y, ldy, n, px, py, rpb, ws.gpart, ws.prm, cond_flag);
      PF_LAUNCHED();
    }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // reduce the partials in place so that consumers read one matrix
  if (nb > 1) {
    const int m = px * py;
    k_gram_reduce<<<(m + GR_OUT - 1) / GR_OUT, GR_OUT * GR_SUB, 0, s>>>(ws.gpart, nb, m);
    PF_LAUNCHED();
    e = cudaGetLastError();
  }
  *nblocks_out = 1;
  return e;
}

cudaError_t launch_chol_inv(cudaStream_t s, const Workspace &ws, int nparts, int n, int p, int pass) {
  k_chol_inv<<<1, NT, kSqBytes, s>>>(ws.gpart, nparts, n, p, pass, ws.Rinv, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_apply_right(cudaStream_t s, const Workspace &ws, const double *Y, int64_t ldy,
                               double *Q, int64_t ldq, int n, int p, const double *R, int upper,
                               int cond_flag) {
  int nb, rpb;
  row_split(n, 4 * ws.num_sms, RC, &nb, &rpb);
  if (p <= 16)
    {
      k_apply_right<16><<<nb, NT, apply_bytes(16), s>>>(Y, ldy, Q, ldq, n, p, R, upper, rpb, ws.prm, cond_flag);
      PF_LAUNCHED();
    }
  else if (p <= 32)
    {
      k_apply_right<32><<<nb, NT, apply_bytes(32), s>>>(Y, ldy, Q, ldq, n, p, R, upper, rpb, ws.prm, cond_flag);
      PF_LAUNCHED();
    }
  else
    {
      k_apply_right<64><<<nb, NT, apply_bytes(64), s>>>(Y, ldy, Q, ldq, n, p, R, upper, rpb, ws.prm, cond_flag);
      PF_LAUNCHED();
    }
  return cudaGetLastError();
}

cudaError_t launch_rotate_resid(cudaStream_t s, const Workspace &ws, const double *Q, int64_t ldq,
                                const double *W, int64_t ldw, int n, int p, const double *theta,
                                double *V, int64_t ldv, double *resid_out) {
  int nb, rpb;
  row_split(n, kMaxGramBlocks, 64, &nb, &rpb);
  if (p <= 16)
    {
      k_rotate_resid<16><<<nb, NT, rotate_bytes(16), s>>>(Q, ldq, W, ldw, n, p, ws.Yeig, theta, V, ldv, rpb, ws.gpart);
      PF_LAUNCHED();
    }
  else if (p <= 32)
    {
      k_rotate_resid<32><<<nb, NT, rotate_bytes(32), s>>>(Q, ldq, W, ldw, n, p, ws.Yeig, theta, V, ldv, rpb, ws.gpart);
      PF_LAUNCHED();
    }
  else
    {
      k_rotate_resid<64><<<nb, NT, rotate_bytes(64), s>>>(Q, ldq, W, ldw, n, p, ws.Yeig, theta, V, ldv, rpb, ws.gpart);
      PF_LAUNCHED();
    }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_resid_final<<<1, kMaxP, 0, s>>>(ws.gpart, nb, p, resid_out ? resid_out : ws.resid);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_lowrank_coef(cudaStream_t s, const Workspace &ws, int nparts, const double *lam,
                                int r, int p, int clamp) {
  k_lowrank_coef<<<1, NT, 0, s>>>(ws.gpart, nparts, lam, r, p, clamp, ws.T);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
