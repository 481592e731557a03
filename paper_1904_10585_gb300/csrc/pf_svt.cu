// Polynomial-filtered SVT for matrix completion (Sec. 5.2.1, Eq. (svt)).
//
// The dual variable x lives on the sample set Omega; Y = A*(x) is the sparse
// n x n matrix with the values x on Omega.  One step:
//   interval   a = 0 (Y^T Y is PSD), b by the previous smallest Ritz value,
//              upper bound ||Y||_1 ||Y||_inf >= sigma_max^2;
//   filter     d Chebyshev products of Y^T Y, each two CSR SpMMs (Y, then
//              Y^T through the transposed pattern), the recurrence fused into
//              the second;
//   CholQR2    (shared with the other problems);
//   Ritz       B = Y Q, B^T B = Wr diag(theta) Wr^T (Jacobi), right
//              vectors Q Wr, scaled left vectors L = B Wr (= U_left sigma);
//   update     w = P_Omega(L diag((sigma - mu)_+ / sigma) (Q Wr)^T),
//              x <- x + tau (m - w), and the report sums.
#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int NT = 256;
constexpr int WPB = NT / 32;

// Y_out = op(X) with op(X) = S X (S the CSR matrix, values vals[e] or
// vals[perm[e]]), then the recurrence epilogue on the base block Xr:
//   PLAIN: Y = op(X);  FIRST: Y = (op(X) - c Xr) / e;  RECUR: 2 (op(X) - c Xr) / e - Yprev.
// Half-warps take alternate entries of a row; lanes cover 16 columns each.
template <int JG>
__global__ void __launch_bounds__(NT) k_svt_spmm(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ vals, const int32_t *__restrict__ perm, int n, int p,
    const double *__restrict__ X, int64_t ldx, const double *__restrict__ Xr, int64_t ldr,
    const double *Yprev, int64_t ldp, double *Ynext, int64_t ldn, const Params *__restrict__ prm,
    int mode) {
  double c = 0.0, alpha = 1.0;
  if (mode != MODE_PLAIN) {
    c = prm->c;
    alpha = (mode == MODE_FIRST ? 1.0 : 2.0) / prm->e;
  }
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const int warps = gridDim.x * WPB;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double acc[JG];
#pragma unroll
    for (int g = 0; g < JG; ++g) acc[g] = 0.0;
    const int e0 = rowptr[row], e1 = rowptr[row + 1];
    for (int base = e0; base < e1; base += 32) {
      const int my = base + lane;
      const int mcol = my < e1 ? colind[my] : 0;
      const double mv = my < e1 ? vals[perm != nullptr ? perm[my] : my] : 0.0;
      const int cnt = min(32, e1 - base);
      for (int k = 0; k < cnt; k += 2) {
        const int kk = k + half;  // half 0: even entries, half 1: odd entries
        const int col = __shfl_sync(0xffffffffu, mcol, kk);
        const double v = __shfl_sync(0xffffffffu, mv, kk);
        const double *xr = X + (int64_t)col * ldx;
#pragma unroll
        for (int g = 0; g < JG; ++g) {
          const int j = hl + 16 * g;
          if (j < p) acc[g] = fma(v, xr[j], acc[g]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < JG; ++g) acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], 16);
    if (half == 0) {
#pragma unroll
      for (int g = 0; g < JG; ++g) {
        const int j = hl + 16 * g;
        if (j >= p) continue;
        double y = acc[g];
        if (mode != MODE_PLAIN) {
          y = alpha * (y - c * Xr[(int64_t)row * ldr + j]);
          if (mode == MODE_RECUR) y -= Yprev[(int64_t)row * ldp + j];
        }
        Ynext[(int64_t)row * ldn + j] = y;
      }
    }
  }
}

// Largest absolute row sum of Y (pattern rows) and of Y^T (transposed rows).
__global__ void __launch_bounds__(NT) k_svt_bounds(const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ t_rowptr,
                                                   const int32_t *__restrict__ t_perm,
                                                   const double *__restrict__ x, int n,
                                                   double *__restrict__ red) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  double rmax = 0.0, cmax = 0.0;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double rs = 0.0, cs = 0.0;
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) rs += fabs(x[e]);
    for (int e = t_rowptr[row] + lane; e < t_rowptr[row + 1]; e += 32) cs += fabs(x[t_perm[e]]);
    rs = warp_sum(rs);
    cs = warp_sum(cs);
    rmax = fmax(rmax, rs);
    cmax = fmax(cmax, cs);
  }
  rmax = block_reduce(rmax, sh, 2);
  cmax = block_reduce(cmax, sh, 2);
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth + 0] = rmax;
    red[blockIdx.x * kRedWidth + 1] = cmax;
  }
}

// a = 0, ub = ||Y||_inf ||Y||_1, b by reading R4 (the a >= 0 start rule when
// there is no previous Ritz value), c and e of the Chebyshev map.
__global__ void __launch_bounds__(NT) k_svt_interval_final(const double *__restrict__ red, int nb,
                                                           const double *__restrict__ theta,
                                                           int p, Params *prm) {
  __shared__ double sh[32];
  double r = 0.0, c = 0.0;
  for (int q = threadIdx.x; q < nb; q += NT) {
    r = fmax(r, red[q * kRedWidth + 0]);
    c = fmax(c, red[q * kRedWidth + 1]);
  }
  r = block_reduce(r, sh, 2);
  c = block_reduce(c, sh, 2);
  if (threadIdx.x != 0) return;
  const double a = 0.0, ub = r * c, eta = prm->eta;
  double b = prm->have_prev ? (1.0 - eta) * theta[p - 1] + eta * a : a + (1.0 - eta) * (ub - a);
  const double g = 1e-3;
  if (!(b - a >= g)) b = a + g;
  prm->a = a;
  prm->b = b;
  prm->ub = ub;
  prm->c = 0.5 * (a + b);
  prm->e = 0.5 * (b - a);
  prm->flags = 0;
}

// w_e = sum_l L[i][l] s_l R[j][l], s_l = (sigma_l - mu)_+ / sigma_l with
// sigma_l = sqrt(theta_l); r_e = m_e - w_e; x_e += tau r_e.  Partial sums:
// sum r^2, sum m x (before the update), sum m^2.
__global__ void __launch_bounds__(NT) k_svt_update(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ mvals, int n, int p, const double *__restrict__ L, int64_t ldl,
    const double *__restrict__ R, int64_t ldr, const double *__restrict__ theta, double mu,
    double tau, double *__restrict__ x, double *__restrict__ red) {
  __shared__ double sl[kMaxP];
  __shared__ double wv[WPB][kMaxP];
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int warps = gridDim.x * WPB;
  // singular values above mu lead (theta is sorted descending)
  int keep = 0;
  for (int l = 0; l < p; ++l) keep += (theta[l] > 0.0 && sqrt(theta[l]) > mu) ? 1 : 0;
  for (int l = threadIdx.x; l < p; l += NT) {
    const double sg = theta[l] > 0.0 ? sqrt(theta[l]) : 0.0;
    sl[l] = sg > mu ? (sg - mu) / sg : 0.0;
  }
  __syncthreads();
  double rr = 0.0, mx = 0.0, mm = 0.0;
  for (int row = blockIdx.x * WPB + w; row < n; row += warps) {
    for (int l = lane; l < keep; l += 32) wv[w][l] = L[(int64_t)row * ldl + l] * sl[l];
    __syncwarp();
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const int col = colind[e];
      double wsum = 0.0;
      for (int l = 0; l < keep; ++l) wsum = fma(wv[w][l], R[(int64_t)col * ldr + l], wsum);
      const double m = mvals[e];
      const double r = m - wsum;
      const double xo = x[e];
      x[e] = fma(tau, r, xo);
      rr = fma(r, r, rr);
      mx = fma(m, xo, mx);
      mm = fma(m, m, mm);
    }
    __syncwarp();
  }
  rr = block_reduce(rr, sh, 0);
  mx = block_reduce(mx, sh, 0);
  mm = block_reduce(mm, sh, 0);
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth + 0] = rr;
    red[blockIdx.x * kRedWidth + 1] = mx;
    red[blockIdx.x * kRedWidth + 2] = mm;
  }
}

__global__ void __launch_bounds__(NT) k_svt_report(const double *__restrict__ red, int nb,
                                                   const double *__restrict__ theta, int p,
                                                   double mu, Params *prm) {
  __shared__ double sh[32];
  double rr = 0.0, mx = 0.0, mm = 0.0;
  for (int q = threadIdx.x; q < nb; q += NT) {
    rr += red[q * kRedWidth + 0];
    mx += red[q * kRedWidth + 1];
    mm += red[q * kRedWidth + 2];
  }
  rr = block_reduce(rr, sh, 0);
  mx = block_reduce(mx, sh, 0);
  mm = block_reduce(mm, sh, 0);
  if (threadIdx.x != 0) return;
  double f = 0.0;
  int svp = 0;
  bool bad = false;
  for (int l = 0; l < p; ++l) {
    const double th = theta[l];
    if (!isfinite(th)) bad = true;
    const double sg = th > 0.0 ? sqrt(th) : 0.0;
    if (sg > mu) {
      f = fma(sg - mu, sg - mu, f);
      ++svp;
    }
  }
  prm->obj = 0.5 * f - mx;
  prm->kkt = mm > 0.0 ? sqrt(rr / mm) : 0.0;
  prm->pinf = sqrt(rr);
  prm->dinf = 0.0;
  prm->gap = 0.0;
  prm->r_plus = svp;
  prm->theta_max = theta[0];
  prm->theta_min = theta[p - 1];
  prm->have_prev = 1;
  if (bad) prm->flags |= 4;
}

__global__ void k_svt_init(const double *__restrict__ mvals, int64_t nnz, double tau,
                           double *__restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] = tau * mvals[e];
}

// ---------------------------------------------------------------------------
// PFNNLS (Sec. 5.2.2): accelerated proximal gradient on
// mu ||X||_* + 1/2 ||P_Omega(X) - b||^2 with X = L diag(s) R^T, the previous
// iterate Lp diag(sp) Rp^T, and G = (1+beta) X - beta Xp - A*(A(Y) - b).
// ---------------------------------------------------------------------------

// beta = (t_prev - 1) / t and the low-rank coefficients of G:
// coef = [(1 + beta) s, -beta sp]  (2p values)
__global__ void k_nnls_coef(const double *__restrict__ fsv, int p, double *__restrict__ coef,
                            Params *prm) {
  const double beta = (prm->nn_tp - 1.0) / prm->nn_t;
  for (int l = threadIdx.x; l < p; l += blockDim.x) {
    coef[l] = (1.0 + beta) * fsv[l];
    coef[p + l] = -beta * fsv[p + l];
  }
  if (threadIdx.x == 0) prm->nn_beta = beta;
}

// r_e = A(Y) - b on Omega with Y = (1 + beta) X - beta Xp; partial sum of
// (x_e - m_e)^2 (the objective's data term at X).
__global__ void __launch_bounds__(NT) k_nnls_resid(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ mvals, int n, int p, const double *__restrict__ fac, int64_t ldf,
    const double *__restrict__ fsv, const Params *__restrict__ prm, double *__restrict__ r,
    double *__restrict__ red) {
  __shared__ double wl[WPB][kMaxP / 2], wp[WPB][kMaxP / 2];
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int warps = gridDim.x * WPB;
  const double beta = prm->nn_beta;
  double dd = 0.0;
  for (int row = blockIdx.x * WPB + w; row < n; row += warps) {
    const double *fr = fac + (int64_t)row * ldf;
    for (int l = lane; l < p; l += 32) {
      wl[w][l] = fr[l] * fsv[l];
      wp[w][l] = fr[p + l] * fsv[p + l];
    }
    __syncwarp();
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const double *fc = fac + (int64_t)colind[e] * ldf;
      double xn = 0.0, xp = 0.0;
      for (int l = 0; l < p; ++l) {
        xn = fma(wl[w][l], fc[2 * p + l], xn);
        xp = fma(wp[w][l], fc[3 * p + l], xp);
      }
      const double m = mvals[e];
      r[e] = (1.0 + beta) * xn - beta * xp - m;
      dd = fma(xn - m, xn - m, dd);
    }
    __syncwarp();
  }
  dd = block_reduce(dd, sh, 0);
  if (threadIdx.x == 0) red[blockIdx.x * kRedWidth] = dd;
}

// Interval on G^T G: a = 0, ub = (max|coef_X| + max|coef_Xp| + sqrt(||r||_1 ||r||_inf))^2.
__global__ void __launch_bounds__(NT) k_nnls_interval_final(const double *__restrict__ red,
                                                            int nb,
                                                            const double *__restrict__ coef,
                                                            const double *__restrict__ theta,
                                                            int p, Params *prm) {
  __shared__ double sh[32];
  double rmax = 0.0, cmax = 0.0;
  for (int q = threadIdx.x; q < nb; q += NT) {
    rmax = fmax(rmax, red[q * kRedWidth + 0]);
    cmax = fmax(cmax, red[q * kRedWidth + 1]);
  }
  rmax = block_reduce(rmax, sh, 2);
  cmax = block_reduce(cmax, sh, 2);
  if (threadIdx.x != 0) return;
  double c1 = 0.0, c2 = 0.0;
  for (int l = 0; l < p; ++l) {
    c1 = fmax(c1, fabs(coef[l]));
    c2 = fmax(c2, fabs(coef[p + l]));
  }
  const double lr = c1 + c2 + sqrt(rmax * cmax);
  const double a = 0.0, ub = lr * lr, eta = prm->eta;
  double b = prm->have_prev ? (1.0 - eta) * theta[p - 1] + eta * a : a + (1.0 - eta) * (ub - a);
  if (!(b - a >= 1e-3)) b = a + 1e-3;
  prm->a = a;
  prm->b = b;
  prm->ub = ub;
  prm->c = 0.5 * (a + b);
  prm->e = 0.5 * (b - a);
  prm->flags = 0;
}

// New factors from the Ritz step: sigma = sqrt(theta+), kept while sigma > mu
// and l < cap; (L, R) move to (Lp, Rp), L = (B Y)[:, l] / sigma_l, R = V.
__global__ void k_nnls_factors(int n, int p, double *__restrict__ fac, int64_t ldf,
                               const double *__restrict__ BY, const double *__restrict__ V,
                               int64_t ldv, const double *__restrict__ theta, int cap,
                               const Params *__restrict__ prm) {
  const double mu = prm->nn_mu;
  const int64_t total = (int64_t)n * p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / p;
    const int l = (int)(idx - i * p);
    double *fr = fac + i * ldf;
    fr[p + l] = fr[l];
    fr[3 * p + l] = fr[2 * p + l];
    const double th = theta[l];
    const double sg = th > 0.0 ? sqrt(th) : 0.0;
    const bool keep = sg > mu && l < cap;
    fr[l] = keep ? BY[i * p + l] / sg : 0.0;
    fr[2 * p + l] = keep ? V[i * ldv + l] : 0.0;
  }
}

// Report and state update: s_new, ||X_new - X||_F / max(1, ||X_new||_F) from
// G1 = L_new^T Lp (in T) and G2 = R_new^T Rp (in gpart), objective
// mu sum s + 1/2 sum (x - m)^2 at X; then (s, sp), t, mu advance.
__global__ void __launch_bounds__(NT) k_nnls_report(const double *__restrict__ G1,
                                                    const double *__restrict__ G2,
                                                    const double *__restrict__ red, int nb,
                                                    const double *__restrict__ theta, int p,
                                                    int cap, double *__restrict__ fsv,
                                                    Params *prm) {
  __shared__ double sh[32];
  __shared__ double snew[kMaxP];
  const double mu = prm->nn_mu;
  for (int l = threadIdx.x; l < p; l += NT) {
    const double th = theta[l];
    const double sg = th > 0.0 ? sqrt(th) : 0.0;
    snew[l] = (sg > mu && l < cap) ? sg - mu : 0.0;
  }
  double dd = 0.0;
  for (int q = threadIdx.x; q < nb; q += NT) dd += red[q * kRedWidth];
  dd = block_reduce(dd, sh, 0);  // also orders the snew writes
  double cross = 0.0;
  for (int idx = threadIdx.x; idx < p * p; idx += NT) {
    const int a = idx / p, b = idx % p;
    cross = fma(snew[a] * fsv[b], G1[idx] * G2[idx], cross);
  }
  cross = block_reduce(cross, sh, 0);
  if (threadIdx.x != 0) return;
  double nn = 0.0, no = 0.0, so = 0.0;
  int svp = 0;
  bool bad = false;
  for (int l = 0; l < p; ++l) {
    nn = fma(snew[l], snew[l], nn);
    no = fma(fsv[l], fsv[l], no);
    so += fsv[l];
    if (snew[l] > 0.0) ++svp;
    if (!isfinite(theta[l])) bad = true;
  }
  const double rel = sqrt(fmax(nn + no - 2.0 * cross, 0.0)) / fmax(1.0, sqrt(nn));
  prm->obj = mu * so + 0.5 * dd;
  prm->kkt = mu <= prm->nn_mubar ? rel : fmax(rel, 1.0);
  prm->pinf = rel;
  prm->dinf = mu;
  prm->gap = 0.0;
  prm->r_plus = svp;
  prm->theta_max = theta[0];
  prm->theta_min = theta[p - 1];
  prm->have_prev = 1;
  if (bad) prm->flags |= 4;
  for (int l = 0; l < p; ++l) {
    fsv[p + l] = fsv[l];
    fsv[l] = snew[l];
  }
  const double t = prm->nn_t;
  prm->nn_tp = t;
  prm->nn_t = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
  prm->nn_mu = fmax(0.7 * mu, prm->nn_mubar);
}

__global__ void __launch_bounds__(NT) k_nnls_init_final(const double *__restrict__ red, int nb,
                                                        double mu0, double mubar_rel, int p,
                                                        double *__restrict__ fsv, Params *prm) {
  __shared__ double sh[32];
  double rmax = 0.0, cmax = 0.0;
  for (int q = threadIdx.x; q < nb; q += NT) {
    rmax = fmax(rmax, red[q * kRedWidth + 0]);
    cmax = fmax(cmax, red[q * kRedWidth + 1]);
  }
  rmax = block_reduce(rmax, sh, 2);
  cmax = block_reduce(cmax, sh, 2);
  for (int l = threadIdx.x; l < 2 * p; l += NT) fsv[l] = 0.0;
  if (threadIdx.x != 0) return;
  const double m0 = mu0 > 0.0 ? mu0 : 0.1 * sqrt(rmax * cmax);
  prm->nn_mu = m0;
  prm->nn_mubar = mubar_rel * m0;
  prm->nn_t = 1.0;
  prm->nn_tp = 1.0;
  prm->nn_beta = 0.0;
}

int row_blocks(int n, int num_sms) {
  int b = (n + WPB - 1) / WPB;
  const int cap = 4 * num_sms < kMaxRedBlocks ? 4 * num_sms : kMaxRedBlocks;
  if (b > cap) b = cap;
  return b < 1 ? 1 : b;
}

double *red_slot(const Workspace &ws, int k) {
  return ws.red + (int64_t)k * kMaxRedBlocks * kRedWidth;
}

}  // namespace

cudaError_t launch_svt_spmm(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                            const int32_t *colind, const double *vals, const int32_t *perm, int n,
                            const double *X, int64_t ldx, const double *Xr, int64_t ldr,
                            const double *Yprev, int64_t ldp, double *Ynext, int64_t ldn,
                            int mode) {
  const int p = ws.p;
  int blocks = (n + WPB - 1) / WPB;
  if (blocks > 8 * ws.num_sms) blocks = 8 * ws.num_sms;
  if (blocks < 1) blocks = 1;
#define PF_SVT_SPMM(JGV)                                                                       \
  k_svt_spmm<JGV><<<blocks, NT, 0, s>>>(rowptr, colind, vals, perm, n, p, X, ldx, Xr, ldr,     \
                                        Yprev, ldp, Ynext, ldn, ws.prm, mode)
  if (p <= 16) { PF_SVT_SPMM(1); }
  else if (p <= 32) { PF_SVT_SPMM(2); }
  else if (p <= 48) { PF_SVT_SPMM(3); }
  else { PF_SVT_SPMM(4); }
#undef PF_SVT_SPMM
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_svt_interval(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                const int32_t *t_rowptr, const int32_t *t_perm, const double *x,
                                int n, const double *theta) {
  const int nb = row_blocks(n, ws.num_sms);
  double *slot = red_slot(ws, SLOT_INTERVAL);
  k_svt_bounds<<<nb, NT, 0, s>>>(rowptr, t_rowptr, t_perm, x, n, slot);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_svt_interval_final<<<1, NT, 0, s>>>(slot, nb, theta, ws.p, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_svt_update(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                              const int32_t *colind, const double *mvals, int n, const double *L,
                              int64_t ldl, const double *R, int64_t ldr, const double *theta,
                              double mu, double tau, double *x) {
  const int nb = row_blocks(n, ws.num_sms);
  double *slot = red_slot(ws, SLOT_SDDMM);
  k_svt_update<<<nb, NT, 0, s>>>(rowptr, colind, mvals, n, ws.p, L, ldl, R, ldr, theta, mu, tau,
                                 x, slot);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_svt_report<<<1, NT, 0, s>>>(slot, nb, theta, ws.p, mu, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_nnls_init(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                             const int32_t *t_rowptr, const int32_t *t_perm, const double *mvals,
                             int n, double mu0, double mubar_rel, double *fsv) {
  const int nb = row_blocks(n, ws.num_sms);
  double *slot = red_slot(ws, SLOT_INTERVAL);
  k_svt_bounds<<<nb, NT, 0, s>>>(rowptr, t_rowptr, t_perm, mvals, n, slot);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nnls_init_final<<<1, NT, 0, s>>>(slot, nb, mu0, mubar_rel, ws.p, fsv, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

// coefficients, residual r = A(Y) - b, its row/column bounds and the interval
cudaError_t launch_nnls_residual(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                 const int32_t *colind, const int32_t *t_rowptr,
                                 const int32_t *t_perm, const double *mvals, int n,
                                 const double *fac, int64_t ldfac, const double *fsv, double *r,
                                 const double *theta) {
  const int p = ws.p;
  k_nnls_coef<<<1, 64, 0, s>>>(fsv, p, ws.resid, ws.prm);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nb = row_blocks(n, ws.num_sms);
  k_nnls_resid<<<nb, NT, 0, s>>>(rowptr, colind, mvals, n, p, fac, ldfac, fsv, ws.prm, r,
                                 red_slot(ws, SLOT_SDDMM));
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double *slot = red_slot(ws, SLOT_INTERVAL);
  k_svt_bounds<<<nb, NT, 0, s>>>(rowptr, t_rowptr, t_perm, r, n, slot);
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nnls_interval_final<<<1, NT, 0, s>>>(slot, nb, ws.resid, theta, p, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

// new factors, the two p x p Grams of the change and the report
cudaError_t launch_nnls_update(cudaStream_t s, const Workspace &ws, int n, double *fac,
                               int64_t ldfac, double *fsv, const double *BY, const double *V,
                               int64_t ldv, const double *theta, int cap) {
  const int p = ws.p;
  int64_t blocks = ((int64_t)n * p + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  if (blocks < 1) blocks = 1;
  k_nnls_factors<<<(int)blocks, 256, 0, s>>>(n, p, fac, ldfac, BY, V, ldv, theta, cap, ws.prm);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int nbg = 0;
  e = launch_gram(s, ws, fac, ldfac, fac + p, ldfac, n, p, p, 0, &nbg);  // L_new^T Lp
  if (e != cudaSuccess) return e;
  e = launch_copy_block(s, ws, ws.gpart, p, p, p, ws.T, p);
  if (e != cudaSuccess) return e;
  e = launch_gram(s, ws, fac + 2 * p, ldfac, fac + 3 * p, ldfac, n, p, p, 0, &nbg);  // R_new^T Rp
  if (e != cudaSuccess) return e;
  const int nb = row_blocks(n, ws.num_sms);
  k_nnls_report<<<1, NT, 0, s>>>(ws.T, ws.gpart, red_slot(ws, SLOT_SDDMM), nb, theta, p, cap, fsv,
                                 ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_svt_init(cudaStream_t s, const Workspace &ws, const double *mvals, int64_t nnz,
                            double tau, double *x) {
  int64_t blocks = (nnz + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  if (blocks < 1) blocks = 1;
  k_svt_init<<<(int)blocks, 256, 0, s>>>(mvals, nnz, tau, x);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
