// Problem-level FP64 kernels: the low-rank + sparse iteration matrix of PSD
// completion, the interval [a, b] of Sec. 4.1, the max-cut DRS update of
// Eqs. (PFAM1)-(PFAM2) with its KKT report, and the completion residual /
// fixed-point report of PFPG (Eqs. (pfpg1)-(pfpg2)).
#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int NT = 256;
constexpr int WPB = NT / 32;  // warps per block

// ---------------------------------------------------------------------------
// Low-rank + sparse operator with the Chebyshev epilogue:
//   op(X)_i = sum_l Uf_il T_l. + sscale * sum_e S_e X_{col_e} + shift X_i
//   Ynext   = alpha (op(X) - c X) - beta Yprev   (mode as in the dense path)
// One warp per row; lanes own columns j = lane, lane + 32.
// ---------------------------------------------------------------------------
template <int JN>
__global__ void __launch_bounds__(NT) k_lrsp_apply(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ svals, int n, int p, const double *__restrict__ Uf, int64_t lduf,
    int r, const double *__restrict__ T, double sscale, double shift, const double *X, int64_t ldx,
    const double *Yprev, int64_t ldp, double *Ynext, int64_t ldn, const Params *__restrict__ prm,
    int mode) {
  __shared__ double Ts[kMaxP * kMaxP];
  for (int idx = threadIdx.x; idx < r * p; idx += NT) Ts[idx] = T[idx];
  __syncthreads();
  double c = 0.0, alpha = 1.0;
  if (mode != MODE_PLAIN) {
    c = prm->c;
    alpha = (mode == MODE_FIRST ? 1.0 : 2.0) / prm->e;
  }
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double acc[JN];
#pragma unroll
    for (int q = 0; q < JN; ++q) acc[q] = 0.0;
    if (svals != nullptr) {
      const int e0 = rowptr[row], e1 = rowptr[row + 1];
      for (int base = e0; base < e1; base += 32) {
        const int my = base + lane;
        const int mcol = my < e1 ? colind[my] : 0;
        const double mv = my < e1 ? svals[my] : 0.0;
        const int cnt = min(32, e1 - base);
        for (int k = 0; k < cnt; ++k) {
          const int col = __shfl_sync(0xffffffffu, mcol, k);
          const double v = __shfl_sync(0xffffffffu, mv, k);
#pragma unroll
          for (int q = 0; q < JN; ++q) {
            const int j = lane + 32 * q;
            if (j < p) acc[q] = fma(v, X[(int64_t)col * ldx + j], acc[q]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < JN; ++q) {
      const int j = lane + 32 * q;
      if (j >= p) continue;
      double lr = 0.0;
      for (int l = 0; l < r; ++l) lr = fma(Uf[(int64_t)row * lduf + l], Ts[l * p + j], lr);
      const double xij = X[(int64_t)row * ldx + j];
      const double o = lr + sscale * acc[q] + shift * xij;
      double y;
      if (mode == MODE_PLAIN) y = o;
      else {
        y = alpha * (o - c * xij);
        if (mode == MODE_RECUR) y -= Yprev[(int64_t)row * ldp + j];
      }
      Ynext[(int64_t)row * ldn + j] = y;
    }
  }
}

// ---------------------------------------------------------------------------
// Interval (Sec. 4.1).  Gershgorin bounds of the sparse/diagonal part D of the
// iteration matrix: max-cut D = -tC - Diag(lam); completion D = -tS - t mu I.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_interval_rows(int kind, const int32_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ colind,
                                                      const double *__restrict__ vals, int n,
                                                      const double *__restrict__ lam,
                                                      const Params *__restrict__ prm,
                                                      double *__restrict__ red) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  const double t = prm->t, mu = prm->mu;
  double lo = INFINITY, hi = -INFINITY;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double dg = 0.0, off = 0.0;
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const double v = vals[e];
      if (colind[e] == row) dg += v;
      else off += fabs(v);
    }
    dg = warp_sum(dg);
    off = warp_sum(off);
    const double d = (kind == PF_PROBLEM_MAXCUT) ? (-t * dg - lam[row]) : (-t * dg - t * mu);
    const double o = t * off;
    lo = fmin(lo, d - o);
    hi = fmax(hi, d + o);
  }
  lo = block_reduce(lo, sh, 1);
  hi = block_reduce(hi, sh, 2);
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth + 0] = lo;
    red[blockIdx.x * kRedWidth + 1] = hi;
  }
}

__global__ void k_interval_final(const double *__restrict__ red, int nb,
                                 const double *__restrict__ theta, int p, Params *prm) {
  if (threadIdx.x != 0) return;
  double a = INFINITY, ubs = -INFINITY;
  for (int q = 0; q < nb; ++q) {
    a = fmin(a, red[q * kRedWidth + 0]);
    ubs = fmax(ubs, red[q * kRedWidth + 1]);
  }
  const int have = prm->have_prev;
  const double thmax = have ? fmax(theta[0], 0.0) : 0.0;
  double ub = fmax(ubs + thmax, 0.0);
  const double eta = prm->eta;
  double b;
  if (!have) b = a < 0.0 ? eta * a : a + (1.0 - eta) * (ub - a);
  else b = (1.0 - eta) * theta[p - 1] + eta * a;
  const double g = 1e-3 * fmax(1.0, fabs(a));
  if (!(b - a >= g)) b = a + g;
  prm->a = a;
  prm->b = b;
  prm->ub = ub;
  prm->c = 0.5 * (a + b);
  prm->e = 0.5 * (b - a);
  prm->flags = 0;
}

// ---------------------------------------------------------------------------
// Max-cut initial state: Z^1 = I - t offdiag(C), lam = -t diag(C) - 1.
// ---------------------------------------------------------------------------
__global__ void k_fill(double *x, int64_t rows, int64_t cols, int64_t ld, double v, int identity) {
  const int64_t total = rows * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / cols, j = idx - i * cols;
    x[i * ld + j] = identity ? (i == j ? 1.0 : 0.0) : v;
  }
}

__global__ void __launch_bounds__(NT) k_maxcut_init_scatter(const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ colind,
                                                            const double *__restrict__ vals, int n,
                                                            double t, double *Z, int64_t ldz,
                                                            double *lam) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double dg = 0.0;
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const int j = colind[e];
      if (j == row) dg += vals[e];
      else Z[(int64_t)row * ldz + j] = -t * vals[e];
    }
    dg = warp_sum(dg);
    if (lane == 0) lam[row] = -t * dg - 1.0;
  }
}

__global__ void __launch_bounds__(NT) k_sumsq(const double *__restrict__ v, int64_t m,
                                              double *__restrict__ red) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < m; i += (int64_t)gridDim.x * NT)
    s = fma(v[i], v[i], s);
  s = block_reduce(s, sh, 0);
  if (threadIdx.x == 0) red[blockIdx.x * kRedWidth] = s;
}

__global__ void k_cnorm_final(const double *__restrict__ red, int nb, Params *prm) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nb; ++q) s += red[q * kRedWidth];
  prm->Cnorm = sqrt(s);
}

// ---------------------------------------------------------------------------
// Max-cut DRS update (Eq. (PFAM1) with the prox of G taken with the minus
// sign): X~ = V diag(max(theta,0)) V^T, lam = diag(2X~ - Z - tC) - 1,
// Z+ = X~ - tC - Diag(lam).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_maxcut_lambda(const int32_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ colind,
                                                      const double *__restrict__ vals, int n,
                                                      int p, const double *__restrict__ V,
                                                      int64_t ldv, const double *__restrict__ theta,
                                                      const double *__restrict__ Z, int64_t ldz,
                                                      double *__restrict__ lam,
                                                      const Params *__restrict__ prm,
                                                      double *__restrict__ red) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  const double t = prm->t;
  double spinf = 0.0, slam = 0.0;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double dx = 0.0;
    for (int l = lane; l < p; l += 32) {
      const double th = theta[l];
      if (th > 0.0) {
        const double v = V[(int64_t)row * ldv + l];
        dx = fma(th * v, v, dx);
      }
    }
    dx = warp_sum(dx);
    double cii = 0.0;
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32)
      if (colind[e] == row) cii += vals[e];
    cii = warp_sum(cii);
    const double l_new = 2.0 * dx - Z[(int64_t)row * ldz + row] - t * cii - 1.0;
    if (lane == 0) {
      lam[row] = l_new;
      spinf = fma(dx - 1.0, dx - 1.0, spinf);
      slam += l_new;
    }
  }
  spinf = block_reduce(spinf, sh, 0);
  slam = block_reduce(slam, sh, 0);
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth + 0] = spinf;
    red[blockIdx.x * kRedWidth + 1] = slam;
  }
}

constexpr int EB = 32;  // expand tile (EB x EB outputs, 2 x 2 per thread)

template <int PT>
__global__ void __launch_bounds__(NT) k_maxcut_expand(const int32_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ colind,
                                                      const double *__restrict__ vals, int n,
                                                      int p, const double *__restrict__ V,
                                                      int64_t ldv, const double *__restrict__ theta,
                                                      const double *__restrict__ lam, double *Z,
                                                      int64_t ldz, const Params *__restrict__ prm,
                                                      double *__restrict__ red) {
  __shared__ double Vi[EB][PT + 1];
  __shared__ double Vj[EB][PT + 1];
  __shared__ double Ct[EB][EB + 1];
  __shared__ double sh[32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const double t = prm->t;
  int rp = 0;
  for (int l = 0; l < p; ++l) rp += theta[l] > 0.0 ? 1 : 0;
  const int tiles1 = (n + EB - 1) / EB;
  const int64_t ntiles = (int64_t)tiles1 * tiles1;
  double dsum = 0.0, cx = 0.0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = (int)(tile / tiles1) * EB, j0 = (int)(tile % tiles1) * EB;
    __syncthreads();
    for (int idx = tid; idx < EB * PT; idx += NT) {
      const int r = idx / PT, l = idx % PT;
      const int gi = i0 + r, gj = j0 + r;
      const bool lv = l < rp;
      Vi[r][l] = (lv && gi < n) ? V[(int64_t)gi * ldv + l] * theta[l] : 0.0;
      Vj[r][l] = (lv && gj < n) ? V[(int64_t)gj * ldv + l] : 0.0;
    }
    for (int idx = tid; idx < EB * EB; idx += NT) Ct[idx / EB][idx % EB] = 0.0;
    __syncthreads();
    if (tid < EB && i0 + tid < n) {
      const int row = i0 + tid;
      int lo = rowptr[row], hi = rowptr[row + 1];
      const int end = hi;
      while (lo < hi) {  // first entry with col >= j0
        const int mid = (lo + hi) >> 1;
        if (colind[mid] < j0) lo = mid + 1;
        else hi = mid;
      }
      for (int e = lo; e < end; ++e) {
        const int col = colind[e];
        if (col >= j0 + EB) break;
        Ct[tid][col - j0] = vals[e];
      }
    }
    __syncthreads();
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int l = 0; l < rp; ++l) {
      const double a0 = Vi[ty * 2][l], a1 = Vi[ty * 2 + 1][l];
      const double b0 = Vj[tx][l], b1 = Vj[tx + 16][l];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int li = ty * 2 + i, gi = i0 + li;
      if (gi >= n) continue;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int lj = tx + 16 * j, gj = j0 + lj;
        if (gj >= n) continue;
        const double cij = Ct[li][lj];
        double znew = acc[i][j] - t * cij;
        if (gi == gj) znew -= lam[gi];
        double *zp = Z + (int64_t)gi * ldz + gj;
        const double d = *zp - znew;
        dsum = fma(d, d, dsum);
        cx = fma(cij, acc[i][j], cx);
        *zp = znew;
      }
    }
  }
  dsum = block_reduce(dsum, sh, 0);
  cx = block_reduce(cx, sh, 0);
  if (tid == 0) {
    red[blockIdx.x * kRedWidth + 0] = dsum;
    red[blockIdx.x * kRedWidth + 1] = cx;
  }
}

__global__ void k_maxcut_kkt(const double *__restrict__ red_lam, int nb_lam,
                             const double *__restrict__ red_exp, int nb_exp,
                             const double *__restrict__ theta, int n, int p, Params *prm) {
  if (threadIdx.x != 0) return;
  double spinf = 0.0, slam = 0.0, dsum = 0.0, cx = 0.0;
  for (int q = 0; q < nb_lam; ++q) {
    spinf += red_lam[q * kRedWidth + 0];
    slam += red_lam[q * kRedWidth + 1];
  }
  for (int q = 0; q < nb_exp; ++q) {
    dsum += red_exp[q * kRedWidth + 0];
    cx += red_exp[q * kRedWidth + 1];
  }
  const double t = prm->t;
  const double pinf = sqrt(spinf) / (1.0 + sqrt((double)n));
  const double dinf = sqrt(dsum) / (t * (1.0 + prm->Cnorm));
  const double pobj = cx;
  const double dobj = -slam / t;
  const double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
  prm->obj = pobj;
  prm->pinf = pinf;
  prm->dinf = dinf;
  prm->gap = gap;
  prm->kkt = fmax(pinf, fmax(dinf, gap));
  int rp = 0;
  for (int l = 0; l < p; ++l) rp += theta[l] > 0.0 ? 1 : 0;
  prm->r_plus = rp;
  prm->theta_max = theta[0];
  prm->theta_min = theta[p - 1];
  prm->have_prev = 1;
}

// ---------------------------------------------------------------------------
// PSD completion: S = P_Omega(X - M) with X = V diag(max(theta,0)) V^T.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_completion_residual(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const float *__restrict__ mvals, int n, int p, const double *__restrict__ V, int64_t ldv,
    const double *__restrict__ theta, double *__restrict__ S, double *__restrict__ red) {
  __shared__ double wv[WPB][kMaxP];
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int warps = gridDim.x * WPB;
  int rp = 0;
  for (int l = 0; l < p; ++l) rp += theta[l] > 0.0 ? 1 : 0;
  double ssq = 0.0;
  for (int row = blockIdx.x * WPB + w; row < n; row += warps) {
    for (int l = lane; l < rp; l += 32) wv[w][l] = V[(int64_t)row * ldv + l] * theta[l];
    __syncwarp();
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const int col = colind[e];
      double x = 0.0;
      for (int l = 0; l < rp; ++l) x = fma(wv[w][l], V[(int64_t)col * ldv + l], x);
      const double s = x - (double)mvals[e];
      S[e] = s;
      ssq = fma(s, s, ssq);
    }
    __syncwarp();
  }
  ssq = block_reduce(ssq, sh, 0);
  if (threadIdx.x == 0) red[blockIdx.x * kRedWidth] = ssq;
}

__global__ void k_save_prev(const double *__restrict__ V, int64_t ldv, const double *theta, int n,
                            int p, double *__restrict__ Vprev, double *__restrict__ thprev) {
  const int64_t total = (int64_t)n * p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / p;
    const int j = (int)(idx - i * p);
    Vprev[idx] = V[i * ldv + j];
    if (idx < p) thprev[idx] = theta[idx];
  }
}

// kkt = ||X_k - X_{k+1}||_F / (1 + ||X_k||_F + t ||S||_F), objective at X_k.
// Uses M = Vprev^T V (Gram partials) and orthonormal Ritz vectors.
__global__ void __launch_bounds__(NT) k_completion_kkt(const double *__restrict__ gpart, int nparts,
                                                       const double *__restrict__ red_s, int nb_s,
                                                       const double *__restrict__ thprev,
                                                       const double *__restrict__ theta, int p,
                                                       Params *prm) {
  __shared__ double sh[32];
  const int tid = threadIdx.x;
  double cross = 0.0;
  for (int idx = tid; idx < p * p; idx += NT) {
    const int a = idx / p, b = idx % p;
    const double wa = fmax(thprev[a], 0.0), wb = fmax(theta[b], 0.0);
    if (wa == 0.0 || wb == 0.0) continue;
    double m = 0.0;
    for (int q = 0; q < nparts; ++q) m += gpart[(int64_t)q * p * p + idx];
    cross = fma(wa * wb, m * m, cross);
  }
  cross = block_reduce(cross, sh, 0);
  if (tid != 0) return;
  double ssq = 0.0;
  for (int q = 0; q < nb_s; ++q) ssq += red_s[q * kRedWidth];
  double n1 = 0.0, n2 = 0.0, tr = 0.0;
  int rp = 0;
  for (int l = 0; l < p; ++l) {
    const double wa = fmax(thprev[l], 0.0), wb = fmax(theta[l], 0.0);
    n1 = fma(wa, wa, n1);
    n2 = fma(wb, wb, n2);
    tr += wa;
    rp += theta[l] > 0.0 ? 1 : 0;
  }
  const double diff2 = n1 - 2.0 * cross + n2;
  const double t = prm->t, mu = prm->mu;
  const double snorm = sqrt(ssq);
  prm->obj = 0.5 * ssq + mu * tr;
  prm->kkt = sqrt(fmax(diff2, 0.0)) / (1.0 + sqrt(n1) + t * snorm);
  prm->pinf = 0.0;
  prm->dinf = 0.0;
  prm->gap = 0.0;
  prm->r_plus = rp;
  prm->theta_max = theta[0];
  prm->theta_min = theta[p - 1];
  prm->have_prev = 1;
}

__global__ void k_params_init(Params *prm, double eta, double t, double mu, int degree,
                              int precision) {
  Params z = {};
  z.eta = eta;
  z.t = t;
  z.mu = mu;
  z.degree = degree;
  z.precision = precision;
  z.a = -1.0;
  z.b = 1.0;
  z.c = 0.0;
  z.e = 1.0;
  *prm = z;
}

int red_blocks(int n, int num_sms) {
  int b = (n + WPB - 1) / WPB;
  const int cap = 4 * num_sms < kMaxRedBlocks ? 4 * num_sms : kMaxRedBlocks;
  if (b > cap) b = cap;
  return b < 1 ? 1 : b;
}

}  // namespace

cudaError_t launch_lowrank_sparse_apply(cudaStream_t s, const Workspace &ws, const Op &op,
                                        const double *X, int64_t ldx, const double *Yprev,
                                        int64_t ldp, double *Ynext, int64_t ldn, int mode) {
  const int n = op.n, p = ws.p;
  int r = op.r;
  if (r > 0 && op.Uf != nullptr) {
    int nb = 0;
    cudaError_t e = launch_gram(s, ws, op.Uf, op.lduf, X, ldx, n, r, p, 0, &nb);
    if (e != cudaSuccess) return e;
    e = launch_lowrank_coef(s, ws, nb, op.lam, r, p, op.clamp);
    if (e != cudaSuccess) return e;
  } else {
    r = 0;
  }
  int blocks = (n + WPB - 1) / WPB;
  if (blocks > 8 * ws.num_sms) blocks = 8 * ws.num_sms;
  if (p <= 32)
    {
      k_lrsp_apply<1><<<blocks, NT, 0, s>>>(op.rowptr, op.colind, op.vals, n, p, op.Uf, op.lduf, r,
                                            ws.T, op.sscale, op.shift, X, ldx, Yprev, ldp, Ynext,
                                            ldn, ws.prm, mode);
      PF_LAUNCHED();
    }
  else
    {
      k_lrsp_apply<2><<<blocks, NT, 0, s>>>(op.rowptr, op.colind, op.vals, n, p, op.Uf, op.lduf, r,
                                            ws.T, op.sscale, op.shift, X, ldx, Yprev, ldp, Ynext,
                                            ldn, ws.prm, mode);
      PF_LAUNCHED();
    }
  return cudaGetLastError();
}

static double *slot(const Workspace &ws, int k) {
  return ws.red + (int64_t)k * kMaxRedBlocks * kRedWidth;
}

cudaError_t launch_interval(cudaStream_t s, const Workspace &ws, int kind, const int32_t *rowptr,
                            const int32_t *colind, const double *vals, int n, const double *lam,
                            const double *theta, int p) {
  const int nb = red_blocks(n, ws.num_sms);
  k_interval_rows<<<nb, NT, 0, s>>>(kind, rowptr, colind, vals, n, lam, ws.prm,
                                    slot(ws, SLOT_INTERVAL));
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_interval_final<<<1, 32, 0, s>>>(slot(ws, SLOT_INTERVAL), nb, theta, p, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_fill(cudaStream_t s, double *x, int64_t rows, int64_t cols, int64_t ld, double v) {
  int64_t blocks = (rows * cols + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_fill<<<(int)blocks, 256, 0, s>>>(x, rows, cols, ld, v, 0);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_init(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                               const int32_t *colind, const double *vals, int n, double t,
                               double *Z, int64_t ldz, double *lam) {
  int64_t blocks = ((int64_t)n * n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_fill<<<(int)blocks, 256, 0, s>>>(Z, n, n, ldz, 0.0, 1);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_maxcut_init_scatter<<<red_blocks(n, ws.num_sms), NT, 0, s>>>(rowptr, colind, vals, n, t, Z,
                                                                   ldz, lam);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_cnorm(cudaStream_t s, const Workspace &ws, const double *vals, int64_t nnz) {
  int64_t nb = (nnz + NT - 1) / NT;
  if (nb > kMaxRedBlocks) nb = kMaxRedBlocks;
  if (nb < 1) nb = 1;
  k_sumsq<<<(int)nb, NT, 0, s>>>(vals, nnz, slot(ws, SLOT_MISC));
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_cnorm_final<<<1, 32, 0, s>>>(slot(ws, SLOT_MISC), (int)nb, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_update(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                 const int32_t *colind, const double *vals, int n, int p,
                                 const double *V, int64_t ldv, const double *theta, double *Z,
                                 int64_t ldz, double *lam) {
  const int nb1 = red_blocks(n, ws.num_sms);
  k_maxcut_lambda<<<nb1, NT, 0, s>>>(rowptr, colind, vals, n, p, V, ldv, theta, Z, ldz, lam,
                                     ws.prm, slot(ws, SLOT_LAMBDA));
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tiles1 = (n + EB - 1) / EB;
  int64_t nb2 = tiles1 * tiles1;
  if (nb2 > kMaxRedBlocks) nb2 = kMaxRedBlocks;
  if (p <= 16)
    {
      k_maxcut_expand<16><<<(int)nb2, NT, 0, s>>>(rowptr, colind, vals, n, p, V, ldv, theta, lam, Z,
                                                  ldz, ws.prm, slot(ws, SLOT_EXPAND));
      PF_LAUNCHED();
    }
  else if (p <= 32)
    {
      k_maxcut_expand<32><<<(int)nb2, NT, 0, s>>>(rowptr, colind, vals, n, p, V, ldv, theta, lam, Z,
                                                  ldz, ws.prm, slot(ws, SLOT_EXPAND));
      PF_LAUNCHED();
    }
  else
    {
      k_maxcut_expand<64><<<(int)nb2, NT, 0, s>>>(rowptr, colind, vals, n, p, V, ldv, theta, lam, Z,
                                                  ldz, ws.prm, slot(ws, SLOT_EXPAND));
      PF_LAUNCHED();
    }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_maxcut_kkt<<<1, 32, 0, s>>>(slot(ws, SLOT_LAMBDA), nb1, slot(ws, SLOT_EXPAND), (int)nb2, theta,
                                n, p, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_completion_residual(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                       const int32_t *colind, const float *mvals, int n, int p,
                                       const double *V, int64_t ldv, const double *theta,
                                       double *S) {
  const int nb = red_blocks(n, ws.num_sms);
  k_completion_residual<<<nb, NT, 0, s>>>(rowptr, colind, mvals, n, p, V, ldv, theta, S,
                                          slot(ws, SLOT_SDDMM));
  PF_LAUNCHED();
  return cudaGetLastError();
}

// The SDDMM block count must match launch_completion_residual's.
cudaError_t launch_completion_kkt(cudaStream_t s, const Workspace &ws, const double *V, int64_t ldv,
                                  const double *theta, int n, int p) {
  int nb = 0;
  cudaError_t e = launch_gram(s, ws, ws.Vprev, p, V, ldv, n, p, p, 0, &nb);
  if (e != cudaSuccess) return e;
  k_completion_kkt<<<1, NT, 0, s>>>(ws.gpart, nb, slot(ws, SLOT_SDDMM), red_blocks(n, ws.num_sms),
                                    ws.thprev, theta, p, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_save_prev(cudaStream_t s, const Workspace &ws, const double *V, int64_t ldv,
                             const double *theta, int n, int p) {
  int64_t blocks = ((int64_t)n * p + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) blocks = 1;
  k_save_prev<<<(int)blocks, 256, 0, s>>>(V, ldv, theta, n, p, ws.Vprev, ws.thprev);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_params_init(cudaStream_t s, Params *prm, double eta, double t, double mu,
                               int degree, int precision) {
  k_params_init<<<1, 1, 0, s>>>(prm, eta, t, mu, degree, precision);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
