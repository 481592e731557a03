// Problem-level FP64 kernels: the low-rank + sparse iteration matrix of PSD
// completion, the interval [a, b] of Sec. 4.1, the max-cut DRS update of
// Eqs. (PFAM1)-(PFAM2) with its KKT report, and the completion residual /
// fixed-point report of PFPG (Eqs. (pfpg1)-(pfpg2)).
#include <cuda_bf16.h>

#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int NT = 256;
constexpr int WPB = NT / 32;  // warps per block

// ---------------------------------------------------------------------------
// Low-rank + sparse operator with the Chebyshev epilogue:
//   op(X)_i = sum_l Uf_il T_l. + sscale * sum_e S_e X_{col_e} + shift X_i
//   Ynext   = alpha (op(X) - c X) - beta Yprev   (mode as in the dense path)
// Both sums run in double-float on the FP32 pipe (GB300 runs FP64 at 1/64 of
// FP32): operands as float pairs, products accumulated by the Dot2 scheme
// of Ogita, Rump and Oishi (TwoProduct of the leading parts, TwoSum of the
// running sum, product errors and first-order terms in the low part; within
// a few units of m 2^-48 of sum |x_k y_k| for m terms), two columns per
// packed .f32x2 instruction.
// ---------------------------------------------------------------------------
// The block X (n x p, ldx) as float pairs (df_split), row-major with the even
// row stride pe = p + (p & 1) (a zero pair pads odd p), so that two adjacent
// elements of a row load as one 16-byte vector.
__global__ void k_split_pairs(const double *__restrict__ X, int64_t ldx, int n, int p,
                              float2 *__restrict__ Xs) {
  const int pe = p + (p & 1);
  const int64_t total = (int64_t)n * pe;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / pe;
    const int j = (int)(idx - i * pe);
    Xs[idx] = j < p ? df_split(X[i * ldx + j]) : make_float2(0.f, 0.f);
  }
}

// The block X as column pairs of float pairs: row i holds pc = ceil(p / 2)
// 16-byte groups, group c = (hi(2c), hi(2c + 1), lo(2c), lo(2c + 1)) (zero
// past column p - 1), so that one 16-byte load gives a packed operand pair.
__global__ void k_split_pairs4(const double *__restrict__ X, int64_t ldx, int n, int p,
                               float4 *__restrict__ Xs4) {
  const int pc = (p + 1) >> 1;
  const int64_t total = (int64_t)n * pc;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / pc;
    const int c = (int)(idx - i * pc);
    const float2 u = df_split(X[i * ldx + 2 * c]);
    const float2 v = 2 * c + 1 < p ? df_split(X[i * ldx + 2 * c + 1]) : make_float2(0.f, 0.f);
    Xs4[idx] = make_float4(u.x, v.x, u.y, v.y);
  }
}

// One warp per row, in eight groups of four lanes: lane h of a group covers
// the column pairs c = h, h + 4, ... (JG of them: p <= 8 JG).  Group q takes
// the row's entries q, q + 8, ... (each value split into a pair and scaled
// by sscale as a pair, the gathered row of X as stored column pairs, 16
// bytes per load) and the low-rank terms l = q, q + 8, ... (U_il split, T as
// column pairs in shared memory).  The eight groups' sums combine by a fixed
// xor tree of pair additions, and group q then finishes column pair q + 8k
// of its lanes in FP64 (widening, shift, recurrence, store).
template <int JG>
__global__ void __launch_bounds__(NT) k_lrsp_apply(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ svals, int n, int p, const double *__restrict__ Uf, int64_t lduf,
    int r, const double *__restrict__ T, double sscale, double shift, const double *X, int64_t ldx,
    const double *Yprev, int64_t ldp, double *Ynext, int64_t ldn, const Params *__restrict__ prm,
    int mode, const int32_t *__restrict__ perm, const double *Xr, int64_t ldr,
    const float4 *__restrict__ Xs4) {
  const int pc = (p + 1) >> 1;  // column pairs
  __shared__ float4 Ts[kMaxP * kMaxP / 2];  // T (r x p) as column pairs, r pc groups
  for (int idx = threadIdx.x; idx < r * pc; idx += NT) {
    const int l = idx / pc, c = idx - l * pc;
    const float2 u = df_split(T[l * p + 2 * c]);
    const float2 v = 2 * c + 1 < p ? df_split(T[l * p + 2 * c + 1]) : make_float2(0.f, 0.f);
    Ts[idx] = make_float4(u.x, v.x, u.y, v.y);
  }
  __syncthreads();
  double c = 0.0, alpha = 1.0;
  if (mode != MODE_PLAIN) {
    c = prm->c;
    alpha = (mode == MODE_FIRST ? 1.0 : 2.0) / prm->e;
  }
  const float2 ss = df_split(sscale);
  const int lane = threadIdx.x & 31, gq = lane >> 2, h = lane & 3;
  const int warps = gridDim.x * WPB;
  const double *Xb = Xr != nullptr ? Xr : X;  // the block of the shift and recurrence terms
  const int64_t ldb = Xr != nullptr ? ldr : ldx;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    f2x a1[JG], a2[JG];
#pragma unroll
    for (int g = 0; g < JG; ++g) a1[g] = a2[g] = 0ull;
    if (svals != nullptr) {
      const int e0 = rowptr[row], e1 = rowptr[row + 1];
      for (int base = e0; base < e1; base += 32) {
        const int my = base + lane;
        const int mcol = my < e1 ? colind[my] : 0;
        const float2 mv = df_mul(df_split(my < e1 ? svals[perm != nullptr ? perm[my] : my] : 0.0),
                                 ss);
        const int cnt = min(32, e1 - base);
        for (int k = 0; k < cnt; k += 8) {
          // group q takes entries k + q; past the chunk's end (kk >= cnt,
          // always < 32 here) the source lane holds col 0, value 0
          const int kk = k + gq;
          const int col = __shfl_sync(0xffffffffu, mcol, kk);
          const float v1 = __shfl_sync(0xffffffffu, mv.x, kk);
          const float v2 = __shfl_sync(0xffffffffu, mv.y, kk);
          const f2x V1 = pk2(v1, v1), NV1 = pk2(-v1, -v1), V2 = pk2(v2, v2);
          const float4 *xr = Xs4 + (int64_t)col * pc;
#pragma unroll
          for (int g = 0; g < JG; ++g) {
            const int cp = h + 4 * g;
            if (cp < pc) {
              const float4 x = xr[cp];
              df_fma2(V1, NV1, V2, pk2(x.x, x.y), pk2(x.z, x.w), a1[g], a2[g]);
            }
          }
        }
      }
    }
    if (r > 0) {
      const double *ur = Uf + (int64_t)row * lduf;
      for (int l = gq; l < r; l += 8) {
        const float2 u = df_split(ur[l]);
        const f2x U1 = pk2(u.x, u.x), NU1 = pk2(-u.x, -u.x), U2 = pk2(u.y, u.y);
        const float4 *tr = Ts + l * pc;
#pragma unroll
        for (int g = 0; g < JG; ++g) {
          const int cp = h + 4 * g;
          if (cp < pc) {
            const float4 x = tr[cp];
            df_fma2(U1, NU1, U2, pk2(x.x, x.y), pk2(x.z, x.w), a1[g], a2[g]);
          }
        }
      }
    }
#pragma unroll
    for (int g = 0; g < JG; ++g) {
#pragma unroll
      for (int off = 4; off < 32; off <<= 1) {
        const f2x b1 = shfl_xor2(a1[g], off), b2 = shfl_xor2(a2[g], off);
        df_add2(b1, b2, a1[g], a2[g]);
      }
    }
#pragma unroll
    for (int g = 0; g < JG; ++g) {
      const int cp = h + 4 * g;
      if ((g & 7) != gq || cp >= pc) continue;
      float s1[2], s2[2];
      upk2(a1[g], s1[0], s1[1]);
      upk2(a2[g], s2[0], s2[1]);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int j = 2 * cp + t;
        if (j >= p) break;
        const double o0 = df_widen(s1[t]) + df_widen(s2[t]);
        const double xij = Xb[(int64_t)row * ldb + j];
        const double o = fma(shift, xij, o0);
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

// C_ii and the off-diagonal |C| row sums (one warp per row; the same sums
// in the same order as k_interval_rows).
__global__ void __launch_bounds__(NT) k_maxcut_cdata(const int32_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ colind,
                                                     const double *__restrict__ vals, int n,
                                                     double *__restrict__ cdiag,
                                                     double *__restrict__ crsum) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double dg = 0.0, off = 0.0;
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      const double v = vals[e];
      if (colind[e] == row) dg += v;
      else off += fabs(v);
    }
    dg = warp_sum(dg);
    off = warp_sum(off);
    if (lane == 0) {
      cdiag[row] = dg;
      crsum[row] = off;
    }
  }
}

__global__ void __launch_bounds__(NT) k_interval_final(const double *__restrict__ red, int nb,
                                                       const double *__restrict__ theta, int p,
                                                       Params *prm, int use_lanczos,
                                                       double *__restrict__ zero = nullptr,
                                                       int nzero = 0) {
  __shared__ double sh[32];
  for (int i = threadIdx.x; i < nzero; i += NT) zero[i] = 0.0;
  double a = INFINITY, ubs = -INFINITY;
  for (int q = threadIdx.x; q < nb; q += NT) {
    a = fmin(a, red[q * kRedWidth + 0]);
    ubs = fmax(ubs, red[q * kRedWidth + 1]);
  }
  a = block_reduce(a, sh, 1);
  ubs = block_reduce(ubs, sh, 2);
  if (threadIdx.x != 0) return;
  if (use_lanczos) a = prm->a_lz;
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

__global__ void __launch_bounds__(NT) k_cnorm_final(const double *__restrict__ red, int nb,
                                                    Params *prm) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int q = threadIdx.x; q < nb; q += NT) s += red[q * kRedWidth];
  s = block_reduce(s, sh, 0);
  if (threadIdx.x == 0) prm->Cnorm = sqrt(s);
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
                                                      double *__restrict__ red,
                                                      double *__restrict__ xdiag) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  const double t = prm->t;
  double spinf = 0.0, slam = 0.0, sdl2 = 0.0, sxl = 0.0;
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
    const double zii = Z[(int64_t)row * ldz + row];
    const double l_new = 2.0 * dx - zii - t * cii - 1.0;
    if (lane == 0) {
      // Z_k = X~_{k-1} - tC - Diag(lam_k), so X~_{k-1,ii} = Z_ii + t C_ii + lam_k,i; the
      // diagonal terms of ||Z_k - Z_{k+1}||^2 = ||X~_{k-1} - X~_k - Diag(dl)||^2,
      // dl = lam_k - lam_{k+1}
      const double l_old = lam[row];
      const double dl = l_old - l_new;
      const double dxx = (zii + t * cii + l_old) - dx;
      lam[row] = l_new;
      if (xdiag != nullptr) xdiag[row] = dx;
      spinf = fma(dx - 1.0, dx - 1.0, spinf);
      slam += l_new;
      sdl2 = fma(dl, dl, sdl2);
      sxl = fma(dxx, dl, sxl);
    }
  }
  spinf = block_reduce(spinf, sh, 0);
  slam = block_reduce(slam, sh, 0);
  sdl2 = block_reduce(sdl2, sh, 0);
  sxl = block_reduce(sxl, sh, 0);
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth + 0] = spinf;
    red[blockIdx.x * kRedWidth + 1] = slam;
    red[blockIdx.x * kRedWidth + 2] = sdl2;
    red[blockIdx.x * kRedWidth + 3] = sxl;
  }
}

constexpr int EB = 32;  // expand tile (EB x EB outputs, 2 x 2 per thread)

// Z+ is symmetric (X~, C and Diag(lam) are), so only tiles with ti <= tj are
// computed; an off-diagonal tile is also written to its mirror position
// through shared memory (coalesced transposed store).
template <int PT>
__global__ void __launch_bounds__(NT) k_maxcut_expand(const int32_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ colind,
                                                      const double *__restrict__ vals, int n,
                                                      int p, const double *__restrict__ V,
                                                      int64_t ldv, const double *__restrict__ theta,
                                                      const double *__restrict__ lam, double *Z,
                                                      int64_t ldz, const Params *__restrict__ prm,
                                                      double *__restrict__ red) {
  // one buffer: V rows of the tile (Vi, Vj) during the product, then the
  // staged transpose of the mirror tile (EB x (EB + 1) <= 2 EB (PT + 1))
  static_assert(EB * (EB + 1) <= 2 * EB * (PT + 1), "staging tile must fit the V buffers");
  __shared__ double vbuf[2 * EB * (PT + 1)];
  double(*Vi)[PT + 1] = reinterpret_cast<double(*)[PT + 1]>(vbuf);
  double(*Vj)[PT + 1] = reinterpret_cast<double(*)[PT + 1]>(vbuf + EB * (PT + 1));
  double(*Zs)[EB + 1] = reinterpret_cast<double(*)[EB + 1]>(vbuf);
  __shared__ double Ct[EB][EB + 1];
  __shared__ double sh[32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const double t = prm->t;
  int rp = 0;
  for (int l = 0; l < p; ++l) rp += theta[l] > 0.0 ? 1 : 0;
  const int T = (n + EB - 1) / EB;
  const int64_t ntiles = (int64_t)T * (T + 1) / 2;
  double dsum = 0.0, cx = 0.0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // tile -> (ti, tj) with ti <= tj, row-major over the upper triangle
    int ti = 0;
    int64_t rem = tile;
    while (rem >= T - ti) {
      rem -= T - ti;
      ++ti;
    }
    const int tj = ti + (int)rem;
    const int i0 = ti * EB, j0 = tj * EB;
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
    const bool mirror = ti != tj;
    __syncthreads();  // the V buffers are reused below as the staging tile of the mirror
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int li = ty * 2 + i, gi = i0 + li;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int lj = tx + 16 * j, gj = j0 + lj;
        if (gi >= n || gj >= n) continue;
        const double cij = Ct[li][lj];
        double znew = acc[i][j] - t * cij;
        if (gi == gj) znew -= lam[gi];
        double *zp = Z + (int64_t)gi * ldz + gj;
        const double d = *zp - znew;
        dsum = fma(d, d, dsum);
        cx = fma(cij, acc[i][j], cx);
        *zp = znew;
        if (mirror) {
          Zs[lj][li] = znew;  // staged transpose
          const double dm = Z[(int64_t)gj * ldz + gi] - znew;
          dsum = fma(dm, dm, dsum);
          cx = fma(cij, acc[i][j], cx);
        }
      }
    }
    if (mirror) {
      __syncthreads();
      for (int idx = tid; idx < EB * EB; idx += NT) {
        const int r = idx / EB, c = idx % EB;  // row of the mirror tile = column of this one
        const int gr = j0 + r, gc = i0 + c;
        if (gr < n && gc < n) Z[(int64_t)gr * ldz + gc] = Zs[r][c];
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

// Max-cut report.  dsum = ||Z_k - Z_{k+1}||_F^2 comes either from the
// expansion's entrywise sums (red_exp[0]) or, when G = Vprev^T V is given,
// from the factors: ||X~_{k-1} - X~_k||^2 = sum thp^2 + sum th^2
// - 2 sum_ab thp_a th_b G_ab^2 (positive parts; both bases orthonormal), plus
// the diagonal terms ||dl||^2 - 2 <diag(X~_{k-1} - X~_k), dl> from
// k_maxcut_lambda.  The factor form cancels terms of size ||X~||^2, so it
// carries a relative error of about u ||X~||^2 / ||Z_k - Z_{k+1}||^2.
__global__ void __launch_bounds__(NT) k_maxcut_kkt(const double *__restrict__ red_lam, int nb_lam,
                                                   const double *__restrict__ red_exp, int nb_exp,
                                                   const double *__restrict__ theta, int n, int p,
                                                   Params *prm, const double *__restrict__ gram,
                                                   const double *__restrict__ thp) {
  // eight sums reduced together (one pass through shared memory, in a fixed
  // order): spinf, slam, sdl2, sxl, dsum, cx, cross, and n1 + n2 split as
  // two values below
  constexpr int K = 9;
  __shared__ double sh[NT / 32][K];
  __shared__ int rp_s;
  double v[K] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int q = tid; q < nb_lam; q += NT) {
    v[0] += red_lam[q * kRedWidth + 0];
    v[1] += red_lam[q * kRedWidth + 1];
    v[2] += red_lam[q * kRedWidth + 2];
    v[3] += red_lam[q * kRedWidth + 3];
  }
  for (int q = tid; q < nb_exp; q += NT) {
    v[4] += red_exp[q * kRedWidth + 0];
    v[5] += red_exp[q * kRedWidth + 1];
  }
  if (gram != nullptr) {
    for (int idx = tid; idx < p * p; idx += NT) {
      const int a = idx / p, b = idx % p;
      const double wa = fmax(thp[a], 0.0), wb = fmax(theta[b], 0.0);
      if (wa == 0.0 || wb == 0.0) continue;
      const double m = gram[idx];
      v[6] = fma(wa * wb, m * m, v[6]);
    }
    if (tid < p) {
      const double wa = fmax(thp[tid], 0.0), wb = fmax(theta[tid], 0.0);
      v[7] = wa * wa;
      v[8] = wb * wb;
    }
  }
  if (tid == 0) {
    int rp = 0;
    for (int l = 0; l < p; ++l) rp += theta[l] > 0.0 ? 1 : 0;
    rp_s = rp;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid][k] = v[k];
  __syncthreads();
  if (tid != 0) return;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double a = sh[0][k];
    for (int w = 1; w < NT / 32; ++w) a += sh[w][k];
    v[k] = a;
  }
  const double spinf = v[0], slam = v[1], sdl2 = v[2], sxl = v[3], cx = v[5], cross = v[6];
  double dsum = v[4];
  if (gram != nullptr) dsum = fmax(0.0, (v[7] + v[8] - 2.0 * cross) + sdl2 - 2.0 * sxl);
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
  prm->r_plus = rp_s;
  prm->theta_max = theta[0];
  prm->theta_min = theta[p - 1];
  prm->have_prev = 1;
}

// The first entry of [e0, e1) whose column is >= c (e1 if none), by the
// whole warp (columns sorted within the row): a 32-way search (lane k tests
// entry lo + k step) narrows [lo, hi] until at most 31 entries remain, then
// one ballot over them.
__device__ __forceinline__ int first_col_at_least(const int32_t *__restrict__ colind, int e0,
                                                  int e1, int c, int lane) {
  int lo = e0, hi = e1;  // the answer lies in [lo, hi]
  while (hi - lo > 31) {
    const int step = (hi - lo + 31) / 32;  // >= 1
    const int idx = lo + lane * step;
    const unsigned m = __ballot_sync(0xffffffffu, idx >= hi || colind[idx] >= c);
    if (m == 0u) {  // every tested entry is below c
      lo = lo + 31 * step + 1;
      continue;
    }
    const int f = __ffs(m) - 1;  // tested entry f is >= c (or past the row), f - 1 is not
    if (f > 0) lo = lo + (f - 1) * step + 1;
    hi = min(hi, lo + (f > 0 ? step - 1 : 0));
  }
  const int idx = lo + lane;  // lane 31 is at or past hi
  const unsigned m = __ballot_sync(0xffffffffu, idx >= hi || colind[idx] >= c);
  return lo + (__ffs(m) - 1);
}

// ---------------------------------------------------------------------------
// PSD completion: S = P_Omega(X - M) with X = V diag(max(theta,0)) V^T.
// ---------------------------------------------------------------------------
// S = P_Omega(X - M) with X = V diag(max(theta, 0)) V^T, its squared norm,
// and the Gershgorin row bounds of the step's sparse part -tS - t mu I
// (Sec. 4.1, reading R4) for the interval.  One warp per row, four lanes per
// entry, eight entries per step: lane h takes the term pairs (2c, 2c + 1),
// c = h, h + 4, ... (JP of them), the row's W = V theta+ from shared memory
// and V_col from the stored pairs, 16 bytes per load, in two independent
// Dot2 chains (even and odd terms) on the FP32 pipe; so do s = x - M (M is
// exact in fp32) and the |S| row sums.  S is stored in FP64.
// SYM (a symmetric pattern with the map mirror[e] of each entry to its
// transposed entry): only the entries with col >= row are formed, each
// written to both places (half the dot products; ||S||^2 counts the
// off-diagonal ones twice), and the row bounds come from k_completion_rowbounds.
template <int JP, bool SYM>
__global__ void __launch_bounds__(NT) k_completion_residual(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const float *__restrict__ mvals, int n, int p, const double *__restrict__ V, int64_t ldv,
    const double *__restrict__ theta, const float2 *__restrict__ Vs, double *__restrict__ S,
    double *__restrict__ red, double *__restrict__ red_ivl, const Params *__restrict__ prm,
    const int32_t *__restrict__ mirror, int64_t nnz) {
  __shared__ float4 wv[WPB][kMaxP / 2];  // W as term pairs (hi, lo, hi, lo), zero past r_+
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int warps = gridDim.x * WPB;
  int rp = 0;
  for (int l = 0; l < p; ++l) rp += theta[l] > 0.0 ? 1 : 0;
  const int pe = p + (p & 1), pcr = (rp + 1) >> 1;
  const double t = prm->t, mu = prm->mu;
  float q1 = 0.0f, q2 = 0.0f;  // sum of s^2
  double lo = INFINITY, hi = -INFINITY;
  for (int row = blockIdx.x * WPB + w; row < n; row += warps) {
    for (int c = lane; c < pcr; c += 32) {
      const int j0 = 2 * c, j1 = 2 * c + 1;
      const float2 u = df_split(V[(int64_t)row * ldv + j0] * theta[j0]);
      const float2 v = j1 < rp ? df_split(V[(int64_t)row * ldv + j1] * theta[j1])
                               : make_float2(0.f, 0.f);
      wv[w][c] = make_float4(u.x, u.y, v.x, v.y);
    }
    __syncwarp();
    float o1 = 0.0f, o2 = 0.0f;  // sum of |S_ij|, j != i
    double dg = 0.0;
    const int gq = lane >> 2, gl = lane & 3;
    const int e1 = rowptr[row + 1];
    const int ebeg = SYM ? first_col_at_least(colind, rowptr[row], e1, row, lane) : rowptr[row];
    for (int base = ebeg; base < e1; base += 8) {
      const int e = base + gq;
      const bool valid = e < e1;
      const int col = valid ? colind[e] : 0;
      const float4 *vc = reinterpret_cast<const float4 *>(Vs + (int64_t)col * pe);
      float a1 = 0.0f, a2 = 0.0f, b1 = 0.0f, b2 = 0.0f;
      if (valid) {
#pragma unroll
        for (int k = 0; k < JP; ++k) {
          const int c = gl + 4 * k;
          if (c < pcr) {
            const float4 x = vc[c];
            const float4 wq = wv[w][c];
            df_fma(wq.x, wq.y, x.x, x.y, a1, a2);
            df_fma(wq.z, wq.w, x.z, x.w, b1, b2);
          }
        }
      }
      df_add(b1, b2, a1, a2);
#pragma unroll
      for (int off = 2; off > 0; off >>= 1) {
        const float c1 = __shfl_xor_sync(0xffffffffu, a1, off);
        const float c2 = __shfl_xor_sync(0xffffffffu, a2, off);
        df_add(c1, c2, a1, a2);
      }
      if (!valid || gl != 0) continue;
      // s = (a1 + a2) - M by TwoSum of a1 and -M
      const float m = -mvals[e];
      const float s1 = __fadd_rn(a1, m);
      const float bp = __fsub_rn(s1, a1);
      const float s2 = __fadd_rn(a2, __fadd_rn(__fsub_rn(a1, __fsub_rn(s1, bp)), __fsub_rn(m, bp)));
      const double sv = df_widen(s1) + df_widen(s2);
      S[e] = sv;
      if constexpr (SYM) {
        if (col != row) {
          const int m2 = mirror[e];
          if ((unsigned long long)m2 < (unsigned long long)nnz) S[m2] = sv;
          df_fma(2.0f * s1, 2.0f * s2, s1, s2, q1, q2);  // the entry and its mirror
        } else {
          df_fma(s1, s2, s1, s2, q1, q2);
        }
        continue;
      }
      df_fma(s1, s2, s1, s2, q1, q2);
      if (col == row) {
        dg += sv;
      } else {
        // |s| as a pair (s1 = 0 leaves s = s2)
        const float u1 = s1 != 0.0f ? fabsf(s1) : fabsf(s2);
        const float u2 = s1 != 0.0f ? (s1 < 0.0f ? -s2 : s2) : 0.0f;
        const float tt = __fadd_rn(o1, u1);
        const float b2 = __fsub_rn(tt, o1);
        o2 = __fadd_rn(o2, __fadd_rn(__fadd_rn(__fsub_rn(o1, __fsub_rn(tt, b2)),
                                               __fsub_rn(u1, b2)), u2));
        o1 = tt;
      }
    }
    if constexpr (!SYM) {
      // the row's sums over the warp (pairs by TwoSum, the diagonal is in one lane)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float b1 = __shfl_xor_sync(0xffffffffu, o1, off);
        const float c2 = __shfl_xor_sync(0xffffffffu, o2, off);
        const float tt = __fadd_rn(o1, b1);
        const float bb = __fsub_rn(tt, o1);
        o2 = __fadd_rn(__fadd_rn(o2, c2), __fadd_rn(__fsub_rn(o1, __fsub_rn(tt, bb)), __fsub_rn(b1, bb)));
        o1 = tt;
      }
      const unsigned has = __ballot_sync(0xffffffffu, dg != 0.0);
      dg = has ? __shfl_sync(0xffffffffu, dg, __ffs(has) - 1) : 0.0;
      if (lane == 0) {
        const double d = -t * dg - t * mu, o = t * (df_widen(o1) + df_widen(o2));
        lo = fmin(lo, d - o);
        hi = fmax(hi, d + o);
      }
    }
    __syncwarp();
  }
  double ssq = df_widen(q1) + df_widen(q2);
  ssq = block_reduce(ssq, sh, 0);
  if (!SYM) {
    lo = block_reduce(lo, sh, 1);
    hi = block_reduce(hi, sh, 2);
  }
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth] = ssq;
    if (!SYM) {
      red_ivl[blockIdx.x * kRedWidth + 0] = lo;
      red_ivl[blockIdx.x * kRedWidth + 1] = hi;
    }
  }
}

// The Gershgorin row bounds of -tS - t mu I (Sec. 4.1, reading R4) from the
// stored S (after the symmetric residual): one warp per row, |S_ij| summed as
// float pairs (TwoSum), the diagonal in FP64.  Same grid as the residual
// kernel, so the interval's final reduction reads the same block count.
__global__ void __launch_bounds__(NT) k_completion_rowbounds(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ S, int n, double *__restrict__ red_ivl,
    const Params *__restrict__ prm) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  const double t = prm->t, mu = prm->mu;
  double lo = INFINITY, hi = -INFINITY;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    // four independent pair sums per lane (four loads in flight), combined
    // in a fixed order
    float o1 = 0.0f, o2 = 0.0f;
    float p1[4] = {0.f, 0.f, 0.f, 0.f}, p2[4] = {0.f, 0.f, 0.f, 0.f};
    double dg = 0.0;
    const int e1 = rowptr[row + 1];
    for (int e = rowptr[row] + lane; e < e1; e += 128) {
      double v[4];
      int c[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int ek = e + 32 * k;
        v[k] = ek < e1 ? S[ek] : 0.0;
        c[k] = ek < e1 ? colind[ek] : -1;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (c[k] == row) {
          dg += v[k];
        } else {
          // |v| as a pair: the pair of v with both signs flipped when v < 0
          // (float sign flips; an FP64 fabs would occupy GB300's FP64 pipe)
          const float2 u = df_split(v[k]);
          const float sg = u.x < 0.0f ? -1.0f : 1.0f;
          df_add(sg * u.x, sg * u.y, p1[k], p2[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) df_add(p1[k], p2[k], o1, o2);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float b1 = __shfl_xor_sync(0xffffffffu, o1, off);
      const float c2 = __shfl_xor_sync(0xffffffffu, o2, off);
      const float tt = __fadd_rn(o1, b1);
      const float bb = __fsub_rn(tt, o1);
      o2 = __fadd_rn(__fadd_rn(o2, c2), __fadd_rn(__fsub_rn(o1, __fsub_rn(tt, bb)), __fsub_rn(b1, bb)));
      o1 = tt;
    }
    const unsigned has = __ballot_sync(0xffffffffu, dg != 0.0);
    dg = has ? __shfl_sync(0xffffffffu, dg, __ffs(has) - 1) : 0.0;
    if (lane == 0) {
      const double d = -t * dg - t * mu, o = t * (df_widen(o1) + df_widen(o2));
      lo = fmin(lo, d - o);
      hi = fmax(hi, d + o);
    }
  }
  lo = block_reduce(lo, sh, 1);
  hi = block_reduce(hi, sh, 2);
  if (threadIdx.x == 0) {
    red_ivl[blockIdx.x * kRedWidth + 0] = lo;
    red_ivl[blockIdx.x * kRedWidth + 1] = hi;
  }
}

// Checks a mirror map of a CSR pattern: entry e = (i, j) must map to an
// entry of row j whose column is i.  Sets *bad on any violation (or index
// out of range); one thread per entry, the row of e by binary search.
__global__ void k_mirror_check(const int32_t *__restrict__ rowptr,
                               const int32_t *__restrict__ colind,
                               const int32_t *__restrict__ mirror, int n, int64_t nnz,
                               int *__restrict__ bad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;  // the row i with rowptr[i] <= e < rowptr[i + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (rowptr[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const int i = lo, j = colind[e];
    const int m = mirror[e];
    const bool ok = m >= 0 && (int64_t)m < nnz && j >= 0 && j < n && rowptr[j] <= m &&
                    m < rowptr[j + 1] && colind[m] == i;
    if (!ok) atomicOr(bad, 1);
  }
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
  double ssq = 0.0;
  for (int q = tid; q < nb_s; q += NT) ssq += red_s[q * kRedWidth];
  ssq = block_reduce(ssq, sh, 0);
  if (tid != 0) return;
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
                                        int64_t ldp, double *Ynext, int64_t ldn, int mode,
                                        const double *Xr, int64_t ldr) {
  const int n = op.n, p = ws.p;
  int r = op.r;
  if (op.vals != nullptr) {
    // the block as column pairs of float pairs (rows gathered by column)
    int64_t nb = ((int64_t)n * ((p + 1) / 2) + 255) / 256;
    if (nb > 8 * ws.num_sms) nb = 8 * ws.num_sms;
    k_split_pairs4<<<(int)nb, 256, 0, s>>>(X, ldx, n, p, reinterpret_cast<float4 *>(ws.Xs));
    PF_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (r > 0 && op.Uf != nullptr) {
    int nb = 0;
    const double *Rf = op.Vf != nullptr ? op.Vf : op.Uf;
    const int64_t ldrf = op.Vf != nullptr ? op.ldvf : op.lduf;
    cudaError_t e = launch_gram(s, ws, Rf, ldrf, X, ldx, n, r, p, 0, &nb);
    if (e != cudaSuccess) return e;
    e = launch_lowrank_coef(s, ws, nb, op.lam, r, p, op.clamp);
    if (e != cudaSuccess) return e;
  } else {
    r = 0;
  }
  if (r * ((p + 1) / 2) > kMaxP * kMaxP / 2) return cudaErrorInvalidValue;
  int blocks = (n + WPB - 1) / WPB;
  if (blocks > 8 * ws.num_sms) blocks = 8 * ws.num_sms;
#define PF_LRSP(JGV)                                                                            \
  k_lrsp_apply<JGV><<<blocks, NT, 0, s>>>(op.rowptr, op.colind, op.vals, n, p, op.Uf, op.lduf, r, \
                                          ws.T, op.sscale, op.shift, X, ldx, Yprev, ldp, Ynext,  \
                                          ldn, ws.prm, mode, op.perm, Xr, ldr,                   \
                                          reinterpret_cast<const float4 *>(ws.Xs))
  // JG column pairs per lane, 4 lanes: p <= 8 JG
  switch ((p + 7) / 8) {
    case 1: PF_LRSP(1); break;
    case 2: PF_LRSP(2); break;
    case 3: PF_LRSP(3); break;
    case 4: PF_LRSP(4); break;
    case 5: PF_LRSP(5); break;
    case 6: PF_LRSP(6); break;
    case 7: PF_LRSP(7); break;
    default: PF_LRSP(8); break;
  }
#undef PF_LRSP
  PF_LAUNCHED();
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
  k_interval_final<<<1, NT, 0, s>>>(slot(ws, SLOT_INTERVAL), nb, theta, p, ws.prm, 0);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_interval_rows(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                 const int32_t *colind, const double *vals, int n,
                                 const double *lam) {
  k_interval_rows<<<red_blocks(n, ws.num_sms), NT, 0, s>>>(PF_PROBLEM_MAXCUT, rowptr, colind, vals,
                                                           n, lam, ws.prm, slot(ws, SLOT_INTERVAL));
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_interval_final(cudaStream_t s, const Workspace &ws, int n, const double *theta,
                                  int p, double *zero, int nzero) {
  k_interval_final<<<1, NT, 0, s>>>(slot(ws, SLOT_INTERVAL), red_blocks(n, ws.num_sms), theta, p,
                                    ws.prm, 0, zero, nzero);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_cdata(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                const int32_t *colind, const double *vals, int n) {
  k_maxcut_cdata<<<red_blocks(n, ws.num_sms), NT, 0, s>>>(rowptr, colind, vals, n, ws.oz.cdiag,
                                                          ws.oz.crsum);
  PF_LAUNCHED();
  return cudaGetLastError();
}

// Width growth (Sec. 4.2): columns [p_old, p_new) of U take the guard
// columns of the same index, those of V become zero (the iterate, held by its
// positive Ritz pairs, is unchanged), theta repeats its smallest value.
__global__ void k_grow_block(double *U, int64_t ldu, double *V, int64_t ldv, double *theta, int n,
                             int p_old, int p_new, const double *__restrict__ guard, int64_t ldg) {
  const int w = p_new - p_old;
  const int64_t total = (int64_t)n * w;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / w;
    const int j = p_old + (int)(idx - i * w);
    U[i * ldu + j] = guard[i * ldg + j];
    V[i * ldv + j] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x < w) theta[p_old + threadIdx.x] = theta[p_old - 1];
}

cudaError_t launch_grow_block(cudaStream_t s, const Workspace &ws, double *U, int64_t ldu,
                              double *V, int64_t ldv, double *theta, int n, int p_old, int p_new,
                              const double *guard, int64_t ldg) {
  if (p_old < 1 || p_new <= p_old || p_new > kMaxP) return cudaErrorInvalidValue;
  int64_t blocks = ((int64_t)n * (p_new - p_old) + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  if (blocks < 1) blocks = 1;
  k_grow_block<<<(int)blocks, 256, 0, s>>>(U, ldu, V, ldv, theta, n, p_old, p_new, guard, ldg);
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
  k_cnorm_final<<<1, NT, 0, s>>>(slot(ws, SLOT_MISC), (int)nb, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_update(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                 const int32_t *colind, const double *vals, int n, int p,
                                 const double *V, int64_t ldv, const double *theta, double *Z,
                                 int64_t ldz, double *lam, bool sliced) {
  const int nb1 = red_blocks(n, ws.num_sms);
  cudaError_t e;
  if (sliced) {
    // lam, the report's row sums, the next step's interval bounds and the
    // digit planes of W and V in one pass over the rows
    e = launch_oz_maxcut_rows(s, ws, n, p, V, ldv, theta, Z, ldz, lam, nb1,
                              slot(ws, SLOT_LAMBDA), slot(ws, SLOT_INTERVAL));
    if (e != cudaSuccess) return e;
    // the dual residual from the factors (the previous Ritz pairs were saved
    // to Vprev / thprev at the start of the step), so the expansion writes Z
    // without reading the old one
    int ng = 0;
    e = launch_gram(s, ws, ws.Vprev, p, V, ldv, n, p, p, 0, &ng);
    if (e != cudaSuccess) return e;
    int nbx = 0;
    e = launch_oz_expand(s, ws, rowptr, colind, vals, n, p, V, ldv, theta, lam, Z, ldz,
                         slot(ws, SLOT_EXPAND), &nbx);
    if (e != cudaSuccess) return e;
    k_maxcut_kkt<<<1, NT, 0, s>>>(slot(ws, SLOT_LAMBDA), nb1, slot(ws, SLOT_EXPAND), nbx, theta,
                                  n, p, ws.prm, ws.gpart, ws.thprev);
    PF_LAUNCHED();
    return cudaGetLastError();
  }
  k_maxcut_lambda<<<nb1, NT, 0, s>>>(rowptr, colind, vals, n, p, V, ldv, theta, Z, ldz, lam,
                                     ws.prm, slot(ws, SLOT_LAMBDA), nullptr);
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tiles1 = (n + EB - 1) / EB;
  int64_t nb2 = tiles1 * (tiles1 + 1) / 2;
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
  k_maxcut_kkt<<<1, NT, 0, s>>>(slot(ws, SLOT_LAMBDA), nb1, slot(ws, SLOT_EXPAND), (int)nb2, theta,
                                n, p, ws.prm, nullptr, nullptr);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_completion_residual(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                       const int32_t *colind, const float *mvals, int n, int p,
                                       const double *V, int64_t ldv, const double *theta,
                                       double *S, const int32_t *mirror, int64_t nnz) {
  // V as float pairs (the rows the entries gather), then the entries
  int64_t ns = ((int64_t)n * (p + (p & 1)) + 255) / 256;
  if (ns > 8 * ws.num_sms) ns = 8 * ws.num_sms;
  k_split_pairs<<<(int)ns, 256, 0, s>>>(V, ldv, n, p, ws.Xs);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nb = red_blocks(n, ws.num_sms);
#define PF_RESID(JPV)                                                                          \
  do {                                                                                         \
    if (mirror != nullptr)                                                                     \
      k_completion_residual<JPV, true><<<nb, NT, 0, s>>>(                                      \
          rowptr, colind, mvals, n, p, V, ldv, theta, ws.Xs, S, slot(ws, SLOT_SDDMM),          \
          slot(ws, SLOT_INTERVAL), ws.prm, mirror, nnz);                                       \
    else                                                                                       \
      k_completion_residual<JPV, false><<<nb, NT, 0, s>>>(                                     \
          rowptr, colind, mvals, n, p, V, ldv, theta, ws.Xs, S, slot(ws, SLOT_SDDMM),          \
          slot(ws, SLOT_INTERVAL), ws.prm, nullptr, nnz);                                      \
  } while (0)
  // JP term pairs per lane, 4 lanes per entry: p <= 8 JP
  switch ((p + 7) / 8) {
    case 1: PF_RESID(1); break;
    case 2: PF_RESID(2); break;
    case 3: PF_RESID(3); break;
    case 4: PF_RESID(4); break;
    case 5: PF_RESID(5); break;
    case 6: PF_RESID(6); break;
    case 7: PF_RESID(7); break;
    default: PF_RESID(8); break;
  }
#undef PF_RESID
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess || mirror == nullptr) return e;
  k_completion_rowbounds<<<nb, NT, 0, s>>>(rowptr, colind, S, n, slot(ws, SLOT_INTERVAL), ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_mirror_check(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                const int32_t *colind, const int32_t *mirror, int n, int64_t nnz,
                                int *bad) {
  int64_t nb = (nnz + 255) / 256;
  if (nb > 8 * ws.num_sms) nb = 8 * ws.num_sms;
  if (nb < 1) nb = 1;
  k_mirror_check<<<(int)nb, 256, 0, s>>>(rowptr, colind, mirror, n, nnz, bad);
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

namespace {
__global__ void k_export_info(const Params *__restrict__ prm, pf_iter_info *__restrict__ info,
                              int degree, int precision) {
  if (threadIdx.x != 0) return;
  pf_iter_info r;
  r.a = prm->a;
  r.b = prm->b;
  r.obj = prm->obj;
  r.kkt = prm->kkt;
  r.pinf = prm->pinf;
  r.dinf = prm->dinf;
  r.gap = prm->gap;
  r.theta_max = prm->theta_max;
  r.theta_min = prm->theta_min;
  r.r_plus = prm->r_plus;
  r.flags = prm->flags;
  r.degree = degree;
  r.precision = precision;
  r.jacobi_sweeps = prm->sweeps;
  r.reserved = 0;
  *info = r;
}
}  // namespace

namespace {
// End of a step: count consecutive steps whose positive Ritz count fills the
// block (r_plus >= p - 2) and flag saturation after 20 (flags bit 4).
__global__ void k_step_end(Params *prm, int p) {
  if (threadIdx.x != 0) return;
  const int run = prm->r_plus >= p - 2 ? prm->sat_run + 1 : 0;
  prm->sat_run = run;
  if (run >= 20) prm->flags |= 16;
}
}  // namespace

cudaError_t launch_step_end(cudaStream_t s, const Workspace &ws) {
  k_step_end<<<1, 32, 0, s>>>(ws.prm, ws.p);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_export_info(cudaStream_t s, const Workspace &ws, int degree, int precision) {
  k_export_info<<<1, 32, 0, s>>>(ws.prm, ws.info, degree, precision);
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

// ===========================================================================
// Structured max-cut iteration matrix Z = X~ - tC - Diag(lam), applied without
// forming Z (the update of Eq. (PFAM1) shows Z_{k+1} is exactly this
// low-rank + sparse + diagonal sum).
// ===========================================================================
namespace pf {
namespace {

// S' = -tC - Diag(lam) on C's pattern (C stores every diagonal entry).
__global__ void __launch_bounds__(NT) k_maxcut_sparse_part(const int32_t *__restrict__ rowptr,
                                                           const int32_t *__restrict__ colind,
                                                           const double *__restrict__ vals, int n,
                                                           const double *__restrict__ lam,
                                                           const Params *__restrict__ prm,
                                                           double *__restrict__ Sout) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  const double t = prm->t;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
      double v = -t * vals[e];
      if (colind[e] == row) v -= lam[row];
      Sout[e] = v;
    }
  }
}

// lam_new = 2 diag(X~) - diag(Z) - t diag(C) - 1 with
// diag(Z) = diag(X~prev) - t diag(C) - lam_prev, i.e.
// lam_new = 2 dX - dXprev + lam_prev - 1; plus the KKT partial sums and
// <C, X~> = sum_i sum_l theta+_l V_il (C V)_il.  C is symmetric, so each row
// takes its diagonal entry once and the entries right of it twice; the
// product C V of those entries runs like the SpMM (half-warps alternate
// entries, lanes cover 16 columns each, whole rows of V per entry).
template <int JG>
__global__ void __launch_bounds__(NT) k_maxcut_struct_update(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ vals, int n, int p, const double *__restrict__ V, int64_t ldv,
    const double *__restrict__ theta, const double *__restrict__ Vp, int64_t ldvp,
    const double *__restrict__ thp, double *__restrict__ lam, double *__restrict__ red) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const int warps = gridDim.x * WPB;
  double thpos[JG];
#pragma unroll
  for (int g = 0; g < JG; ++g) {
    const int j = hl + 16 * g;
    thpos[g] = (j < p && theta[j] > 0.0) ? theta[j] : 0.0;
  }
  double s_pinf = 0.0, s_lam = 0.0, s_cross = 0.0, s_d2 = 0.0, s_cx = 0.0;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double dx = 0.0, dxp = 0.0;
    for (int l = lane; l < p; l += 32) {
      const double th = theta[l], tp = thp[l];
      const double v = V[(int64_t)row * ldv + l];
      const double vp = Vp[(int64_t)row * ldvp + l];
      if (th > 0.0) dx = fma(th * v, v, dx);
      if (tp > 0.0) dxp = fma(tp * vp, vp, dxp);
    }
    dx = warp_sum(dx);
    dxp = warp_sum(dxp);
    // first entry at or right of the diagonal (columns sorted)
    int lo = rowptr[row], hi = rowptr[row + 1];
    const int e1 = hi;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (colind[mid] < row) lo = mid + 1;
      else hi = mid;
    }
    double acc[JG];
#pragma unroll
    for (int g = 0; g < JG; ++g) acc[g] = 0.0;
    for (int base = lo; base < e1; base += 32) {
      const int my = base + lane;
      const int mcol = my < e1 ? colind[my] : 0;
      const double mv = my < e1 ? (mcol == row ? vals[my] : 2.0 * vals[my]) : 0.0;
      const int cnt = min(32, e1 - base);
      for (int k = 0; k < cnt; k += 2) {
        const int kk = k + half;  // half 0: even entries, half 1: odd entries
        const int col = __shfl_sync(0xffffffffu, mcol, kk);
        const double v = __shfl_sync(0xffffffffu, mv, kk);
        const double *vr = V + (int64_t)col * ldv;
#pragma unroll
        for (int g = 0; g < JG; ++g) {
          const int j = hl + 16 * g;
          if (j < p) acc[g] = fma(v, vr[j], acc[g]);
        }
      }
    }
    double cx = 0.0;
#pragma unroll
    for (int g = 0; g < JG; ++g) {
      const int j = hl + 16 * g;
      if (j < p) cx = fma(thpos[g] * V[(int64_t)row * ldv + j], acc[g], cx);
    }
    cx = warp_sum(cx);
    if (lane == 0) {
      const double lp = lam[row];
      const double ln = 2.0 * dx - dxp + lp - 1.0;
      const double dl = ln - lp;
      lam[row] = ln;
      s_pinf = fma(dx - 1.0, dx - 1.0, s_pinf);
      s_lam += ln;
      s_cross = fma(dl, dxp - dx, s_cross);
      s_d2 = fma(dl, dl, s_d2);
      s_cx += cx;
    }
  }
  s_pinf = block_reduce(s_pinf, sh, 0);
  s_lam = block_reduce(s_lam, sh, 0);
  s_cross = block_reduce(s_cross, sh, 0);
  s_d2 = block_reduce(s_d2, sh, 0);
  s_cx = block_reduce(s_cx, sh, 0);
  if (threadIdx.x == 0) {
    double *o = red + (int64_t)blockIdx.x * 2 * kRedWidth;
    o[0] = s_pinf;
    o[1] = s_lam;
    o[2] = s_cross;
    o[3] = s_d2;
    o[4] = s_cx;
  }
}

// KKT of the structured update.  ||Z_k - Z_{k+1}||^2 = ||A||^2 + 2 sum dl (A_ii)
// + sum dl^2 with A = X~prev - X~ and ||A||^2 from M = Vprev^T V.
__global__ void __launch_bounds__(NT) k_maxcut_struct_kkt(const double *__restrict__ gpart,
                                                          int nparts,
                                                          const double *__restrict__ red, int nb,
                                                          const double *__restrict__ thp,
                                                          const double *__restrict__ theta, int n,
                                                          int p, Params *prm) {
  __shared__ double sh[32];
  const int tid = threadIdx.x;
  double cross = 0.0;
  for (int idx = tid; idx < p * p; idx += NT) {
    const int a = idx / p, b = idx % p;
    const double wa = fmax(thp[a], 0.0), wb = fmax(theta[b], 0.0);
    if (wa == 0.0 || wb == 0.0) continue;
    double m = 0.0;
    for (int q = 0; q < nparts; ++q) m += gpart[(int64_t)q * p * p + idx];
    cross = fma(wa * wb, m * m, cross);
  }
  cross = block_reduce(cross, sh, 0);
  double s_pinf = 0.0, s_lam = 0.0, s_cr = 0.0, s_d2 = 0.0, s_cx = 0.0;
  for (int q = tid; q < nb; q += NT) {
    const double *o = red + (int64_t)q * 2 * kRedWidth;
    s_pinf += o[0];
    s_lam += o[1];
    s_cr += o[2];
    s_d2 += o[3];
    s_cx += o[4];
  }
  s_pinf = block_reduce(s_pinf, sh, 0);
  s_lam = block_reduce(s_lam, sh, 0);
  s_cr = block_reduce(s_cr, sh, 0);
  s_d2 = block_reduce(s_d2, sh, 0);
  s_cx = block_reduce(s_cx, sh, 0);
  if (tid != 0) return;
  double n1 = 0.0, n2 = 0.0;
  int rp = 0;
  for (int l = 0; l < p; ++l) {
    const double wa = fmax(thp[l], 0.0), wb = fmax(theta[l], 0.0);
    n1 = fma(wa, wa, n1);
    n2 = fma(wb, wb, n2);
    rp += theta[l] > 0.0 ? 1 : 0;
  }
  const double a2 = n1 - 2.0 * cross + n2;
  const double d2 = a2 + 2.0 * s_cr + s_d2;
  const double t = prm->t;
  const double pinf = sqrt(s_pinf) / (1.0 + sqrt((double)n));
  const double dinf = sqrt(fmax(d2, 0.0)) / (t * (1.0 + prm->Cnorm));
  const double pobj = s_cx;
  const double dobj = -s_lam / t;
  const double gap = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
  prm->obj = pobj;
  prm->pinf = pinf;
  prm->dinf = dinf;
  prm->gap = gap;
  prm->kkt = fmax(pinf, fmax(dinf, gap));
  prm->r_plus = rp;
  prm->theta_max = theta[0];
  prm->theta_min = theta[p - 1];
  prm->have_prev = 1;
}

// lam = -t diag(C) - 1 (the state after the DRS step from Z^0 = 0).
__global__ void __launch_bounds__(NT) k_maxcut_init_lam(const int32_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ colind,
                                                        const double *__restrict__ vals, int n,
                                                        double t, double *__restrict__ lam) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    double dg = 0.0;
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32)
      if (colind[e] == row) dg += vals[e];
    dg = warp_sum(dg);
    if (lane == 0) lam[row] = -t * dg - 1.0;
  }
}

// Scale of the low-precision shadow: s >= spectral radius of
// Z = X~ - tC - Diag(lam): Gershgorin of the sparse part plus theta_max.
__global__ void __launch_bounds__(NT) k_lp_scale_final(const double *__restrict__ red, int nb,
                                                       const double *__restrict__ theta,
                                                       Params *prm) {
  __shared__ double sh[32];
  double lo = INFINITY, hi = -INFINITY;
  for (int q = threadIdx.x; q < nb; q += NT) {
    lo = fmin(lo, red[q * kRedWidth + 0]);
    hi = fmax(hi, red[q * kRedWidth + 1]);
  }
  lo = block_reduce(lo, sh, 1);
  hi = block_reduce(hi, sh, 2);
  if (threadIdx.x != 0) return;
  const double thmax = fmax(theta[0], 0.0);
  double s = fmax(fabs(lo), fabs(hi + thmax));
  if (!(s > 0.0) || !isfinite(s)) s = 1.0;
  prm->lp_scale = s;
}

// Dense low-precision shadow Z_lp = (X~ - tC - Diag(lam)) / s, computed in
// fp32 (CUDA cores), tile EL x EL, written as bf16 or fp32.
constexpr int EL = 64;
template <int PT, bool F32OUT>
__global__ void __launch_bounds__(NT) k_maxcut_expand_lp(const int32_t *__restrict__ rowptr,
                                                         const int32_t *__restrict__ colind,
                                                         const double *__restrict__ vals, int n,
                                                         int p, const double *__restrict__ V,
                                                         int64_t ldv,
                                                         const double *__restrict__ theta,
                                                         const double *__restrict__ lam,
                                                         void *Zlp, int64_t ldz,
                                                         const Params *__restrict__ prm) {
  extern __shared__ float dynf[];
  float(*Vi)[PT + 1] = reinterpret_cast<float(*)[PT + 1]>(dynf);
  float(*Vj)[PT + 1] = reinterpret_cast<float(*)[PT + 1]>(dynf + EL * (PT + 1));
  float(*Ct)[EL + 1] = reinterpret_cast<float(*)[EL + 1]>(dynf + 2 * EL * (PT + 1));
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float t = (float)prm->t;
  const float inv_s = (float)(1.0 / prm->lp_scale);
  int rp = 0;
  for (int l = 0; l < p; ++l) rp += theta[l] > 0.0 ? 1 : 0;
  const int tiles1 = (n + EL - 1) / EL;
  const int64_t ntiles = (int64_t)tiles1 * tiles1;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i0 = (int)(tile / tiles1) * EL, j0 = (int)(tile % tiles1) * EL;
    __syncthreads();
    for (int idx = tid; idx < EL * PT; idx += NT) {
      const int r = idx / PT, l = idx % PT;
      const int gi = i0 + r, gj = j0 + r;
      const bool lv = l < rp;
      Vi[r][l] = (lv && gi < n) ? (float)(V[(int64_t)gi * ldv + l] * theta[l]) : 0.f;
      Vj[r][l] = (lv && gj < n) ? (float)V[(int64_t)gj * ldv + l] : 0.f;
    }
    for (int idx = tid; idx < EL * EL; idx += NT) Ct[idx / EL][idx % EL] = 0.f;
    __syncthreads();
    if (tid < EL && i0 + tid < n) {
      const int row = i0 + tid;
      int lo = rowptr[row], hi = rowptr[row + 1];
      const int end = hi;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (colind[mid] < j0) lo = mid + 1;
        else hi = mid;
      }
      for (int e = lo; e < end; ++e) {
        const int col = colind[e];
        if (col >= j0 + EL) break;
        Ct[tid][col - j0] = (float)vals[e];
      }
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int l = 0; l < rp; ++l) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Vi[ty * 4 + i][l];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Vj[tx + 16 * j][l];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int li = ty * 4 + i, gi = i0 + li;
      if (gi >= n) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int lj = tx + 16 * j, gj = j0 + lj;
        if (gj >= n) continue;
        float z = acc[i][j] - t * Ct[li][lj];
        if (gi == gj) z -= (float)lam[gi];
        z *= inv_s;
        if (F32OUT) reinterpret_cast<float *>(Zlp)[(int64_t)gi * ldz + gj] = z;
        else reinterpret_cast<__nv_bfloat16 *>(Zlp)[(int64_t)gi * ldz + gj] = __float2bfloat16_rn(z);
      }
    }
  }
}

constexpr size_t expand_lp_bytes(int PT) {
  return (size_t)(2 * EL * (PT + 1) + EL * (EL + 1)) * sizeof(float);
}

}  // namespace

cudaError_t configure_sparse() {
  cudaError_t e;
#define PF_SET(fn, bytes)                                                                   \
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes)); \
  if (e != cudaSuccess) return e;
  PF_SET((k_maxcut_expand_lp<16, false>), expand_lp_bytes(16))
  PF_SET((k_maxcut_expand_lp<32, false>), expand_lp_bytes(32))
  PF_SET((k_maxcut_expand_lp<64, false>), expand_lp_bytes(64))
  PF_SET((k_maxcut_expand_lp<16, true>), expand_lp_bytes(16))
  PF_SET((k_maxcut_expand_lp<32, true>), expand_lp_bytes(32))
  PF_SET((k_maxcut_expand_lp<64, true>), expand_lp_bytes(64))
#undef PF_SET
  return cudaSuccess;
}

namespace {
__global__ void k_copy_block(const double *__restrict__ src, int64_t lds, int n, int p,
                             double *__restrict__ dst, int64_t ldd) {
  const int64_t total = (int64_t)n * p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / p;
    const int j = (int)(idx - i * p);
    dst[i * ldd + j] = src[i * lds + j];
  }
}
}  // namespace

cudaError_t launch_copy_block(cudaStream_t s, const Workspace &ws, const double *src, int64_t lds,
                              int n, int p, double *dst, int64_t ldd) {
  int64_t blocks = ((int64_t)n * p + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  if (blocks < 1) blocks = 1;
  k_copy_block<<<(int)blocks, 256, 0, s>>>(src, lds, n, p, dst, ldd);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_sparse_part(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                      const int32_t *colind, const double *vals, int n,
                                      const double *lam, double *Sout) {
  k_maxcut_sparse_part<<<red_blocks(n, ws.num_sms), NT, 0, s>>>(rowptr, colind, vals, n, lam,
                                                                  ws.prm, Sout);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_struct_update(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                        const int32_t *colind, const double *vals, int n, int p,
                                        const double *V, int64_t ldv, const double *theta,
                                        double *lam) {
  const int nb = red_blocks(n, ws.num_sms);
  double *red = slot(ws, SLOT_LAMBDA);  // 2 * kRedWidth doubles per block: spans LAMBDA + EXPAND
#define PF_SU(JGV)                                                                           \
  k_maxcut_struct_update<JGV><<<nb, NT, 0, s>>>(rowptr, colind, vals, n, p, V, ldv, theta,      \
                                                ws.Vprev, p, ws.thprev, lam, red)
  if (p <= 16) { PF_SU(1); }
  else if (p <= 32) { PF_SU(2); }
  else if (p <= 48) { PF_SU(3); }
  else { PF_SU(4); }
#undef PF_SU
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int ng = 0;
  e = launch_gram(s, ws, ws.Vprev, p, V, ldv, n, p, p, 0, &ng);
  if (e != cudaSuccess) return e;
  k_maxcut_struct_kkt<<<1, NT, 0, s>>>(ws.gpart, ng, red, nb, ws.thprev, theta, n, p, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_init_lam(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                                   const int32_t *colind, const double *vals, int n, double t,
                                   double *lam) {
  k_maxcut_init_lam<<<red_blocks(n, ws.num_sms), NT, 0, s>>>(rowptr, colind, vals, n, t, lam);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_maxcut_lp_shadow(cudaStream_t s, const Workspace &ws, bool f32out,
                                    const int32_t *rowptr, const int32_t *colind,
                                    const double *vals, int n, int p, const double *V, int64_t ldv,
                                    const double *theta, const double *lam, void *Zlp,
                                    int64_t ldz) {
  // scale from the Gershgorin bounds of -tC - Diag(lam) plus theta_max
  const int nb = red_blocks(n, ws.num_sms);
  k_interval_rows<<<nb, NT, 0, s>>>(PF_PROBLEM_MAXCUT, rowptr, colind, vals, n, lam, ws.prm,
                                    slot(ws, SLOT_MISC));
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_lp_scale_final<<<1, NT, 0, s>>>(slot(ws, SLOT_MISC), nb, theta, ws.prm);
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // tensor-core expansion (tf32 MMA over the r+ <= 64 factors)
  return launch_tc_expand(s, ws, f32out, rowptr, colind, vals, n, V, ldv, theta, lam, Zlp, ldz);
}

// fp32 CUDA-core expansion (the reference form of the tensor-core kernel).
cudaError_t launch_maxcut_lp_shadow_fp32(cudaStream_t s, const Workspace &ws, bool f32out,
                                         const int32_t *rowptr, const int32_t *colind,
                                         const double *vals, int n, int p, const double *V,
                                         int64_t ldv, const double *theta, const double *lam,
                                         void *Zlp, int64_t ldz) {
  const int64_t tiles1 = (n + EL - 1) / EL;
  int64_t blocks = tiles1 * tiles1;
  if (blocks > 8 * ws.num_sms) blocks = 8 * ws.num_sms;
#define PF_EXP(PTV)                                                                             \
  if (f32out)                                                                                   \
    k_maxcut_expand_lp<PTV, true><<<(int)blocks, NT, expand_lp_bytes(PTV), s>>>(                 \
        rowptr, colind, vals, n, p, V, ldv,                                                     \
                                                             theta, lam, Zlp, ldz, ws.prm);     \
  else                                                                                          \
    k_maxcut_expand_lp<PTV, false><<<(int)blocks, NT, expand_lp_bytes(PTV), s>>>(                \
        rowptr, colind, vals, n, p, V, ldv, theta, lam, Zlp, ldz, ws.prm);
  if (p <= 16) { PF_EXP(16) }
  else if (p <= 32) { PF_EXP(32) }
  else { PF_EXP(64) }
#undef PF_EXP
  PF_LAUNCHED();
  return cudaGetLastError();
}

// ===========================================================================
// Nearest correlation estimation (Sec. 5.1): gradient method on the dual
// F(x) = 1/2 ||P_+(G + Diag x)||^2 - 1^T x, grad F = diag(P_+(G + Diag x)) - 1,
// with P_+ taken from the positive Ritz pairs of the filtered subspace.  The
// dense FP64 iteration matrix B = G + Diag(x) lives in the problem's Z; only
// its diagonal changes between iterations.
// ===========================================================================
namespace {

// diag(G), off-diagonal |G| row sums, x^0 = 1 - diag(G), diag(B^0) = 1.
__global__ void __launch_bounds__(NT) k_nce_init(double *Z, int64_t ldz, int n,
                                                 double *__restrict__ gdiag,
                                                 double *__restrict__ rsum,
                                                 double *__restrict__ x,
                                                 double *__restrict__ hist, Params *prm) {
  const int lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) prm->acc_count = hist != nullptr ? 1 : 0;
  const int warps = gridDim.x * WPB;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    const double *zr = Z + (int64_t)row * ldz;
    double s = 0.0;
    for (int j = lane; j < n; j += 32)
      if (j != row) s += fabs(zr[j]);
    s = warp_sum(s);
    if (lane == 0) {
      const double g = zr[row];
      gdiag[row] = g;
      rsum[row] = s;
      x[row] = 1.0 - g;
      if (hist != nullptr) hist[row] = 1.0 - g;
      Z[(int64_t)row * ldz + row] = 1.0;
    }
  }
}

// Gershgorin bounds of B = G + Diag(x): B_ii -/+ rowsum_i (into the interval slot).
__global__ void __launch_bounds__(NT) k_nce_rows(const double *Z, int64_t ldz, int n,
                                                 const double *__restrict__ rsum,
                                                 double *__restrict__ red) {
  __shared__ double sh[32];
  double lo = INFINITY, hi = -INFINITY;
  for (int i = blockIdx.x * NT + threadIdx.x; i < n; i += gridDim.x * NT) {
    const double d = Z[(int64_t)i * ldz + i];
    lo = fmin(lo, d - rsum[i]);
    hi = fmax(hi, d + rsum[i]);
  }
  lo = block_reduce(lo, sh, 1);
  hi = block_reduce(hi, sh, 2);
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth + 0] = lo;
    red[blockIdx.x * kRedWidth + 1] = hi;
  }
}

// g = diag(X~) - 1 with X~ = V diag(max(theta,0)) V^T; x <- x - tau g;
// diag(B) <- diag(G) + x.  Partial sums: sum g^2, sum x (before the step).
__global__ void __launch_bounds__(NT) k_nce_update(double *Z, int64_t ldz, int n, int p,
                                                   const double *__restrict__ V, int64_t ldv,
                                                   const double *__restrict__ theta,
                                                   const double *__restrict__ gdiag,
                                                   double *__restrict__ x, double tau,
                                                   double *__restrict__ red,
                                                   double *__restrict__ hist,
                                                   const Params *__restrict__ prm) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  double *hrow = hist != nullptr ? hist + (int64_t)prm->acc_count * n : nullptr;
  double sg = 0.0, sx = 0.0;
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
    if (lane == 0) {
      const double g = dx - 1.0;
      const double xo = x[row];
      const double xn = xo - tau * g;
      x[row] = xn;
      if (hrow != nullptr) hrow[row] = xn;
      Z[(int64_t)row * ldz + row] = gdiag[row] + xn;
      sg = fma(g, g, sg);
      sx += xo;
    }
  }
  sg = block_reduce(sg, sh, 0);
  sx = block_reduce(sx, sh, 0);
  if (threadIdx.x == 0) {
    red[blockIdx.x * kRedWidth + 0] = sg;
    red[blockIdx.x * kRedWidth + 1] = sx;
  }
}

__global__ void __launch_bounds__(NT) k_nce_report(const double *__restrict__ red, int nb,
                                                   const double *__restrict__ theta, int p,
                                                   int accel, Params *prm) {
  __shared__ double sh[32];
  double sg = 0.0, sx = 0.0;
  for (int q = threadIdx.x; q < nb; q += NT) {
    sg += red[q * kRedWidth + 0];
    sx += red[q * kRedWidth + 1];
  }
  sg = block_reduce(sg, sh, 0);
  sx = block_reduce(sx, sh, 0);
  if (threadIdx.x != 0) return;
  double f = 0.0;
  int rp = 0;
  for (int l = 0; l < p; ++l) {
    const double th = theta[l];
    if (th > 0.0) {
      f = fma(th, th, f);
      ++rp;
    }
  }
  const double gnorm = sqrt(sg);
  if (!(prm->g0 > 0.0)) prm->g0 = gnorm;
  prm->obj = 0.5 * f - sx;
  prm->kkt = prm->g0 > 0.0 ? gnorm / prm->g0 : 0.0;
  prm->pinf = gnorm;  // ||grad F(x_k)|| (absolute), reported in the pinf slot
  prm->dinf = 0.0;
  prm->gap = 0.0;
  prm->r_plus = rp;
  prm->theta_max = theta[0];
  prm->theta_min = theta[p - 1];
  prm->have_prev = 1;
  if (accel) prm->acc_count += 1;
}

// ---------------------------------------------------------------------------
// Lanczos estimate of lambda_min(B), B = G + Diag(x) dense (Sec. 4.1): k
// steps from q_0 = 1/sqrt(n) with full reorthogonalisation (classical
// Gram-Schmidt against every basis vector).  Step j is two launches:
//   k_lz_matvec: beta_{j-1} = ||w_{j-1}|| (each block sums the partials in
//     the same order), q_j = w_{j-1} / beta_{j-1}, y = B q_j - beta_{j-1}
//     q_{j-1}, partials of c_i = q_i^T y for i <= j;
//   k_lz_update: c = Q_j^T y, alpha_j = c_j, w = y - Q_j c, partial ||w||^2.
// lz rows: 0..k-1 = q_j; k = y; k+1 = w.  A zero (or non-finite) beta ends
// the process (lz_m = steps taken); later launches do nothing.
// ---------------------------------------------------------------------------
constexpr int kLzStride = 16;  // partials per block (>= kLanczos)
static_assert(kLanczos <= kLzStride, "Lanczos partial stride");

__device__ __forceinline__ double sum_partials(const double *__restrict__ red, int nb, int stride) {
  double v = 0.0;
  for (int q = 0; q < nb; ++q) v += red[q * stride];
  return v;
}

__global__ void __launch_bounds__(NT) k_lz_matvec(const double *__restrict__ Z, int64_t ldz, int n,
                                                  int j, double *lz,
                                                  const double *__restrict__ wpart, int nbp,
                                                  double *__restrict__ cpart, Params *prm) {
  __shared__ double sh[32];
  __shared__ double s_scale, s_beta;
  double *Q = lz;
  double *y = lz + (int64_t)kLanczos * n;
  const double *w = lz + (int64_t)(kLanczos + 1) * n;
  if (j > 0 && prm->lz_m < j) return;  // ended earlier
  if (threadIdx.x == 0) {
    if (j == 0) {
      s_scale = 1.0 / sqrt((double)n);
      s_beta = 0.0;
      if (blockIdx.x == 0) prm->lz_m = kLanczos;
    } else {
      const double beta = sqrt(sum_partials(wpart, nbp, kRedWidth));
      if (blockIdx.x == 0) prm->lz_beta[j - 1] = beta;
      s_beta = beta;
      s_scale = (beta > 0.0 && isfinite(beta)) ? 1.0 / beta : 0.0;
      if (s_scale == 0.0 && blockIdx.x == 0) prm->lz_m = j;
    }
  }
  __syncthreads();
  const double sc = s_scale, be = s_beta;
  if (sc == 0.0) return;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * WPB;
  double part[kLanczos];
#pragma unroll
  for (int i = 0; i < kLanczos; ++i) part[i] = 0.0;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    const double *zr = Z + (int64_t)row * ldz;
    double acc = 0.0;
    if (j == 0) {
      for (int c = lane; c < n; c += 32) acc += zr[c];
    } else {
      for (int c = lane; c < n; c += 32) acc = fma(zr[c], w[c], acc);
    }
    acc = warp_sum(acc) * sc;
    if (lane == 0) {
      const double q = j == 0 ? sc : w[row] * sc;
      Q[(int64_t)j * n + row] = q;
      double yv = acc;
      if (j > 0) yv -= be * Q[(int64_t)(j - 1) * n + row];
      y[row] = yv;
#pragma unroll
      for (int i = 0; i < kLanczos; ++i) {
        if (i < j) part[i] = fma(Q[(int64_t)i * n + row], yv, part[i]);
        else if (i == j) part[i] = fma(q, yv, part[i]);
      }
    }
  }
  for (int i = 0; i <= j; ++i) {
    const double v = block_reduce(part[i], sh, 0);
    if (threadIdx.x == 0) cpart[blockIdx.x * kLzStride + i] = v;
  }
}

__global__ void __launch_bounds__(NT) k_lz_update(int n, int j, double *lz,
                                                  const double *__restrict__ cpart, int nb,
                                                  double *__restrict__ wpart_out, Params *prm) {
  __shared__ double sh[32];
  __shared__ double s_c[kLanczos];
  if (prm->lz_m <= j) return;
  const double *Q = lz;
  const double *y = lz + (int64_t)kLanczos * n;
  double *w = lz + (int64_t)(kLanczos + 1) * n;
  // c_i: 16 lanes (a half-warp) per coefficient, strided partial sums and a
  // fixed shuffle tree
  if (threadIdx.x < 16 * (j + 1)) {
    const int i = threadIdx.x >> 4, sub = threadIdx.x & 15;
    double c = 0.0;
    for (int b = sub; b < nb; b += 16) c += cpart[b * kLzStride + i];
    for (int off = 8; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffu << (threadIdx.x & 16), c, off);
    if (sub == 0) {
      s_c[i] = c;
      if (blockIdx.x == 0 && i == j) prm->lz_alpha[j] = c;
    }
  }
  __syncthreads();
  double part = 0.0;
  for (int r = blockIdx.x * NT + threadIdx.x; r < n; r += gridDim.x * NT) {
    double v = y[r];
    for (int i = 0; i <= j; ++i) v -= s_c[i] * Q[(int64_t)i * n + r];
    w[r] = v;
    part = fma(v, v, part);
  }
  part = block_reduce(part, sh, 0);
  if (threadIdx.x == 0) wpart_out[blockIdx.x * kRedWidth] = part;
}

// Smallest eigenvalue theta of the m x m Lanczos tridiagonal by bisection on
// the Sturm count, its eigenvector by inverse iteration with the shift just
// below theta (T - sigma I is then positive definite: the LDL^T sweep needs
// no pivoting), and a = theta - beta_{m-1} |s_{m-1}|.
__device__ int sturm_below(const double *al, const double *be, int m, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
    d = (al[i] - x) - (i > 0 ? b2 / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

__global__ void k_lz_final(const double *__restrict__ wpart, int nb, Params *prm) {
  // one warp: the Sturm counts of a multisection round run on all lanes
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  const int m = prm->lz_m;
  double al[16], be[16];
  for (int i = 0; i < m; ++i) al[i] = prm->lz_alpha[i];
  for (int i = 0; i + 1 < m; ++i) be[i] = prm->lz_beta[i];
  double blast;
  if (m == kLanczos) {
    double v = 0.0;
    for (int q = lane; q < nb; q += 32) v += wpart[q * kRedWidth];
    blast = sqrt(warp_sum(v));
  } else {
    blast = prm->lz_beta[m - 1];
  }
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  // multisection for the smallest eigenvalue: the interval [a0, b0] keeps
  // count(a0) = 0 and count(b0) >= 1; each round evaluates 32 interior points
  double a0 = lo, b0 = hi;
  for (int round = 0; round < 24; ++round) {
    const double x = a0 + (b0 - a0) * ((double)(lane + 1) / 33.0);
    const bool inside = x > a0 && x < b0;
    const bool hit = inside && sturm_below(al, be, m, x) >= 1;
    const unsigned hmask = __ballot_sync(0xffffffffu, hit);
    const unsigned imask = __ballot_sync(0xffffffffu, inside);
    if (imask == 0u) break;
    double na = a0, nb2 = b0;
    if (hmask != 0u) {
      const int k = __ffs(hmask) - 1;
      nb2 = __shfl_sync(0xffffffffu, x, k);
      // largest inside point below lane k (its count is 0)
      const unsigned below = imask & ((1u << k) - 1u);
      if (below != 0u) na = __shfl_sync(0xffffffffu, x, 31 - __clz(below));
    } else {
      na = __shfl_sync(0xffffffffu, x, 31 - __clz(imask));
    }
    if (na == a0 && nb2 == b0) break;
    a0 = na;
    b0 = nb2;
  }
  if (lane != 0) return;
  const double theta = b0;
  double s[16];
  double res = 0.0;
  if (m == 1) {
    res = fabs(blast);
  } else {
    const double sigma = theta - 1e-10 * fmax(hi - lo, 1e-300);
    for (int i = 0; i < m; ++i) s[i] = 1.0;
    for (int rep = 0; rep < 3; ++rep) {
      // solve (T - sigma I) z = s by the LDL^T sweep, in place
      double d[16], l[16];
      d[0] = al[0] - sigma;
      for (int i = 1; i < m; ++i) {
        l[i] = be[i - 1] / d[i - 1];
        d[i] = (al[i] - sigma) - l[i] * be[i - 1];
      }
      for (int i = 1; i < m; ++i) s[i] -= l[i] * s[i - 1];
      s[m - 1] /= d[m - 1];
      for (int i = m - 2; i >= 0; --i) s[i] = s[i] / d[i] - l[i + 1] * s[i + 1];
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm = fma(s[i], s[i], nrm);
      nrm = sqrt(nrm);
      for (int i = 0; i < m; ++i) s[i] /= nrm;
    }
    res = fabs(blast) * fabs(s[m - 1]);
  }
  prm->a_lz = theta - res;
}

// ---------------------------------------------------------------------------
// Extrapolation of Sec. 4.3 over the window x_0..x_{l+1} (rows of hist).
// All three kernels are launched every step and act only when the window is
// full, so the step stays one fixed launch sequence (graph-capturable).
// ---------------------------------------------------------------------------

// Partial sums of D^T D (upper triangle, row-major pair order), D_j =
// x_{j+1} - x_j, over this block's rows: out[block][pair].
template <int L1>
__global__ void __launch_bounds__(NT) k_rna_gram(const double *__restrict__ hist, int n,
                                                 const Params *__restrict__ prm,
                                                 double *__restrict__ out) {
  constexpr int NPAIR = L1 * (L1 + 1) / 2;
  if (prm->acc_count != L1 + 1) return;
  __shared__ double sh[32];
  double acc[NPAIR];
#pragma unroll
  for (int q = 0; q < NPAIR; ++q) acc[q] = 0.0;
  for (int r = blockIdx.x * NT + threadIdx.x; r < n; r += gridDim.x * NT) {
    double d[L1];
    double prev = hist[r];
#pragma unroll
    for (int j = 0; j < L1; ++j) {
      const double cur = hist[(int64_t)(j + 1) * n + r];
      d[j] = cur - prev;
      prev = cur;
    }
    int q = 0;
#pragma unroll
    for (int i = 0; i < L1; ++i)
#pragma unroll
      for (int j = i; j < L1; ++j) {
        acc[q] = fma(d[i], d[j], acc[q]);
        ++q;
      }
  }
#pragma unroll
  for (int q = 0; q < NPAIR; ++q) {
    const double v = block_reduce(acc[q], sh, 0);
    if (threadIdx.x == 0) out[blockIdx.x * NPAIR + q] = v;
  }
}

// Fixed-order sum of the partials, M = D^T D + lam tr(D^T D) I, Cholesky
// solve M z = 1, c = z / 1^T z.  acc_go: 1 combine, 2 restart the window from
// the current iterate (non-positive pivot), 0 nothing due.
__global__ void k_rna_solve(const double *__restrict__ part, int nb, int l1, double lam_rel,
                            Params *prm) {
  __shared__ double pair[(PF_MAX_ACCEL + 1) * (PF_MAX_ACCEL + 2) / 2];
  const bool due = prm->acc_count == l1 + 1;
  if (!due) {
    if (threadIdx.x == 0) prm->acc_go = 0;
    return;
  }
  const int npair = l1 * (l1 + 1) / 2;
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += part[b * npair + q];
    pair[q] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double M[PF_MAX_ACCEL + 1][PF_MAX_ACCEL + 1];
  int q = 0;
  double tr = 0.0;
  for (int i = 0; i < l1; ++i)
    for (int j = i; j < l1; ++j) {
      M[i][j] = M[j][i] = pair[q++];
      if (i == j) tr += M[i][i];
    }
  for (int i = 0; i < l1; ++i) M[i][i] += lam_rel * tr;
  // Cholesky M = L L^T in place (lower triangle)
  bool ok = tr > 0.0 && isfinite(tr);
  for (int j = 0; j < l1 && ok; ++j) {
    double dj = M[j][j];
    for (int k = 0; k < j; ++k) dj -= M[j][k] * M[j][k];
    if (!(dj > 0.0)) { ok = false; break; }
    const double ljj = sqrt(dj);
    M[j][j] = ljj;
    for (int i = j + 1; i < l1; ++i) {
      double v = M[i][j];
      for (int k = 0; k < j; ++k) v -= M[i][k] * M[j][k];
      M[i][j] = v / ljj;
    }
  }
  double z[PF_MAX_ACCEL + 1];
  double sz = 0.0;
  if (ok) {
    for (int i = 0; i < l1; ++i) {  // L w = 1
      double v = 1.0;
      for (int k = 0; k < i; ++k) v -= M[i][k] * z[k];
      z[i] = v / M[i][i];
    }
    for (int i = l1 - 1; i >= 0; --i) {  // L^T z = w
      double v = z[i];
      for (int k = i + 1; k < l1; ++k) v -= M[k][i] * z[k];
      z[i] = v / M[i][i];
    }
    for (int i = 0; i < l1; ++i) sz += z[i];
    ok = sz != 0.0 && isfinite(sz);
  }
  if (ok)
    for (int i = 0; i < l1; ++i) prm->acc_c[i] = z[i] / sz;
  prm->acc_go = ok ? 1 : 2;
  prm->acc_count = 1;
}

// x = sum_{i<=l} c_i x_i; diag(B) <- diag(G) + x; the window restarts at x.
__global__ void __launch_bounds__(NT) k_rna_combine(double *__restrict__ hist, int n, int l1,
                                                    double *__restrict__ x, double *Z,
                                                    int64_t ldz,
                                                    const double *__restrict__ gdiag,
                                                    const Params *__restrict__ prm) {
  const int go = prm->acc_go;
  if (go == 0) return;
  double c[PF_MAX_ACCEL + 1];
  for (int i = 0; i < l1; ++i) c[i] = prm->acc_c[i];
  for (int r = blockIdx.x * NT + threadIdx.x; r < n; r += gridDim.x * NT) {
    double xn;
    if (go == 1) {
      xn = 0.0;
      for (int i = 0; i < l1; ++i) xn = fma(c[i], hist[(int64_t)i * n + r], xn);
      x[r] = xn;
      Z[(int64_t)r * ldz + r] = gdiag[r] + xn;
    } else {
      xn = x[r];
    }
    hist[r] = xn;
  }
}

}  // namespace

cudaError_t launch_nce_init(cudaStream_t s, const Workspace &ws, double *Z, int64_t ldz, int n,
                            double *x, double *hist) {
  k_nce_init<<<red_blocks(n, ws.num_sms), NT, 0, s>>>(Z, ldz, n, ws.gdiag, ws.rsum, x, hist,
                                                      ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_nce_interval(cudaStream_t s, const Workspace &ws, const double *Z, int64_t ldz,
                                int n, const double *theta, int p) {
  // Lanczos estimate of the lower end a
  const int nbm = red_blocks(n, ws.num_sms);
  int nbu = (n + NT - 1) / NT;
  if (nbu > 2 * ws.num_sms) nbu = 2 * ws.num_sms;
  // c partials (kLzStride per block) from the start of the reduction array,
  // ||w||^2 partials in the last two slots (no overlap: 4 x 152 x 16 doubles
  // < 4 slots)
  double *apart = ws.red;
  double *wp[2] = {slot(ws, SLOT_RESID), slot(ws, SLOT_MISC)};
  static_assert((size_t)kMaxRedBlocks * kLzStride <= (size_t)SLOT_RESID * kMaxRedBlocks * kRedWidth,
                "Lanczos partials overlap");
  for (int j = 0; j < kLanczos; ++j) {
    k_lz_matvec<<<nbm, NT, 0, s>>>(Z, ldz, n, j, ws.lz, wp[(j + 1) & 1], nbu, apart, ws.prm);
    PF_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_lz_update<<<nbu, NT, 0, s>>>(n, j, ws.lz, apart, nbm, wp[j & 1], ws.prm);
    PF_LAUNCHED();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_lz_final<<<1, 32, 0, s>>>(wp[(kLanczos - 1) & 1], nbu, ws.prm);
  PF_LAUNCHED();
  cudaError_t e0 = cudaGetLastError();
  if (e0 != cudaSuccess) return e0;
  int nb = (n + NT - 1) / NT;
  if (nb > kMaxRedBlocks) nb = kMaxRedBlocks;
  k_nce_rows<<<nb, NT, 0, s>>>(Z, ldz, n, ws.rsum, slot(ws, SLOT_INTERVAL));
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_interval_final<<<1, NT, 0, s>>>(slot(ws, SLOT_INTERVAL), nb, theta, p, ws.prm, 1);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_nce_update(cudaStream_t s, const Workspace &ws, double *Z, int64_t ldz, int n,
                              int p, const double *V, int64_t ldv, const double *theta, double *x,
                              double tau, double *hist, int accel_l, double accel_lam) {
  const int nb = red_blocks(n, ws.num_sms);
  const bool acc = hist != nullptr && accel_l > 0;
  k_nce_update<<<nb, NT, 0, s>>>(Z, ldz, n, p, V, ldv, theta, ws.gdiag, x, tau,
                                 slot(ws, SLOT_LAMBDA), acc ? hist : nullptr, ws.prm);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nce_report<<<1, NT, 0, s>>>(slot(ws, SLOT_LAMBDA), nb, theta, p, acc ? 1 : 0, ws.prm);
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess || !acc) return e;
  // the whole reduction array (every slot) holds the Gram partials: at most
  // 512 blocks x 28 pairs <= kRedSlots * kMaxRedBlocks * kRedWidth doubles
  static_assert(512 * (PF_MAX_ACCEL + 1) * (PF_MAX_ACCEL + 2) / 2 <=
                    kRedSlots * kMaxRedBlocks * kRedWidth,
                "extrapolation partials exceed the reduction array");
  const int l1 = accel_l + 1;
  int gb = (n + NT - 1) / NT;
  if (gb > 512) gb = 512;
  if (gb > 2 * ws.num_sms) gb = 2 * ws.num_sms;
  if (gb < 1) gb = 1;
  switch (l1) {
#define PF_RNA(L)                                                         \
  case L:                                                                 \
    k_rna_gram<L><<<gb, NT, 0, s>>>(hist, n, ws.prm, ws.red);             \
    break;
    PF_RNA(2) PF_RNA(3) PF_RNA(4) PF_RNA(5) PF_RNA(6) PF_RNA(7)
#undef PF_RNA
    default: return cudaErrorInvalidValue;
  }
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rna_solve<<<1, 32, 0, s>>>(ws.red, gb, l1, accel_lam > 0.0 ? accel_lam : 1e-10, ws.prm);
  PF_LAUNCHED();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rna_combine<<<red_blocks(n, ws.num_sms), NT, 0, s>>>(hist, n, l1, x, Z, ldz, ws.gdiag,
                                                          ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
