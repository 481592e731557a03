// p x p symmetric eigensolve of the Rayleigh-Ritz step (Sec. 2.2, Eq. (RR):
// H = Y Theta Y^T) by parallel cyclic Jacobi on one CTA, in double-float
// arithmetic on the FP32 pipe.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, and a Jacobi round is a
// chain of dependent operations: an FP64 round holds the FP64 pipe for
// dozens of cycles per operation (an FP64 one-CTA version of this kernel
// spent 217 us per call at p = 32, an 8-CTA cluster version 1.3-2.7 ms at
// p = 64).  Here H and the eigenvector matrix are carried as unevaluated
// pairs of floats x = x.h + x.l (about 2^-48 relative, from an exact split
// of each FP64 entry) and every operation of a round runs on the FP32 pipe,
// two lanes at a time where the packed .f32x2 instructions apply.
//   * H is first scaled by an exact power of two so that its largest entry
//     lies in [0.5, 1): float's exponent range then covers every entry that
//     FP64 resolves relative to ||H|| (entries below 1e-30 ||H|| count as
//     zero);
//   * round r of a sweep pairs the indices by the circle method (p/2
//     disjoint pairs, every pair once per sweep);
//   * the rotations are rational in the half-angle tangent u of a
//     single-precision angle (c = (1 - u^2) / (1 + u^2), s = 2u / (1 + u^2)):
//     orthogonal to pair precision whatever u is, annihilating h_kl to about
//     1e-6 of itself, which keeps the quadratic convergence of the sweeps;
//   * a round reads one copy of H and writes the other: one thread per 2 x 2
//     block (i, j >= i) forms J_i^T H_ij J_j and its mirror, other threads
//     rotate the eigenvector rows, and four lanes per pair form the next
//     round's rotations at the same time, from the three entries of the
//     pair's diagonal block that this round produces (computed by those
//     lanes exactly as the block threads compute them): one block barrier
//     per round;
//   * the sweep loop stops when off(H)^2 <= 1e-30 ||H||_F^2 (or after 40
//     sweeps); eigenvalues are sorted descending (ties by index) and
//     returned in FP64, as are the eigenvectors.
#include "pf_internal.cuh"

namespace pf {

namespace {

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// al x + be y for pairs: the leading products exactly (TwoProduct by FMA:
// ne = p - al.h x.h is minus the product's error), their sum exactly
// (TwoSum), the product errors and the first-order terms in float, and the
// fast two-sum to renormalise (exact when |sum| >= |lo|; where the products
// cancel, |sum| < |lo|, its error stays within 2^-24 |lo|, about 2^-48 of the
// products: the accuracy of the pair arithmetic itself).  df_lin2 below runs
// the same operations, in the same order, on two lanes of packed pairs.
__device__ __forceinline__ float2 df_lin(float2 al, float2 x, float2 be, float2 y) {
  const float p1 = __fmul_rn(al.x, x.x), ne1 = __fmaf_rn(-al.x, x.x, p1);
  const float p2 = __fmul_rn(be.x, y.x), ne2 = __fmaf_rn(-be.x, y.x, p2);
  const float sh = __fadd_rn(p1, p2), bp = __fsub_rn(sh, p1);
  const float e3 = __fadd_rn(__fsub_rn(p1, __fsub_rn(sh, bp)), __fsub_rn(p2, bp));
  float lo = __fsub_rn(e3, __fadd_rn(ne1, ne2));
  lo = __fmaf_rn(al.x, x.y, lo);
  lo = __fmaf_rn(al.y, x.x, lo);
  lo = __fmaf_rn(be.x, y.y, lo);
  lo = __fmaf_rn(be.y, y.x, lo);
  const float h = __fadd_rn(sh, lo);
  return make_float2(h, __fsub_rn(lo, __fsub_rn(h, sh)));
}

struct dpair {  // two pairs: lane e is h_e + l_e
  f2x h, l;
};
struct dcoef {  // coefficients of df_lin2: al, be per lane, with -al.h, -be.h
  f2x ah, al, nah, bh, bl, nbh;
};
__device__ __forceinline__ dcoef mk_coef(float2 a0, float2 a1, float2 b0, float2 b1) {
  dcoef c;
  c.ah = pk2(a0.x, a1.x);
  c.al = pk2(a0.y, a1.y);
  c.nah = pk2(-a0.x, -a1.x);
  c.bh = pk2(b0.x, b1.x);
  c.bl = pk2(b0.y, b1.y);
  c.nbh = pk2(-b0.x, -b1.x);
  return c;
}
__device__ __forceinline__ dpair dp_bcast(float2 v) { return {pk2(v.x, v.x), pk2(v.y, v.y)}; }
__device__ __forceinline__ void dp_split(dpair v, float2 &e0, float2 &e1) {
  upk2(v.h, e0.x, e1.x);
  upk2(v.l, e0.y, e1.y);
}
__device__ __forceinline__ dpair df_lin2(const dcoef &c, dpair x, dpair y) {
  const f2x p1 = mul2(c.ah, x.h), ne1 = fma2(c.nah, x.h, p1);
  const f2x p2 = mul2(c.bh, y.h), ne2 = fma2(c.nbh, y.h, p2);
  const f2x sh = add2(p1, p2), bp = sub2(sh, p1);
  const f2x e3 = add2(sub2(p1, sub2(sh, bp)), sub2(p2, bp));
  f2x lo = sub2(e3, add2(ne1, ne2));
  lo = fma2(c.ah, x.l, lo);
  lo = fma2(c.al, x.h, lo);
  lo = fma2(c.bh, y.l, lo);
  lo = fma2(c.bl, y.h, lo);
  const f2x h = add2(sh, lo);
  return {h, sub2(lo, sub2(h, sh))};
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
// The rotation of the pair (k, l) as pairs (c, s): the half-angle tangent
// u = tan(theta / 2) = t / (1 + sqrt(1 + t^2)), t = tan(theta) the smaller
// root of t^2 + 2 tau t - 1 = 0 with tau = (h_ll - h_kk) / (2 h_kl), from the
// hardware's approximate reciprocal and square root (u to a few units of
// 2^-23: the rotation annihilates h_kl to about 1e-6 of itself, and the
// sweeps converge quadratically all the same); then c = (1 - u^2) / (1 + u^2)
// and s = 2u / (1 + u^2) from the exact float u: u^2 exact, the reciprocal
// refined to about 2^-47 by a Newton step and its FMA residual, so that
// c^2 + s^2 = 1 within a few units of 2^-46 whatever u is.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void df_rotation(float2 hkk, float2 hll, float2 hkl, float2 &c,
                                            float2 &s) {
  c = make_float2(1.0f, 0.0f);
  s = make_float2(0.0f, 0.0f);
  const float h32 = hkl.x;
  if (!(fabsf(h32) > 0.5e-17f * (fabsf(hkk.x) + fabsf(hll.x))) || !(fabsf(h32) >= 1e-30f))
    return;
  const float d32 = __fadd_rn(__fsub_rn(hll.x, hkk.x), __fsub_rn(hll.y, hkk.y));
  if (!isfinite(d32)) return;
  const float tau = d32 * rcp_fast(2.0f * h32);
  float t32;
  if (fabsf(tau) > 1e18f) t32 = 0.5f * rcp_fast(tau);
  else t32 = copysignf(rcp_fast(fabsf(tau) + sqrt_fast(fmaf(tau, tau, 1.0f))), tau);
  const float u = t32 * rcp_fast(1.0f + sqrt_fast(fmaf(t32, t32, 1.0f)));  // |u| <= tan(pi/8)
  const float q = __fmul_rn(u, u), qe = __fmaf_rn(u, u, -q);  // u^2 = q + qe
  float dh, dl, nh, nl;
  two_sum(1.0f, q, dh, dl);
  dl = __fadd_rn(dl, qe);
  two_sum(1.0f, -q, nh, nl);
  nl = __fsub_rn(nl, qe);
  float r1 = rcp_fast(dh);
  r1 = __fmaf_rn(r1, __fmaf_rn(-dh, r1, 1.0f), r1);
  const float res = __fmaf_rn(-dl, r1, __fmaf_rn(-dh, r1, 1.0f));  // 1 - (dh + dl) r1
  const float rl = __fmul_rn(r1, res);
  const float rh = __fadd_rn(r1, rl);
  const float2 r = make_float2(rh, __fsub_rn(rl, __fsub_rn(rh, r1)));
  c = df_mul(make_float2(nh, nl), r);
  s = df_mul(make_float2(2.0f * u, 0.0f), r);
}

__device__ __forceinline__ float block_sum_f(float v, float *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  float w = 0.0f;
  for (int i = 0; i < nw; ++i) w += sh[i];  // the same order in every thread
  return w;
}

constexpr int DLD = kMaxP + 1;  // row stride of the pair arrays (float2)
constexpr int kTri = (kMaxP / 2) * (kMaxP / 2 + 1) / 2;

// The round-robin order (circle method over m players, position 0 fixed):
// the player at position pos in round r, the position of player x in round
// r, and the pair of a position (pair i holds positions i and m - 1 - i).
__device__ __forceinline__ int rr_player(int pos, int r, int m) {
  if (pos == 0) return 0;
  const int q = pos - 1 + r;  // < 2 (m - 1)
  return 1 + (q >= m - 1 ? q - (m - 1) : q);
}
__device__ __forceinline__ int rr_pos(int x, int r, int m) {
  if (x == 0) return 0;
  int q = x - 1 - r;  // > -(m - 1)
  if (q < 0) q += m - 1;
  return q + 1;
}

// Entry (x, y) of H' = J^T H J for the rotations of one round (pair arrays
// pk, pl, rotations c, s, flags act), formed exactly as the block phase forms
// it: block (I, J) of the pairs of x and y with I <= J (entry (y, x) of it
// when the pair of x comes after the pair of y), its column of M = B J_J,
// then the row of J_I^T M.
__device__ __forceinline__ float2 rotated_entry(const float2 *__restrict__ H, int p, int m,
                                                int r, int x, int y, const int *pk,
                                                const int *pl, const float2 *cs,
                                                const float2 *sn, const int *act) {
  const int half = m / 2;
  const int px = rr_pos(x, r, m), py = rr_pos(y, r, m);
  int I = px < half ? px : m - 1 - px, J = py < half ? py : m - 1 - py;
  int al = x == pk[I] ? 0 : 1, be = y == pk[J] ? 0 : 1;
  if (I > J) {
    const int t = I;
    I = J;
    J = t;
    const int u = al;
    al = be;
    be = u;
  }
  if (I == J && al != be) {  // a diagonal block's h01 is its h10
    al = 1;
    be = 0;
  }
  const int ki = pk[I], li = pl[I], kj = pk[J], lj = pl[J];
  const bool ri = li < p, rj = lj < p;
  const float2 z = make_float2(0.0f, 0.0f);
  const float2 a = H[ki * DLD + kj];
  const float2 b = rj ? H[ki * DLD + lj] : z;
  const float2 c = ri ? H[li * DLD + kj] : z;
  const float2 d = (ri && rj) ? H[li * DLD + lj] : z;
  if (!act[I] && !act[J]) return al == 0 ? (be == 0 ? a : b) : (be == 0 ? c : d);
  const float2 ci = cs[I], si = sn[I], cj = cs[J], sj = sn[J];
  const float2 m0 = be == 0 ? df_lin(cj, a, df_neg(sj), b) : df_lin(sj, a, cj, b);
  const float2 m1 = be == 0 ? df_lin(cj, c, df_neg(sj), d) : df_lin(sj, c, cj, d);
  return al == 0 ? df_lin(ci, m0, df_neg(si), m1) : df_lin(si, m0, ci, m1);
}

template <int NTH>
__global__ void __launch_bounds__(NTH)
    k_jacobi_df(const double *__restrict__ Hin, int p, double *__restrict__ Yeig,
                double *__restrict__ theta, Params *prm) {
  extern __shared__ float2 dyn2[];
  // two copies of H (a round reads one and writes the other) and the
  // eigenvector rows, kMaxP x DLD pairs each
  float2 *const H0 = dyn2, *const H1 = dyn2 + kMaxP * DLD, *const V = dyn2 + 2 * kMaxP * DLD;
  // the rotations of two rounds: the current one and the next
  __shared__ float2 cs[2][kMaxP / 2], sn[2][kMaxP / 2];
  __shared__ int pk[2][kMaxP / 2], pl[2][kMaxP / 2], act[2][kMaxP / 2];
  // the blocks (i, j >= i) of the upper block triangle, diagonal included
  __shared__ unsigned char tri_i[kTri], tri_j[kTri];
  __shared__ float redf[NTH / 32];
  __shared__ unsigned hmax;
  __shared__ float2 lam_s[kMaxP];
  __shared__ int rank_s[kMaxP];
  const int tid = threadIdx.x;
  const int m = p + (p & 1);  // players (index p is a dummy when p is odd)
  const int half = m / 2;
  const int nb = half * (half + 1) / 2;
  // Roles in a round: threads [0, at) form the next round's rotations (four
  // lanes per pair: three entries of its diagonal block, then the angle);
  // threads [at, vt0) rotate the blocks of H (one block each); threads
  // [vt0, NTH) the eigenvector rows (one row and pair per item).  At p = 32
  // on 512 threads: 64 angle lanes, 136 blocks, 512 row items on 288
  // threads; at p = 64 on 1024: 128 angle lanes, 528 blocks, 2048 row items
  // on 352 threads.
  const int at = ((4 * half + 31) / 32) * 32;
  const int nbt = min(((nb + 31) / 32) * 32, NTH - at - 32);
  const int vt0 = at + nbt;

  if (tid == 0) {
    hmax = 0u;
    int k = 0;
    for (int i = 0; i < half; ++i)
      for (int j = i; j < half; ++j) {
        tri_i[k] = (unsigned char)i;
        tri_j[k] = (unsigned char)j;
        ++k;
      }
  }
  __syncthreads();
  // H_ab + H_ba, scaled by 2^-K so that its largest entry lies in [0.5, 1)
  // (K from the largest exponent field: the high words of non-negative
  // doubles order like their exponents; one shared atomic per warp), which
  // is sym(H) 2^-kexp with kexp = K - 1.  The scaling edits the exponent
  // field (exact; entries that would leave the normal range are below
  // 2^-1022 of the largest and become zero).
  constexpr int NE = (kMaxP * kMaxP + NTH - 1) / NTH;
  double hs[NE];
  unsigned mx = 0u;
#pragma unroll
  for (int t = 0; t < NE; ++t) {
    const int idx = tid + t * NTH;
    hs[t] = 0.0;
    if (idx < p * p) {
      const int a = idx / p, b = idx % p;
      hs[t] = Hin[a * p + b] + Hin[b * p + a];
      mx = max(mx, (unsigned)((unsigned long long)__double_as_longlong(hs[t]) >> 32) & 0x7FFFFFFFu);
    }
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((tid & 31) == 0) atomicMax(&hmax, mx);
  __syncthreads();
  const int ebits = (int)(hmax >> 20);
  const int K = ebits == 0x7FF ? 1 : ebits - 1022;  // in [-1022, 1025]
  const int kexp = K - 1;
#pragma unroll
  for (int t = 0; t < NE; ++t) {
    const int idx = tid + t * NTH;
    if (idx < p * p) {
      const int a = idx / p, b = idx % p;
      const long long bits = __double_as_longlong(hs[t]);
      const int e = (int)((bits >> 52) & 0x7FF);
      double x = hs[t];  // Inf and NaN stay as they are
      if (e != 0x7FF)
        x = (e == 0 || e - K < 1) ? 0.0 : __longlong_as_double(bits - ((long long)K << 52));
      H0[a * DLD + b] = df_split(x);
      V[a * DLD + b] = make_float2(a == b ? 1.0f : 0.0f, 0.0f);
    }
  }
  const int k1 = kexp / 2, k2 = kexp - k1;  // 2^kexp as two normal factors
  // this thread's first eigenvector item (row r, pair i) and its stride
  const int hh = max(half, 1);
  const int vstride = NTH - vt0;
  const int vq = vstride / hh, vr = vstride - vq * hh;
  const int v0 = tid - vt0;
  const int r0 = v0 >= 0 ? v0 / hh : 0, i0 = v0 >= 0 ? v0 - r0 * hh : 0;
  __syncthreads();

  // the rotation of pair i in set b, its angle from the diagonal block
  // (hkk, hll, hkl)
  auto set_pair = [&](int b, int i, int k, int l, bool real, float2 hkk, float2 hll,
                      float2 hkl) {
    float2 c = make_float2(1.0f, 0.0f), sv = make_float2(0.0f, 0.0f);
    if (real) df_rotation(hkk, hll, hkl, c, sv);
    cs[b][i] = c;
    sn[b][i] = sv;
    pk[b][i] = k;
    pl[b][i] = l;
    act[b][i] = (real && sv.x != 0.0f) ? 1 : 0;
  };
  int cur = 0;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
    const float2 *H = cur ? H1 : H0;
    float off = 0.0f, tot = 0.0f;
    for (int idx = tid; idx < p * p; idx += NTH) {
      const int a = idx / p, b = idx % p;
      const float h = H[a * DLD + b].x;
      tot = fmaf(h, h, tot);
      if (a != b) off = fmaf(h, h, off);
    }
    off = block_sum_f(off, redf);
    tot = block_sum_f(tot, redf);
    if (!(off > 1e-30f * tot)) break;  // the same decision in every thread
    // round 0's rotations from H itself
    if (tid < half) {
      int k = rr_player(tid, 0, m), l = rr_player(m - 1 - tid, 0, m);
      if (k > l) {
        const int t = k;
        k = l;
        l = t;
      }
      const bool real = l < p;
      const float2 z = make_float2(0.0f, 0.0f);
      set_pair(0, tid, k, l, real, H[k * DLD + k], real ? H[l * DLD + l] : z,
               real ? H[k * DLD + l] : z);
    }
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      const int b = round & 1;
      H = cur ? H1 : H0;
      float2 *const Hn = cur ? H0 : H1;
      if (tid < at) {
        // the next round's rotations, from the entries this round produces
        // (formed here as the block phase forms them), while the other warps
        // apply this round's: lane q of pair i forms h_kk (q = 0), h_ll
        // (q = 1) or h_kl (q = 2), lane 0 the angle
        const int i = tid >> 2, q = tid & 3;
        const bool on = i < half && round + 1 < m - 1;  // whole groups of four
        int k = 0, l = 0;
        bool real = false;
        float2 h = make_float2(0.0f, 0.0f);
        if (on) {
          k = rr_player(i, round + 1, m);
          l = rr_player(m - 1 - i, round + 1, m);
          if (k > l) {
            const int t = k;
            k = l;
            l = t;
          }
          real = l < p;
          if (real && q < 3)
            h = rotated_entry(H, p, m, round, q == 1 ? l : k, q == 0 ? k : l, pk[b], pl[b],
                              cs[b], sn[b], act[b]);
        }
        const float hl1 = __shfl_down_sync(0xffffffffu, h.x, 1);
        const float hl2 = __shfl_down_sync(0xffffffffu, h.y, 1);
        const float hk1 = __shfl_down_sync(0xffffffffu, h.x, 2);
        const float hk2 = __shfl_down_sync(0xffffffffu, h.y, 2);
        if (on && q == 0)
          set_pair(b ^ 1, i, k, l, real, h, make_float2(hl1, hl2), make_float2(hk1, hk2));
      } else if (tid < vt0) {
        // blocks (i, j >= i) of H' = J^T H J: B = [a b; c d] the block of H,
        // (m00, m01) = a (cj, sj) + b (-sj, cj), (m10, m11) = c (cj, sj) +
        // d (-sj, cj), then (h00, h01) = ci (m00, m01) - si (m10, m11) and
        // (h10, h11) = si (m00, m01) + ci (m10, m11); the strict upper blocks
        // are mirrored, and a pair's diagonal block takes h10 for both of its
        // off-diagonal entries (symmetric to rounding)
        for (int u = tid - at; u < nb; u += nbt) {
          const int i = tri_i[u], j = tri_j[u];
          const int ki = pk[b][i], li = pl[b][i], kj = pk[b][j], lj = pl[b][j];
          const bool ri = li < p, rj = lj < p;  // false: the partner is the dummy
          const float2 z = make_float2(0.0f, 0.0f);
          const float2 a = H[ki * DLD + kj];
          const float2 bb = rj ? H[ki * DLD + lj] : z;
          const float2 cc = ri ? H[li * DLD + kj] : z;
          const float2 d = (ri && rj) ? H[li * DLD + lj] : z;
          float2 h00 = a, h01 = bb, h10 = cc, h11 = d;
          if (act[b][i] || act[b][j]) {
            const float2 ci = cs[b][i], si = sn[b][i], cj = cs[b][j], sj = sn[b][j];
            const float2 nsi = df_neg(si), nsj = df_neg(sj);
            const dcoef cJ = mk_coef(cj, sj, nsj, cj);
            const dpair m0 = df_lin2(cJ, dp_bcast(a), dp_bcast(bb));
            const dpair m1 = df_lin2(cJ, dp_bcast(cc), dp_bcast(d));
            dp_split(df_lin2(mk_coef(ci, ci, nsi, nsi), m0, m1), h00, h01);
            dp_split(df_lin2(mk_coef(si, si, ci, ci), m0, m1), h10, h11);
          }
          Hn[ki * DLD + kj] = h00;
          if (i != j) Hn[kj * DLD + ki] = h00;
          if (ri) {
            Hn[li * DLD + kj] = h10;
            Hn[kj * DLD + li] = h10;  // the mirror, or the diagonal block's h01
          }
          if (rj && i != j) {
            Hn[ki * DLD + lj] = h01;
            Hn[lj * DLD + ki] = h01;
          }
          if (ri && rj) {
            Hn[li * DLD + lj] = h11;
            if (i != j) Hn[lj * DLD + li] = h11;
          }
        }
      } else {
        // eigenvector rows: (v_k, v_l) <- (c v_k - s v_l, s v_k + c v_l)
        int r = r0, i = i0;
        while (r < p) {
          if (act[b][i]) {
            const int k = pk[b][i], l = pl[b][i];
            float2 *vrow = V + r * DLD;
            const float2 c = cs[b][i], sv = sn[b][i];
            float2 ok, ol;
            dp_split(df_lin2(mk_coef(c, sv, df_neg(sv), c), dp_bcast(vrow[k]), dp_bcast(vrow[l])),
                     ok, ol);
            vrow[k] = ok;
            vrow[l] = ol;
          }
          r += vq;
          i += vr;
          if (i >= half) {
            i -= half;
            ++r;
          }
        }
      }
      __syncthreads();
      cur ^= 1;
    }
    sweeps_done = sweep + 1;
  }
  // eigenvalues, descending (ties by index): ranked by their pairs (the pairs
  // are normalised, so (hi, lo) orders like hi + lo), then unscaled
  const float2 *H = cur ? H1 : H0;
  if (tid < p) lam_s[tid] = H[tid * DLD + tid];
  __syncthreads();
  bool bad = false;
  const double g1 = __longlong_as_double((long long)(1023 + k1) << 52);
  const double g2 = __longlong_as_double((long long)(1023 + k2) << 52);
  for (int j = tid; j < p; j += NTH) {
    const float2 lj = lam_s[j];
    if (!isfinite(lj.x) || !isfinite(lj.y)) bad = true;
    int rk = 0;
    for (int i = 0; i < p; ++i) {
      const float2 li = lam_s[i];
      if (li.x > lj.x || (li.x == lj.x && (li.y > lj.y || (li.y == lj.y && i < j)))) ++rk;
    }
    theta[rk] = (df_widen(lj.x) + df_widen(lj.y)) * g1 * g2;
    rank_s[j] = rk;
  }
  __syncthreads();
  for (int idx = tid; idx < p * p; idx += NTH) {
    const int r = idx / p, j = idx % p;
    const float2 v = V[r * DLD + j];
    Yeig[r * p + rank_s[j]] = df_widen(v.x) + df_widen(v.y);
  }
  if (bad) atomicOr(&prm->flags, 4);
  if (tid == 0) prm->sweeps = sweeps_done;
}

constexpr size_t jacobi_df_bytes() { return (size_t)3 * kMaxP * DLD * sizeof(float2); }

}  // namespace

cudaError_t configure_jacobi() {
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_df<512>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)jacobi_df_bytes());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_jacobi_df<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)jacobi_df_bytes());
}

cudaError_t launch_jacobi(cudaStream_t s, const Workspace &ws, const double *H, int p,
                          double *theta) {
  // 512 threads up to p = 32, 1024 above (the blocks of H alone are 528 at p = 64)
  if (p <= 32) k_jacobi_df<512><<<1, 512, jacobi_df_bytes(), s>>>(H, p, ws.Yeig, theta, ws.prm);
  else k_jacobi_df<1024><<<1, 1024, jacobi_df_bytes(), s>>>(H, p, ws.Yeig, theta, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
