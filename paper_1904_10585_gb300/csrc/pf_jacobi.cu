// p x p symmetric eigensolve of the Rayleigh-Ritz step (Sec. 2.2, Eq. (RR):
// H = Y Theta Y^T) by parallel cyclic Jacobi on a thread-block cluster.
//
// On GB300 a single SM executes about 4 FP64 flop per clock, so a one-block
// Jacobi at p = 64 spends milliseconds per call.  Here the 8 CTAs of a
// cluster share the rotation work of every round:
//   * each CTA keeps a full replica of H (double-buffered in shared memory)
//     and computes all p/2 rotation angles of the round redundantly (the
//     replicas are bitwise identical, so every CTA takes the same branches);
//   * CTA c computes the new rows of H' = J^T H J for its share of the
//     rotation pairs (2 x 2 blocks J_i^T H_ij J_j) and stores them into the
//     next buffer of every CTA of the cluster (distributed shared memory);
//   * CTA c owns a slice of rows of the eigenvector matrix and applies all
//     rotations to it locally;
//   * one cluster barrier per round orders the exchange.
// The sweep loop stops when off(H) <= 1e-15 ||H||_F (or after 40 sweeps);
// eigenvalues are sorted descending (ties by index).
#include <cooperative_groups.h>

#include "pf_internal.cuh"

namespace cg = cooperative_groups;

namespace pf {

namespace {

// 1/x and 1/sqrt(x) in FP64 by Newton-Raphson refinement of a single-precision
// seed (y <- y + y (1 - x y) for 1/x, y <- y + (y/2)(1 - x y^2) for 1/sqrt(x));
// each step doubles the correct bits (24 -> 48 -> full precision).  On GB300
// the FP64 pipe is 1/64 of FP32, and these short FMA chains replace the much
// longer IEEE divide and square-root sequences on the rotation-angle path.
__device__ __forceinline__ double nr_rcp(double x) {
  int e;
  const double m = frexp(x, &e);  // x = m 2^e, 0.5 <= |m| < 1
  double y = (double)__frcp_rn((float)m);
  y = fma(y, fma(-m, y, 1.0), y);
  y = fma(y, fma(-m, y, 1.0), y);
  return ldexp(y, -e);
}

__device__ __forceinline__ double nr_rsqrt(double x) {  // x > 0
  int e;
  double m = frexp(x, &e);
  if (e & 1) {
    m *= 2.0;
    e -= 1;
  }
  double y = (double)rsqrtf((float)m);
  y = fma(0.5 * y, fma(-m * y, y, 1.0), y);
  y = fma(0.5 * y, fma(-m * y, y, 1.0), y);
  return ldexp(y, -e / 2);
}

constexpr int JC = 8;      // CTAs per cluster
constexpr int JNT = 256;   // threads per CTA
constexpr int JLD = kMaxP + 1;
constexpr int JROWS = (kMaxP + JC - 1) / JC;  // eigenvector rows per CTA

__global__ void __cluster_dims__(JC, 1, 1) __launch_bounds__(JNT)
    k_jacobi_cluster(const double *__restrict__ Hin, int p, double *__restrict__ Yeig,
                     double *__restrict__ theta, Params *prm) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ double dyn[];
  double *Hb[2] = {dyn, dyn + kMaxP * JLD};
  double *Vloc = dyn + 2 * kMaxP * JLD;  // JROWS x JLD
  __shared__ double cs[kMaxP / 2], sn[kMaxP / 2];
  __shared__ int pk[kMaxP / 2], pl[kMaxP / 2];
  __shared__ double redsh[32];
  __shared__ double lam_s[kMaxP];
  const int tid = threadIdx.x;
  const int m = p + (p & 1);          // players (index p is a dummy when p is odd)
  const int half = m / 2;
  const int ppc = (half + JC - 1) / JC;
  const int pair0 = rank * ppc, pair1 = min(half, pair0 + ppc);
  const int row0 = rank * JROWS, row1 = min(p, row0 + JROWS);

  // H = sym(reduced Gram matrix); local eigenvector rows = rows of I
  for (int idx = tid; idx < p * p; idx += JNT) {
    const int a = idx / p, b = idx % p;
    Hb[0][a * JLD + b] = 0.5 * (Hin[a * p + b] + Hin[b * p + a]);
  }
  for (int idx = tid; idx < JROWS * p; idx += JNT) {
    const int r = idx / p, b = idx % p;
    Vloc[r * JLD + b] = (row0 + r == b) ? 1.0 : 0.0;
  }
  cluster.sync();  // every CTA has started before any remote store
  int cur = 0;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
    const double *H = Hb[cur];
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < p * p; idx += JNT) {
      const int a = idx / p, b = idx % p;
      const double h = H[a * JLD + b];
      tot = fma(h, h, tot);
      if (a != b) off = fma(h, h, off);
    }
    off = block_reduce(off, redsh, 0);
    tot = block_reduce(tot, redsh, 0);
    if (!(off > 1e-30 * tot)) break;  // identical decision in every CTA
    for (int round = 0; round < m - 1; ++round) {
      H = Hb[cur];
      double *Hn = Hb[cur ^ 1];
      if (tid < half) {
        const int i = tid;
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (m - 1)); };
        int k = player(i), l = player(m - 1 - i);
        if (k > l) { const int tt = k; k = l; l = tt; }
        double c = 1.0, s = 0.0;
        if (l < p) {
          const double hkl = H[k * JLD + l];
          const double hkk = H[k * JLD + k], hll = H[l * JLD + l];
          if (fabs(hkl) > 0.5e-17 * (fabs(hkk) + fabs(hll)) && hkl != 0.0) {
            // t = tan of the angle that annihilates h_kl: the smaller root of
            // t^2 + 2 tau t - 1 = 0, tau = (h_ll - h_kk) / (2 h_kl)
            const double tau = (hll - hkk) * (0.5 * nr_rcp(hkl));
            double t;
            if (fabs(tau) > 1e150) {
              t = 0.5 * nr_rcp(tau);
            } else {
              const double q = fma(tau, tau, 1.0);
              t = (tau >= 0.0 ? 1.0 : -1.0) * nr_rcp(fabs(tau) + q * nr_rsqrt(q));
            }
            c = nr_rsqrt(fma(t, t, 1.0));
            s = t * c;
          }
        }
        cs[i] = c; sn[i] = s; pk[i] = k; pl[i] = l;
      }
      __syncthreads();
      // local eigenvector rows: V <- V J
      for (int idx = tid; idx < (row1 - row0) * half; idx += JNT) {
        const int r = idx / half, i = idx % half;
        const int k = pk[i], l = pl[i];
        if (l >= p || sn[i] == 0.0) continue;
        double *vr = Vloc + r * JLD;
        const double vk = vr[k], vl = vr[l];
        vr[k] = cs[i] * vk - sn[i] * vl;
        vr[l] = sn[i] * vk + cs[i] * vl;
      }
      // new rows of H for the pairs of this CTA: block (i, j) = J_i^T H_ij J_j
      const int nb = (pair1 - pair0) * half;
      for (int idx = tid; idx < nb; idx += JNT) {
        const int i = pair0 + idx / half, j = idx % half;
        const int ki = pk[i], li = pl[i], kj = pk[j], lj = pl[j];
        const double ci = cs[i], si = sn[i], cj = cs[j], sj = sn[j];
        const bool ri = li < p, rj = lj < p;  // false: the partner is the dummy
        const double a = H[ki * JLD + kj];
        const double b = rj ? H[ki * JLD + lj] : 0.0;
        const double c = ri ? H[li * JLD + kj] : 0.0;
        const double d = (ri && rj) ? H[li * JLD + lj] : 0.0;
        // M = B J_j
        const double m00 = cj * a - sj * b, m01 = sj * a + cj * b;
        const double m10 = cj * c - sj * d, m11 = sj * c + cj * d;
        // H' block = J_i^T M
        double h00 = ci * m00 - si * m10, h01 = ci * m01 - si * m11;
        double h10 = si * m00 + ci * m10, h11 = si * m01 + ci * m11;
        if (i == j && si != 0.0) { h01 = 0.0; h10 = 0.0; }
        for (int q = 0; q < JC; ++q) {
          double *dst = cluster.map_shared_rank(Hn, q);
          dst[ki * JLD + kj] = h00;
          if (rj) dst[ki * JLD + lj] = h01;
          if (ri) dst[li * JLD + kj] = h10;
          if (ri && rj) dst[li * JLD + lj] = h11;
        }
      }
      cluster.sync();
      cur ^= 1;
    }
    sweeps_done = sweep + 1;
  }
  // eigenvalues, descending (ties by index); every CTA computes the ranks
  const double *H = Hb[cur];
  if (tid < p) lam_s[tid] = H[tid * JLD + tid];
  __syncthreads();
  bool bad = false;
  for (int j = tid; j < p; j += JNT) {
    const double lj = lam_s[j];
    if (!isfinite(lj)) bad = true;
    int rk = 0;
    for (int i = 0; i < p; ++i) {
      const double li = lam_s[i];
      if (li > lj || (li == lj && i < j)) ++rk;
    }
    if (rank == 0) theta[rk] = lj;
    for (int r = row0; r < row1; ++r) Yeig[r * p + rk] = Vloc[(r - row0) * JLD + j];
  }
  if (bad && rank == 0) atomicOr(&prm->flags, 4);
  if (rank == 0 && tid == 0) prm->sweeps = sweeps_done;
  cluster.sync();  // no CTA leaves while its shared memory may still be written
}

constexpr size_t kJacobiBytes = (size_t)(2 * kMaxP * JLD + JROWS * JLD) * sizeof(double);

}  // namespace

cudaError_t configure_jacobi() {
  return cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kJacobiBytes);
}

cudaError_t launch_jacobi_cluster(cudaStream_t s, const Workspace &ws, const double *H, int p,
                                  double *theta) {
  k_jacobi_cluster<<<JC, JNT, kJacobiBytes, s>>>(H, p, ws.Yeig, theta, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
