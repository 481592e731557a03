// p x p symmetric eigensolve of the Rayleigh-Ritz step (Sec. 2.2, Eq. (RR):
// H = Y Theta Y^T) by parallel cyclic Jacobi on a thread-block cluster.
//
// On GB300 a single SM executes about 4 FP64 flop per clock, so a one-block
// Jacobi at p = 64 spends milliseconds per call.  Here the 8 CTAs of a
// cluster share the rotation work of every round:
//   * each CTA keeps a full replica of H (double-buffered in shared memory)
//     and computes all p/2 rotation angles of the round redundantly (the
//     replicas are bitwise identical, so every CTA takes the same branches);
//     the one-CTA variant (p <= 32) updates a single copy of H in place: the
//     p/2 disjoint pairs split H into 2 x 2 blocks that are read and written
//     by one thread each, and blocks whose two pairs do not rotate are skipped;
//   * on one CTA, the four lanes that form the angle of a pair also rotate
//     the pair's own 2 x 2 diagonal block (one entry each), so the block
//     phase holds only the off-diagonal blocks (at p = 32: 120 instead of
//     136, four warps, one per SM sub-partition); in the cluster, where every
//     CTA forms all angles, the diagonal blocks stay in the block phase (a
//     longer angle chain in every CTA measured slower at p = 64);
//   * CTA c computes the new rows of H' = J^T H J for its share of the
//     rotation pairs (2 x 2 blocks J_i^T H_ij J_j) and stores them into the
//     next buffer of every CTA of the cluster (distributed shared memory);
//     the one-CTA variant (p <= 32) computes the upper block triangle only
//     and mirrors it;
//   * CTA c owns a slice of rows of the eigenvector matrix and applies all
//     rotations to it locally; the rotations of round r are applied to it
//     while the angles of round r + 1 are formed (two rotation sets in
//     shared memory; on one CTA by warps 2..7);
//   * one cluster barrier per round orders the exchange.
// The sweep loop stops when off(H) <= kOffStop ||H||_F (or after 40 sweeps);
// eigenvalues are sorted descending (ties by index).
#include <cooperative_groups.h>

#include "pf_internal.cuh"

namespace cg = cooperative_groups;

namespace pf {

namespace {

// Rotation of the pair (k, l): the tangent t comes from single-precision
// arithmetic (|t| <= 1, the smaller root of t^2 + 2 tau t - 1 = 0 with
// tau = (h_ll - h_kk) / (2 h_kl)), and so does u = tan(theta / 2) =
// t / (1 + sqrt(1 + t^2)).  The rotation is then the rational one,
// c = (1 - u^2) / (1 + u^2), s = 2u / (1 + u^2), formed in FP64 from the
// exact single-precision u (u^2 is exact in FP64) with one Newton
// reciprocal: c^2 + s^2 = 1 to FP64 rounding, and the FP64 chain after the
// single-precision part is a multiply, an add, the reciprocal's four
// operations and a multiply (a reciprocal square root by Newton's method
// needs six).  The rotation annihilates h_kl only to single precision, so
// the updated 2 x 2 block keeps its computed off-diagonal entries; the
// sweeps still converge (each rotation shrinks |h_kl| by ~1e-7 on top of the
// quadratic coupling).  On GB300 the FP64 pipe is 1/64 of FP32, and dependent
// FP64 operations set the length of every rotation round.
__device__ __forceinline__ void rotation(double hkk, double hll, double hkl, double &c,
                                         double &s) {
  c = 1.0;
  s = 0.0;
  if (!(fabs(hkl) > 0.5e-17 * (fabs(hkk) + fabs(hll))) || hkl == 0.0) return;
  const double d = hll - hkk;
  const float h32 = (float)hkl, d32 = (float)d;
  if (fabsf(h32) >= 1e-30f && isfinite(h32) && isfinite(d32)) {
    const float tau = d32 / (2.0f * h32);
    float t32;
    if (fabsf(tau) > 1e18f) t32 = 0.5f / tau;
    else t32 = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
    const float u32 = t32 / (1.0f + sqrtf(fmaf(t32, t32, 1.0f)));  // |u| <= tan(pi/8)
    const double u = (double)u32;
    const double u2 = u * u;  // exact
    const double r = rcp_newton(1.0 + u2);
    c = (1.0 - u2) * r;
    s = (2.0 * u) * r;
    return;
  }
  // outside the single-precision range: the exact FP64 angle
  const double tau = d / (2.0 * hkl);
  double t;
  if (fabs(tau) > 1e150) t = 0.5 / tau;
  else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

// Convergence: off(H)^2 <= kOffStop^2 ||H||_F^2 at the start of a sweep.
constexpr double kOffStop2 = 1e-30;

constexpr int JC = 8;      // CTAs per cluster
constexpr int kJacobiOneCta = 32;  // largest p on one CTA (the cluster above; at p = 64 one CTA took 2.4-3.7 ms per call against the cluster's 1.3 ms)
constexpr int JNT = 256;   // threads per CTA of the cluster version
constexpr int JNB = 256;   // threads of the one-CTA version
constexpr int JLD = kMaxP + 1;

// The sweep loop, on NC CTAs: NC = 8 (a thread-block cluster, distributed
// shared memory, one cluster barrier per round) or NC = 1 (one CTA holds
// everything and a block barrier orders the rounds; at p <= 32 the FP64 work
// of a round is small enough that one SM beats the cluster's barrier and
// broadcast cost).
template <int NC, int NTH>
__device__ __forceinline__ void jacobi_body(const double *__restrict__ Hin, int p,
                                            double *__restrict__ Yeig,
                                            double *__restrict__ theta, Params *prm) {
  constexpr int JROWS = (kMaxP + NC - 1) / NC;  // eigenvector rows per CTA
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = NC > 1 ? (int)cluster.block_rank() : 0;
  auto sync_all = [&]() {
    if constexpr (NC > 1) cluster.sync();
    else __syncthreads();
  };
  constexpr int NHB = NC > 1 ? 2 : 1;  // copies of H (one CTA: in place)
  extern __shared__ double dyn[];
  double *Hb[2] = {dyn, dyn + (NHB - 1) * kMaxP * JLD};
  double *Vloc = dyn + NHB * kMaxP * JLD;  // JROWS x JLD
  // two rotation sets: the current round's and the previous round's, whose
  // eigenvector update runs during the current round's angle phase
  __shared__ double cs[2][kMaxP / 2], sn[2][kMaxP / 2];
  __shared__ int pk[2][kMaxP / 2], pl[2][kMaxP / 2];
  __shared__ int act[2][kMaxP / 2];  // the pair rotates (an integer test, off the FP64 pipe)
  __shared__ double redsh[32];
  __shared__ double lam_s[kMaxP];
  // one CTA: the blocks (i, j > i) of the strict upper block triangle, in order
  __shared__ unsigned char tri_i[NC == 1 ? (kMaxP / 2) * (kMaxP / 2 - 1) / 2 : 1];
  __shared__ unsigned char tri_j[NC == 1 ? (kMaxP / 2) * (kMaxP / 2 - 1) / 2 : 1];
  const int tid = threadIdx.x;
  const int m = p + (p & 1);          // players (index p is a dummy when p is odd)
  const int half = m / 2;
  const int ppc = (half + NC - 1) / NC;
  const int pair0 = rank * ppc, pair1 = min(half, pair0 + ppc);
  const int row0 = rank * JROWS, row1 = min(p, row0 + JROWS);

  if constexpr (NC == 1) {
    if (tid == 0) {
      int k = 0;
      for (int i = 0; i < half; ++i)
        for (int j = i + 1; j < half; ++j) {
          tri_i[k] = (unsigned char)i;
          tri_j[k] = (unsigned char)j;
          ++k;
        }
    }
  }
  // H = sym(reduced Gram matrix); local eigenvector rows = rows of I
  for (int idx = tid; idx < p * p; idx += NTH) {
    const int a = idx / p, b = idx % p;
    Hb[0][a * JLD + b] = 0.5 * (Hin[a * p + b] + Hin[b * p + a]);
  }
  for (int idx = tid; idx < JROWS * p; idx += NTH) {
    const int r = idx / p, b = idx % p;
    Vloc[r * JLD + b] = (row0 + r == b) ? 1.0 : 0.0;
  }
  sync_all();  // every CTA has started before any remote store
  // local eigenvector rows: V <- V J for rotation set b, item idx0, stride
  auto rotate_v = [&](int b, int idx0, int stride) {
    for (int idx = idx0; idx < (row1 - row0) * half; idx += stride) {
      const int r = idx / half, i = idx % half;
      if (!act[b][i]) continue;
      const int k = pk[b][i], l = pl[b][i];
      double *vr = Vloc + r * JLD;
      const double vk = vr[k], vl = vr[l];
      vr[k] = cs[b][i] * vk - sn[b][i] * vl;
      vr[l] = sn[b][i] * vk + cs[b][i] * vl;
    }
  };
  int cur = 0;
  int sweeps_done = 0;
  int set = 0;           // rotation set of the current round
  bool pending = false;  // the other set still has to be applied to V
  for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
    const double *H = Hb[cur];
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < p * p; idx += NTH) {
      const int a = idx / p, b = idx % p;
      const double h = H[a * JLD + b];
      tot = fma(h, h, tot);
      if (a != b) off = fma(h, h, off);
    }
    off = block_reduce(off, redsh, 0);
    tot = block_reduce(tot, redsh, 0);
    if (!(off > kOffStop2 * tot)) break;  // identical decision in every CTA
    for (int round = 0; round < m - 1; ++round) {
      H = Hb[cur];
      double *Hn = Hb[cur ^ 1];
      const int b = set;
      // angle phase: one CTA gives each pair four lanes (threads 4i..4i+3),
      // which form the same rotation and one entry each of the pair's
      // rotated diagonal block; the cluster forms the angles on lanes 0..
      // of warp 0 and rotates the diagonal blocks in the block phase
      constexpr int LPP = NC == 1 ? 4 : 1;  // lanes per pair
      if (tid < LPP * half) {
        const int i = tid / LPP, lq = tid % LPP;
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (m - 1)); };
        int k = player(i), l = player(m - 1 - i);
        if (k > l) { const int tt = k; k = l; l = tt; }
        const bool real = l < p;  // false: the partner is the dummy
        const double hkk = H[k * JLD + k];
        const double hkl = real ? H[k * JLD + l] : 0.0, hlk = real ? H[l * JLD + k] : 0.0;
        const double hll = real ? H[l * JLD + l] : 0.0;
        double c = 1.0, s = 0.0;
        if (real) rotation(hkk, hll, hkl, c, s);
        if (lq == 0) {
          cs[b][i] = c; sn[b][i] = s; pk[b][i] = k; pl[b][i] = l;
          act[b][i] = (real && s != 0.0) ? 1 : 0;
        }
        if constexpr (NC == 1) {
          // the pair's diagonal block J^T B J with B = [a b; b' d]:
          // M = B J has m00 = c a - s b, m01 = s a + c b, m10 = c b' - s d,
          // m11 = s b' + c d; lane 0 forms h00 = c m00 - s m10, lane 1
          // h11 = s m01 + c m11, lane 2 h01 = c m01 - s m11, lane 3
          // h10 = s m00 + c m10 (one instruction stream for all four
          // lanes), and lanes 2, 3 store the symmetrised (h01 + h10) / 2.
          // Skipped when J = I
          const bool sw = lq == 1 || lq == 2;  // lanes using (m01, m11)
          const double al = sw ? s : c, be = sw ? c : -s;
          const double x = fma(al, hkk, be * hkl), y = fma(al, hlk, be * hll);
          const bool so = lq == 1 || lq == 3;  // outputs s x + c y
          const double h = fma(so ? s : c, x, (so ? c : -s) * y);
          // the lanes of this warp in the angle phase: whole groups of four
          const int nact = min(32, LPP * half - (tid & ~31));
          const unsigned gmask = nact >= 32 ? 0xffffffffu : ((1u << nact) - 1u);
          const double hx = __shfl_xor_sync(gmask, h, 1);
          if (s != 0.0) {
            if (lq == 0) Hn[k * JLD + k] = h;
            else if (lq == 1) Hn[l * JLD + l] = h;
            else Hn[lq == 2 ? k * JLD + l : l * JLD + k] = 0.5 * (h + hx);
          }
        }
      }
      if (pending) {
        if constexpr (NC == 1) {
          // the warps after those of the angle phase (LPP half lanes: warps
          // 0-1 at p = 32, 0-3 at p = 64)
          const int va = ((LPP * half + 31) / 32) * 32;
          if (tid >= va) rotate_v(b ^ 1, tid - va, NTH - va);
        } else {
          rotate_v(b ^ 1, tid, NTH);
        }
      }
      __syncthreads();
      // blocks (i, j) = J_i^T H_ij J_j.  One CTA computes the strict upper
      // block triangle in place and mirrors it (H stays exactly symmetric;
      // less than half the FP64 work of the full square); the cluster's CTAs
      // compute the block rows of their pairs, diagonal blocks included, so
      // that their broadcasts stay row-contiguous
      const int nb = NC == 1 ? half * (half - 1) / 2 : (pair1 - pair0) * half;
      for (int idx = tid; idx < nb; idx += NTH) {
        int i, j;
        if constexpr (NC == 1) {
          i = tri_i[idx];
          j = tri_j[idx];
          if (!act[b][i] && !act[b][j]) continue;  // identity block, kept in place
        } else {
          i = pair0 + idx / half;
          j = idx % half;
        }
        const int ki = pk[b][i], li = pl[b][i], kj = pk[b][j], lj = pl[b][j];
        const double ci = cs[b][i], si = sn[b][i], cj = cs[b][j], sj = sn[b][j];
        const bool ri = li < p, rj = lj < p;  // false: the partner is the dummy
        const double a = H[ki * JLD + kj];
        const double b = rj ? H[ki * JLD + lj] : 0.0;
        const double c = ri ? H[li * JLD + kj] : 0.0;
        const double d = (ri && rj) ? H[li * JLD + lj] : 0.0;
        // M = B J_j
        const double m00 = cj * a - sj * b, m01 = sj * a + cj * b;
        const double m10 = cj * c - sj * d, m11 = sj * c + cj * d;
        // H' block = J_i^T M
        const double h00 = ci * m00 - si * m10, h11 = si * m01 + ci * m11;
        double h01 = ci * m01 - si * m11, h10 = si * m00 + ci * m10;
        if (NC > 1 && i == j) h01 = h10 = 0.5 * (h01 + h10);  // the rotated pair block stays symmetric
        for (int q = 0; q < NC; ++q) {
          double *dst = NC > 1 ? cluster.map_shared_rank(Hn, q) : Hn;
          dst[ki * JLD + kj] = h00;
          if (rj) dst[ki * JLD + lj] = h01;
          if (ri) dst[li * JLD + kj] = h10;
          if (ri && rj) dst[li * JLD + lj] = h11;
          if (NC == 1) {  // the mirrored block (j, i), j > i
            dst[kj * JLD + ki] = h00;
            if (rj) dst[lj * JLD + ki] = h01;
            if (ri) dst[kj * JLD + li] = h10;
            if (ri && rj) dst[lj * JLD + li] = h11;
          }
        }
      }
      sync_all();
      if (NHB > 1) cur ^= 1;
      set ^= 1;
      pending = true;
    }
    sweeps_done = sweep + 1;
  }
  if (pending) {
    rotate_v(set ^ 1, tid, NTH);
    __syncthreads();
  }
  // eigenvalues, descending (ties by index); every CTA computes the ranks
  const double *H = Hb[cur];
  if (tid < p) lam_s[tid] = H[tid * JLD + tid];
  __syncthreads();
  bool bad = false;
  for (int j = tid; j < p; j += NTH) {
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
  sync_all();  // no CTA leaves while its shared memory may still be written
}

__global__ void __cluster_dims__(JC, 1, 1) __launch_bounds__(JNT)
    k_jacobi_cluster(const double *__restrict__ Hin, int p, double *__restrict__ Yeig,
                     double *__restrict__ theta, Params *prm) {
  jacobi_body<JC, JNT>(Hin, p, Yeig, theta, prm);
}

__global__ void __launch_bounds__(JNB)
    k_jacobi_block(const double *__restrict__ Hin, int p, double *__restrict__ Yeig,
                   double *__restrict__ theta, Params *prm) {
  jacobi_body<1, JNB>(Hin, p, Yeig, theta, prm);
}

constexpr size_t jacobi_bytes(int nc) {
  return (size_t)((nc > 1 ? 2 : 1) * kMaxP * JLD + ((kMaxP + nc - 1) / nc) * JLD) *
         sizeof(double);
}

}  // namespace

cudaError_t configure_jacobi() {
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_cluster,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)jacobi_bytes(JC));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_jacobi_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)jacobi_bytes(1));
}

cudaError_t launch_jacobi_cluster(cudaStream_t s, const Workspace &ws, const double *H, int p,
                                  double *theta) {
  if (p <= kJacobiOneCta) k_jacobi_block<<<1, JNB, jacobi_bytes(1), s>>>(H, p, ws.Yeig, theta, ws.prm);
  else k_jacobi_cluster<<<JC, JNT, jacobi_bytes(JC), s>>>(H, p, ws.Yeig, theta, ws.prm);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
