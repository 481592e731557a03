// p x p symmetric eigensolve of the Rayleigh-Ritz step (Sec. 2.2, Eq. (RR):
// H = Y Theta Y^T), GB300-first.
//
// On GB300 the FP64 pipe runs at 1/64 of FP32, and a parallel FP64 Jacobi
// spends most of each of its (p - 1) rounds per sweep on the FP64
// rotation-angle chain and on synchronisation.  Here:
//   1. parallel cyclic Jacobi in FP32 (one CTA, block barriers) gives
//      eigenvector approximations X to single precision;
//   2. three FP64 refinement iterations of the Ogita-Aishima method
//      (iterative refinement for the symmetric eigenproblem, 2018):
//        R = I - X^T X,  S = X^T H X,  lambda_i = S_ii / (1 - R_ii),
//        E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) when
//        |lambda_i - lambda_j| > delta, E_ij = R_ij / 2 otherwise,
//        X <- X + X E,
//      each roughly squaring the error of the well-separated pairs;
//      delta = max(2 (||S - D||_F + ||H||_F ||R||_F), 1e-5 ||H||_F);
//   3. after each refinement the eigenvalues closer than delta (clusters,
//      whose vectors the refinement only re-orthogonalises) are resolved by
//      an FP64 Jacobi of the cluster's block of S = X^T H X;
//   4. eigenvalues are the Rayleigh quotients S_ii / (1 - R_ii), sorted
//      descending (ties by index), with the matching columns of X.
// The matrix products are p x p x p FP64 (one output row per block, p
// blocks); the decisions (delta, clusters, ordering) are taken by single
// blocks, so every launch is deterministic.
#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int ENT = 256;          // threads of the single-block kernels
constexpr int ELD = kMaxP + 1;
constexpr double kClusterFloor = 1e-5;
constexpr int kRefineIters = 3;

// ---------------------------------------------------------------------------
// 1. FP32 parallel cyclic Jacobi, one CTA (round-robin pairing; each round
//    rotates p/2 disjoint pairs; H' = J^T H J by 2 x 2 blocks, V <- V J).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(ENT) k_eig32(const double *__restrict__ Hin, int p,
                                               double *__restrict__ X, Params *prm) {
  extern __shared__ float fsm[];
  float *Hb[2] = {fsm, fsm + kMaxP * ELD};
  float *V = fsm + 2 * kMaxP * ELD;
  __shared__ float cs[kMaxP / 2], sn[kMaxP / 2];
  __shared__ int pk[kMaxP / 2], pl[kMaxP / 2];
  __shared__ double redsh[32];
  const int tid = threadIdx.x;
  const int m = p + (p & 1);
  const int half = m / 2;
  for (int idx = tid; idx < p * p; idx += ENT) {
    const int a = idx / p, b = idx % p;
    Hb[0][a * ELD + b] = (float)(0.5 * (Hin[a * p + b] + Hin[b * p + a]));
    V[a * ELD + b] = a == b ? 1.0f : 0.0f;
  }
  __syncthreads();
  int cur = 0, sweeps = 0;
  for (int sweep = 0; sweep < 20 && m > 1; ++sweep) {
    const float *H = Hb[cur];
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < p * p; idx += ENT) {
      const int a = idx / p, b = idx % p;
      const double h = (double)H[a * ELD + b];
      tot = fma(h, h, tot);
      if (a != b) off = fma(h, h, off);
    }
    off = block_reduce(off, redsh, 0);
    tot = block_reduce(tot, redsh, 0);
    if (!(off > 1e-12 * tot)) break;  // single-precision resolution reached
    for (int round = 0; round < m - 1; ++round) {
      H = Hb[cur];
      float *Hn = Hb[cur ^ 1];
      if (tid < half) {
        const int i = tid;
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (m - 1)); };
        int k = player(i), l = player(m - 1 - i);
        if (k > l) { const int tt = k; k = l; l = tt; }
        float c = 1.0f, s = 0.0f;
        if (l < p) {
          const float hkl = H[k * ELD + l], hkk = H[k * ELD + k], hll = H[l * ELD + l];
          if (fabsf(hkl) > 1e-12f * (fabsf(hkk) + fabsf(hll)) && hkl != 0.0f) {
            const float tau = (hll - hkk) / (2.0f * hkl);
            float t;
            if (fabsf(tau) > 1e18f) t = 0.5f / tau;
            else t = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
            c = rsqrtf(fmaf(t, t, 1.0f));
            s = t * c;
          }
        }
        cs[i] = c; sn[i] = s; pk[i] = k; pl[i] = l;
      }
      __syncthreads();
      for (int idx = tid; idx < p * half; idx += ENT) {
        const int r = idx / half, i = idx % half;
        const int k = pk[i], l = pl[i];
        if (l >= p || sn[i] == 0.0f) continue;
        float *vr = V + r * ELD;
        const float vk = vr[k], vl = vr[l];
        vr[k] = cs[i] * vk - sn[i] * vl;
        vr[l] = sn[i] * vk + cs[i] * vl;
      }
      for (int idx = tid; idx < half * half; idx += ENT) {
        const int i = idx / half, j = idx % half;
        const int ki = pk[i], li = pl[i], kj = pk[j], lj = pl[j];
        const float ci = cs[i], si = sn[i], cj = cs[j], sj = sn[j];
        const bool ri = li < p, rj = lj < p;
        const float a = H[ki * ELD + kj];
        const float b = rj ? H[ki * ELD + lj] : 0.0f;
        const float cc = ri ? H[li * ELD + kj] : 0.0f;
        const float d = (ri && rj) ? H[li * ELD + lj] : 0.0f;
        const float m00 = cj * a - sj * b, m01 = sj * a + cj * b;
        const float m10 = cj * cc - sj * d, m11 = sj * cc + cj * d;
        Hn[ki * ELD + kj] = ci * m00 - si * m10;
        if (rj) Hn[ki * ELD + lj] = ci * m01 - si * m11;
        if (ri) Hn[li * ELD + kj] = si * m00 + ci * m10;
        if (ri && rj) Hn[li * ELD + lj] = si * m01 + ci * m11;
      }
      __syncthreads();
      cur ^= 1;
    }
    sweeps = sweep + 1;
  }
  for (int idx = tid; idx < p * p; idx += ENT) {
    const int a = idx / p, b = idx % p;
    X[idx] = (double)V[a * ELD + b];
  }
  if (tid == 0) prm->sweeps = sweeps;
}

// ---------------------------------------------------------------------------
// 2. FP64 refinement products, one output row per block (threads = columns).
// ---------------------------------------------------------------------------
// AX = Hs X with Hs = (H + H^T) / 2
__global__ void k_ref_ax(const double *__restrict__ H, int p, const double *__restrict__ X,
                         double *__restrict__ AX) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= p) return;
  double s = 0.0;
  for (int k = 0; k < p; ++k) s = fma(0.5 * (H[i * p + k] + H[k * p + i]), X[k * p + j], s);
  AX[i * p + j] = s;
}

// S = X^T (AX), R = I - X^T X
__global__ void k_ref_sr(int p, const double *__restrict__ X, const double *__restrict__ AX,
                         double *__restrict__ S, double *__restrict__ R) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= p) return;
  double s = 0.0, r = 0.0;
  for (int k = 0; k < p; ++k) {
    const double xi = X[k * p + i];
    s = fma(xi, AX[k * p + j], s);
    r = fma(xi, X[k * p + j], r);
  }
  S[i * p + j] = s;
  R[i * p + j] = (i == j ? 1.0 : 0.0) - r;
}

// lambda_i = S_ii / (1 - R_ii) and the cluster threshold delta (block-wide).
__device__ double ref_lambda_delta(const double *__restrict__ H, int p,
                                   const double *__restrict__ S, const double *__restrict__ R,
                                   double *lam, double *sh) {
  for (int i = threadIdx.x; i < p; i += blockDim.x) lam[i] = S[i * p + i] / (1.0 - R[i * p + i]);
  __syncthreads();
  double ns = 0.0, nr = 0.0, na = 0.0;
  for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x) {
    const int i = idx / p, j = idx % p;
    const double sd = S[idx] - (i == j ? lam[i] : 0.0);
    ns = fma(sd, sd, ns);
    nr = fma(R[idx], R[idx], nr);
    const double h = 0.5 * (H[idx] + H[j * p + i]);
    na = fma(h, h, na);
  }
  ns = block_reduce(ns, sh, 0);
  nr = block_reduce(nr, sh, 0);
  na = block_reduce(na, sh, 0);
  const double nh = sqrt(na);
  return fmax(2.0 * (sqrt(ns) + nh * sqrt(nr)), kClusterFloor * nh);
}

__global__ void __launch_bounds__(ENT) k_ref_e(const double *__restrict__ H, int p,
                                               const double *__restrict__ S,
                                               const double *__restrict__ R,
                                               double *__restrict__ E) {
  __shared__ double lam[kMaxP];
  __shared__ double sh[32];
  const double delta = ref_lambda_delta(H, p, S, R, lam, sh);
  for (int idx = threadIdx.x; idx < p * p; idx += ENT) {
    const int i = idx / p, j = idx % p;
    double e;
    if (i == j) e = 0.5 * R[idx];
    else if (fabs(lam[i] - lam[j]) > delta) e = (S[idx] + lam[j] * R[idx]) / (lam[j] - lam[i]);
    else e = 0.5 * R[idx];
    E[idx] = e;
  }
}

// X <- X + X E, row i per block
__global__ void k_ref_update(int p, double *__restrict__ X, const double *__restrict__ E) {
  __shared__ double xr[kMaxP];
  const int i = blockIdx.x, j = threadIdx.x;
  if (j < p) xr[j] = X[i * p + j];
  __syncthreads();
  if (j >= p) return;
  double s = xr[j];
  for (int k = 0; k < p; ++k) s = fma(xr[k], E[k * p + j], s);
  X[i * p + j] = s;
}

// rank of lambda_i in descending order, ties by index
__device__ __forceinline__ int desc_rank(const double *lam, int p, int i) {
  const double li = lam[i];
  int rk = 0;
  for (int j = 0; j < p; ++j) {
    const double lj = lam[j];
    if (lj > li || (lj == li && j < i)) ++rk;
  }
  return rk;
}

// ---------------------------------------------------------------------------
// 3. Clusters: runs of the descending eigenvalue order closer than delta;
//    each run's block of S (symmetrised) is diagonalised by cyclic FP64
//    Jacobi and its columns of X are rotated.  One block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(ENT) k_ref_cluster(const double *__restrict__ H, int p,
                                                     const double *__restrict__ S,
                                                     const double *__restrict__ R,
                                                     double *__restrict__ X) {
  extern __shared__ double dsm[];
  double *Xs = dsm;                   // p x ELD
  double *Ac = dsm + kMaxP * ELD;     // cluster block, k x ELD
  double *W = Ac + kMaxP * ELD;       // its eigenvectors, k x ELD
  __shared__ double lam[kMaxP];
  __shared__ int ord[kMaxP];
  __shared__ int cstart[kMaxP], clen[kMaxP];
  __shared__ int ncl;
  __shared__ double sh[32];
  __shared__ double rc, rs;
  __shared__ int ra, rb;
  const int tid = threadIdx.x;
  const double delta = ref_lambda_delta(H, p, S, R, lam, sh);
  for (int i = tid; i < p; i += ENT) ord[desc_rank(lam, p, i)] = i;
  for (int idx = tid; idx < p * p; idx += ENT) Xs[(idx / p) * ELD + idx % p] = X[idx];
  __syncthreads();
  if (tid == 0) {
    int n = 0, q = 0;
    while (q < p) {
      int e = q;
      while (e + 1 < p && fabs(lam[ord[e]] - lam[ord[e + 1]]) <= delta) ++e;
      if (e > q) {
        cstart[n] = q;
        clen[n] = e - q + 1;
        ++n;
      }
      q = e + 1;
    }
    ncl = n;
  }
  __syncthreads();
  for (int cl = 0; cl < ncl; ++cl) {
    const int q0 = cstart[cl], k = clen[cl];
    for (int idx = tid; idx < k * k; idx += ENT) {
      const int a = idx / k, b = idx % k;
      const int ia = ord[q0 + a], ib = ord[q0 + b];
      Ac[a * ELD + b] = 0.5 * (S[ia * p + ib] + S[ib * p + ia]);
      W[a * ELD + b] = a == b ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 30; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (int idx = tid; idx < k * k; idx += ENT) {
        const int a = idx / k, b = idx % k;
        const double h = Ac[a * ELD + b];
        tot = fma(h, h, tot);
        if (a != b) off = fma(h, h, off);
      }
      off = block_reduce(off, sh, 0);
      tot = block_reduce(tot, sh, 0);
      if (!(off > 1e-30 * tot)) break;
      for (int a = 0; a < k - 1; ++a) {
        for (int b = a + 1; b < k; ++b) {
          if (tid == 0) {
            const double hab = Ac[a * ELD + b], haa = Ac[a * ELD + a], hbb = Ac[b * ELD + b];
            double c = 1.0, s = 0.0;
            if (hab != 0.0 && fabs(hab) > 0.5e-17 * (fabs(haa) + fabs(hbb))) {
              const double tau = (hbb - haa) / (2.0 * hab);
              double t;
              if (fabs(tau) > 1e150) t = 0.5 / tau;
              else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
              c = 1.0 / sqrt(1.0 + t * t);
              s = t * c;
            }
            rc = c; rs = s; ra = a; rb = b;
          }
          __syncthreads();
          const double c = rc, s = rs;
          if (s != 0.0) {
            // columns a, b of Ac and W, then rows a, b of Ac
            for (int r = tid; r < k; r += ENT) {
              const double xa = Ac[r * ELD + a], xb = Ac[r * ELD + b];
              Ac[r * ELD + a] = c * xa - s * xb;
              Ac[r * ELD + b] = s * xa + c * xb;
              const double wa = W[r * ELD + a], wb = W[r * ELD + b];
              W[r * ELD + a] = c * wa - s * wb;
              W[r * ELD + b] = s * wa + c * wb;
            }
            __syncthreads();
            for (int r = tid; r < k; r += ENT) {
              const double xa = Ac[a * ELD + r], xb = Ac[b * ELD + r];
              Ac[a * ELD + r] = c * xa - s * xb;
              Ac[b * ELD + r] = s * xa + c * xb;
            }
          }
          __syncthreads();
        }
      }
    }
    // X[:, cluster] <- X[:, cluster] W
    for (int r = tid; r < p; r += ENT) {
      double tmp[kMaxP];
      for (int b = 0; b < k; ++b) {
        double v = 0.0;
        for (int a = 0; a < k; ++a) v = fma(Xs[r * ELD + ord[q0 + a]], W[a * ELD + b], v);
        tmp[b] = v;
      }
      for (int b = 0; b < k; ++b) Xs[r * ELD + ord[q0 + b]] = tmp[b];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < p * p; idx += ENT) X[idx] = Xs[(idx / p) * ELD + idx % p];
}

// ---------------------------------------------------------------------------
// 4. Eigenvalues (Rayleigh quotients), descending order, eigenvectors.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(ENT) k_ref_final(int p, const double *__restrict__ S,
                                                   const double *__restrict__ R,
                                                   const double *__restrict__ X,
                                                   double *__restrict__ Yeig,
                                                   double *__restrict__ theta, Params *prm) {
  __shared__ double lam[kMaxP];
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int i = tid; i < p; i += ENT) lam[i] = S[i * p + i] / (1.0 - R[i * p + i]);
  __syncthreads();
  for (int i = tid; i < p; i += ENT) {
    if (!isfinite(lam[i])) bad = 1;
    const int rk = desc_rank(lam, p, i);
    theta[rk] = lam[i];
    for (int r = 0; r < p; ++r) Yeig[r * p + rk] = X[r * p + i];
  }
  __syncthreads();
  if (tid == 0 && bad) atomicOr(&prm->flags, 4);
}

constexpr size_t kEig32Bytes = (size_t)3 * kMaxP * ELD * sizeof(float);
constexpr size_t kClusterBytes = (size_t)3 * kMaxP * ELD * sizeof(double);

}  // namespace

cudaError_t configure_eig() {
  cudaError_t e = cudaFuncSetAttribute(k_eig32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kEig32Bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_ref_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kClusterBytes);
}

// Eigenpairs of the p x p matrix H (row-major, symmetrised here): theta
// descending, eigenvectors in ws.Yeig (column j for theta_j).  Scratch:
// ws.Rinv (X), ws.T (H X), and the Gram workspace after H (S, R, E).
cudaError_t launch_eigensolve(cudaStream_t s, const Workspace &ws, const double *H, int p,
                              double *theta) {
  double *X = ws.Rinv, *AX = ws.T;
  double *S = ws.gpart + (size_t)p * p;
  double *R = S + (size_t)p * p;
  double *E = R + (size_t)p * p;
  cudaError_t e;
#define PF_EIG_CHECK()            \
  PF_LAUNCHED();                  \
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_eig32<<<1, ENT, kEig32Bytes, s>>>(H, p, X, ws.prm);
  PF_EIG_CHECK();
  for (int it = 0; it < kRefineIters; ++it) {
    k_ref_ax<<<p, kMaxP, 0, s>>>(H, p, X, AX);
    PF_EIG_CHECK();
    k_ref_sr<<<p, kMaxP, 0, s>>>(p, X, AX, S, R);
    PF_EIG_CHECK();
    k_ref_e<<<1, ENT, 0, s>>>(H, p, S, R, E);
    PF_EIG_CHECK();
    k_ref_update<<<p, kMaxP, 0, s>>>(p, X, E);
    PF_EIG_CHECK();
    k_ref_ax<<<p, kMaxP, 0, s>>>(H, p, X, AX);
    PF_EIG_CHECK();
    k_ref_sr<<<p, kMaxP, 0, s>>>(p, X, AX, S, R);
    PF_EIG_CHECK();
    k_ref_cluster<<<1, ENT, kClusterBytes, s>>>(H, p, S, R, X);
    PF_EIG_CHECK();
  }
  k_ref_ax<<<p, kMaxP, 0, s>>>(H, p, X, AX);
  PF_EIG_CHECK();
  k_ref_sr<<<p, kMaxP, 0, s>>>(p, X, AX, S, R);
  PF_EIG_CHECK();
  k_ref_final<<<1, ENT, 0, s>>>(p, S, R, X, ws.Yeig, theta, ws.prm);
  PF_EIG_CHECK();
#undef PF_EIG_CHECK
  return cudaSuccess;
}

}  // namespace pf
