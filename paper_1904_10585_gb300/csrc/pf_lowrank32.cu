// fp32 filter products of the low-rank + sparse iteration matrix.
//
// In a low-precision context the d Chebyshev products (Sec. 2.1, Eq. (cheb))
// of the PSD-completion iteration matrix B = Uf diag(w) Uf^T + s S + shift I
// run in fp32 on the CUDA cores (64x the FP64 rate on GB300; a CSR SpMM with
// p <= 64 columns does not map onto tensor-core tiles); CholQR2 and the
// Rayleigh-Ritz step that follow stay FP64.  The kernels mirror the FP64
// ones: a Gram product Uf^T X with a fixed-order reduction, and the fused
// SpMM + low-rank + recurrence kernel.
#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int NT = 256;
constexpr int WPB = NT / 32;
constexpr int RC = 32;

// fp32 copy of an n x p FP64 block (row-major, ld = p on output)
__global__ void k_to_f32(const double *__restrict__ src, int64_t lds, int n, int p,
                         float *__restrict__ dst) {
  const int64_t total = (int64_t)n * p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / p;
    const int j = (int)(idx - i * p);
    dst[idx] = (float)src[i * lds + j];
  }
}

template <int PT>
__global__ void __launch_bounds__(NT) k_gram32(const float *__restrict__ X, int px,
                                               const float *__restrict__ Y, int py, int n,
                                               int rows_per_block, float *__restrict__ gpart) {
  constexpr int TM = PT / 16, TN = PT / 16;
  __shared__ float Xs[RC][PT + 1];
  __shared__ float Ys[RC][PT + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(n, r0 + rows_per_block);
  for (int rb = r0; rb < r1; rb += RC) {
    for (int e = tid; e < RC * PT; e += NT) {
      const int r = e / PT, c = e % PT, gr = rb + r;
      Xs[r][c] = (gr < r1 && c < px) ? X[(int64_t)gr * px + c] : 0.f;
      Ys[r][c] = (gr < r1 && c < py) ? Y[(int64_t)gr * py + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < RC; ++r) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = Xs[r][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Ys[r][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *out = gpart + (int64_t)blockIdx.x * px * py;
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

// T[l][j] = w_l * sum_q gpart[q][l][j] (w clamped at 0 when `clamp`)
__global__ void k_lowrank_coef32(const float *__restrict__ gpart, int nparts,
                                 const double *__restrict__ lam, int r, int p, int clamp,
                                 float *__restrict__ T) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= r * p) return;
  float s = 0.f;
  for (int q = 0; q < nparts; ++q) s += gpart[(int64_t)q * r * p + idx];
  double w = lam[idx / p];
  if (clamp) w = w > 0.0 ? w : 0.0;
  T[idx] = (float)w * s;
}

template <int JG>
__global__ void __launch_bounds__(NT) k_lrsp_apply32(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ svals, int n, int p, const float *__restrict__ Uf, int r,
    const float *__restrict__ T, float sscale, float shift, const float *X, const float *Yprev,
    float *Ynext, const Params *__restrict__ prm, int mode) {
  __shared__ float Ts[kMaxP * kMaxP];
  for (int idx = threadIdx.x; idx < r * p; idx += NT) Ts[idx] = T[idx];
  __syncthreads();
  float c = 0.f, alpha = 1.f;
  if (mode != MODE_PLAIN) {
    c = (float)prm->c;
    alpha = (float)((mode == MODE_FIRST ? 1.0 : 2.0) / prm->e);
  }
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const int warps = gridDim.x * WPB;
  for (int row = blockIdx.x * WPB + (threadIdx.x >> 5); row < n; row += warps) {
    float acc[JG], lr[JG];
#pragma unroll
    for (int g = 0; g < JG; ++g) acc[g] = lr[g] = 0.f;
    if (svals != nullptr) {
      const int e0 = rowptr[row], e1 = rowptr[row + 1];
      for (int base = e0; base < e1; base += 32) {
        const int my = base + lane;
        const int mcol = my < e1 ? colind[my] : 0;
        const float mv = my < e1 ? (float)svals[my] : 0.f;
        const int cnt = min(32, e1 - base);
        for (int k = 0; k < cnt; k += 2) {
          const int kk = k + half;
          const int col = __shfl_sync(0xffffffffu, mcol, kk);
          const float v = __shfl_sync(0xffffffffu, mv, kk);
          const float *xr = X + (int64_t)col * p;
#pragma unroll
          for (int g = 0; g < JG; ++g) {
            const int j = hl + 16 * g;
            if (j < p) acc[g] = fmaf(v, xr[j], acc[g]);
          }
        }
      }
    }
    const float *ur = Uf + (int64_t)row * r;
    for (int l = half; l < r; l += 2) {
      const float u = ur[l];
#pragma unroll
      for (int g = 0; g < JG; ++g) {
        const int j = hl + 16 * g;
        if (j < p) lr[g] = fmaf(u, Ts[l * p + j], lr[g]);
      }
    }
#pragma unroll
    for (int g = 0; g < JG; ++g) {
      acc[g] += __shfl_xor_sync(0xffffffffu, acc[g], 16);
      lr[g] += __shfl_xor_sync(0xffffffffu, lr[g], 16);
    }
    if (half == 0) {
#pragma unroll
      for (int g = 0; g < JG; ++g) {
        const int j = hl + 16 * g;
        if (j >= p) continue;
        const int64_t o = (int64_t)row * p + j;
        const float xij = X[o];
        const float v = lr[g] + sscale * acc[g] + shift * xij;
        float y;
        if (mode == MODE_PLAIN) y = v;
        else {
          y = alpha * (v - c * xij);
          if (mode == MODE_RECUR) y -= Yprev[o];
        }
        Ynext[o] = y;
      }
    }
  }
}

}  // namespace

cudaError_t launch_to_f32(cudaStream_t s, const Workspace &ws, const double *src, int64_t lds,
                          int n, int p, float *dst) {
  int64_t blocks = ((int64_t)n * p + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  if (blocks < 1) blocks = 1;
  k_to_f32<<<(int)blocks, 256, 0, s>>>(src, lds, n, p, dst);
  PF_LAUNCHED();
  return cudaGetLastError();
}

// One fp32 product of the low-rank + sparse operator with the recurrence
// epilogue.  Uf32 (n x r) is the fp32 copy of the low-rank factor; X, Yprev,
// Ynext are fp32 n x p (ld = p).
cudaError_t launch_lowrank_sparse_apply32(cudaStream_t s, const Workspace &ws, const Op &op,
                                          const float *Uf32, const float *X, const float *Yprev,
                                          float *Ynext, int mode) {
  const int n = op.n, p = ws.p;
  int r = op.r;
  float *T32 = reinterpret_cast<float *>(ws.T);
  float *gp = reinterpret_cast<float *>(ws.gpart);
  if (r > 0 && Uf32 != nullptr) {
    int b = (n + 63) / 64;
    // at most 256 partials: k_lowrank_coef32 sums them in one sequence per entry
    if (b > 256) b = 256;
    if (b < 1) b = 1;
    int rpb = (n + b - 1) / b;
    rpb = ((rpb + RC - 1) / RC) * RC;
    const int nb = (n + rpb - 1) / rpb;
    const int pm = r > p ? r : p;
    if (pm <= 16) k_gram32<16><<<nb, NT, 0, s>>>(Uf32, r, X, p, n, rpb, gp);
    else if (pm <= 32) k_gram32<32><<<nb, NT, 0, s>>>(Uf32, r, X, p, n, rpb, gp);
    else if (pm <= 48) k_gram32<48><<<nb, NT, 0, s>>>(Uf32, r, X, p, n, rpb, gp);
    else k_gram32<64><<<nb, NT, 0, s>>>(Uf32, r, X, p, n, rpb, gp);
    PF_LAUNCHED();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_lowrank_coef32<<<(r * p + 255) / 256, 256, 0, s>>>(gp, nb, op.lam, r, p, op.clamp, T32);
    PF_LAUNCHED();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else {
    r = 0;
  }
  int blocks = (n + WPB - 1) / WPB;
  if (blocks > 8 * ws.num_sms) blocks = 8 * ws.num_sms;
  const float ss = (float)op.sscale, sh = (float)op.shift;
#define PF_LRSP32(JGV)                                                                           \
  k_lrsp_apply32<JGV><<<blocks, NT, 0, s>>>(op.rowptr, op.colind, op.vals, n, p, Uf32, r, T32, \
                                            ss, sh, X, Yprev, Ynext, ws.prm, mode)
  if (p <= 16) { PF_LRSP32(1); }
  else if (p <= 32) { PF_LRSP32(2); }
  else if (p <= 48) { PF_LRSP32(3); }
  else { PF_LRSP32(4); }
#undef PF_LRSP32
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
