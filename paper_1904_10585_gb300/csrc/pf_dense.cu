// Dense FP64 filter product Ynext = alpha (A X - c X) - beta Yprev.
//
// One Chebyshev step of Sec. 2.1 (Eq. (cheb) evaluated by the three-term
// recurrence in the mapped variable (A - cI)/e of Eq. (cheb-linear-map)).  The
// product A X (A dense symmetric n x n, X n x p with p <= 64) is a skinny GEMM
// whose arithmetic is FP64; on GB300 the FP64 pipe (about 1.1 TFLOP/s for the
// whole GPU) bounds it, not HBM (A is read once per product at ~6.7 TB/s).  The
// kernel therefore aims at keeping every SM's FP64 pipe busy:
//   * split-K over (row block, K chunk) work units, sized to ~8 units per SM,
//     so all 152 SMs stay loaded for n of a few thousand;
//   * 64 x BN register-tiled CTAs (4 x BN/16 accumulators per thread);
//   * partial products summed in a fixed order by the epilogue kernel, which
//     also applies the recurrence -- the result is deterministic.
#include "pf_internal.cuh"

namespace pf {

namespace {

constexpr int BM = 64;
constexpr int BK = 16;
constexpr int NT = 256;

template <int BN>
__global__ void __launch_bounds__(NT) k_gemm_f64_splitk(const double *__restrict__ A, int64_t lda,
                                                        const double *__restrict__ X, int64_t ldx,
                                                        int n, int p, int kchunk,
                                                        double *__restrict__ part) {
  constexpr int TM = 4, TN = BN / 16;
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Xs[2][BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int row0 = blockIdx.x * BM;
  const int k0 = blockIdx.y * kchunk;
  const int k1 = min(n, k0 + kchunk);
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  // register staging for the next tile
  double ra[4], rx[(BK * BN + NT - 1) / NT];
  auto load_regs = [&](int kb) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + NT * q, m = e >> 4, k = e & 15;
      const int gr = row0 + m, gk = kb + k;
      ra[q] = (gr < n && gk < k1) ? __ldg(A + (int64_t)gr * lda + gk) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < (BK * BN + NT - 1) / NT; ++q) {
      const int e = tid + NT * q;
      const int k = e / BN, j = e % BN, gk = kb + k;
      rx[q] = (e < BK * BN && gk < k1 && j < p) ? __ldg(X + (int64_t)gk * ldx + j) : 0.0;
    }
  };
  auto store_regs = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + NT * q, m = e >> 4, k = e & 15;
      As[buf][k][m] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < (BK * BN + NT - 1) / NT; ++q) {
      const int e = tid + NT * q;
      if (e < BK * BN) Xs[buf][e / BN][e % BN] = rx[q];
    }
  };

  int buf = 0;
  if (k0 < k1) {
    load_regs(k0);
    store_regs(0);
  }
  __syncthreads();
  for (int kb = k0; kb < k1; kb += BK) {
    const bool more = kb + BK < k1;
    if (more) load_regs(kb + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][k][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Xs[buf][k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) store_regs(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  double *out = part + (int64_t)blockIdx.y * n * p;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = row0 + ty * TM + i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = tx + 16 * j;
      if (c < p) out[(int64_t)r * p + c] = acc[i][j];
    }
  }
}

// Ynext = alpha (sum_s part[s] - c X) - beta Yprev, summing splits in order.
__global__ void k_combine(const double *__restrict__ part, int S, int n, int p,
                          const double *X, int64_t ldx, const double *Yprev, int64_t ldp,
                          double *Ynext, int64_t ldn, const Params *__restrict__ prm, int mode) {
  const int64_t total = (int64_t)n * p;
  double c = 0.0, alpha = 1.0, beta = 0.0;
  if (mode != MODE_PLAIN) {
    c = prm->c;
    alpha = (mode == MODE_FIRST ? 1.0 : 2.0) / prm->e;
    beta = (mode == MODE_RECUR) ? 1.0 : 0.0;
  }
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / p;
    const int j = (int)(idx - i * p);
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += part[(int64_t)q * total + idx];
    double y;
    if (mode == MODE_PLAIN) {
      y = s;
    } else {
      y = alpha * (s - c * X[i * ldx + j]);
      if (mode == MODE_RECUR) y -= beta * Yprev[i * ldp + j];
    }
    Ynext[i * ldn + j] = y;
  }
}

__global__ void k_set_interval(Params *prm, double a, double b) {
  prm->flags = 0;
  prm->a = a;
  prm->b = b;
  prm->c = 0.5 * (a + b);
  prm->e = 0.5 * (b - a);
}

__global__ void k_set_scale(Params *prm, double lp_scale) { prm->lp_scale = lp_scale; }

}  // namespace

cudaError_t launch_set_scale(cudaStream_t s, Params *prm, double lp_scale) {
  k_set_scale<<<1, 1, 0, s>>>(prm, lp_scale);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_set_interval(cudaStream_t s, Params *prm, double a, double b) {
  k_set_interval<<<1, 1, 0, s>>>(prm, a, b);
  PF_LAUNCHED();
  return cudaGetLastError();
}

// Number of K splits for an n x n by n x p product: about 8 work units per SM.
int dense_splits(int n, int num_sms, int *kchunk) {
  const int row_blocks = (n + BM - 1) / BM;
  const int ktiles = (n + BK - 1) / BK;
  int S = (8 * num_sms + row_blocks - 1) / row_blocks;
  S = S < 1 ? 1 : S;
  S = S > kMaxSplitK ? kMaxSplitK : S;
  S = S > ktiles ? ktiles : S;
  const int tiles_per = (ktiles + S - 1) / S;
  *kchunk = tiles_per * BK;
  return (n + *kchunk - 1) / *kchunk;
}

cudaError_t launch_dense_apply(cudaStream_t s, const Workspace &ws, const Op &op, const double *X,
                               int64_t ldx, const double *Yprev, int64_t ldp, double *Ynext,
                               int64_t ldn, int mode) {
  const int n = op.n, p = ws.p;
  int kchunk = 0;
  const int S = dense_splits(n, ws.num_sms, &kchunk);
  dim3 grid((n + BM - 1) / BM, S);
  if (p <= 16)
    {
      k_gemm_f64_splitk<16><<<grid, NT, 0, s>>>(op.A, op.lda, X, ldx, n, p, kchunk, ws.part);
      PF_LAUNCHED();
    }
  else if (p <= 32)
    {
      k_gemm_f64_splitk<32><<<grid, NT, 0, s>>>(op.A, op.lda, X, ldx, n, p, kchunk, ws.part);
      PF_LAUNCHED();
    }
  else
    {
      k_gemm_f64_splitk<64><<<grid, NT, 0, s>>>(op.A, op.lda, X, ldx, n, p, kchunk, ws.part);
      PF_LAUNCHED();
    }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)n * p;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  k_combine<<<blocks, 256, 0, s>>>(ws.part, S, n, p, X, ldx, Yprev, ldp, Ynext, ldn, ws.prm, mode);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf

// ===========================================================================
// Allocation-free dense product (no counterpart in the paper).
//
// Y = A X with the split-K partial sums kept in a file-scope device array
// instead of a context's workspace, for callers that cannot allocate device
// memory themselves.  The array is part of the library image: every GPU on
// which the library is loaded holds it until the process exits.
// ===========================================================================
#include <mutex>

namespace pf {
namespace {

constexpr int64_t kStaticScratchDoubles = (int64_t)2 << 20;  // 2 Mi doubles = 16 MiB
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_static_mutex;
int g_static_sms[kStaticMaxDevices] = {};

// Device address of the scratch array (and SM count) for the current device.
// In host code the array's name only stands in for the device copy, so the
// address comes from cudaGetSymbolAddress with the device current.  It is
// looked up on every call (a host-side lookup, no device work), so a new
// context after cudaDeviceReset gets the array's new address; only the SM
// count, a property of the device, is remembered.
pf_status static_scratch_for_current_device(double **addr, int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PF_ERR_CUDA;
  if (dev < 0 || dev >= kStaticMaxDevices) return PF_ERR_UNSUPPORTED;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr)
    return PF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (g_static_sms[dev] == 0) {
    int count = 0;
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return PF_ERR_CUDA;
    g_static_sms[dev] = count;
  }
  *addr = (double *)p;
  *sms = g_static_sms[dev];
  return PF_OK;
}

}  // namespace
}  // namespace pf

extern "C" pf_status pf_apply_dense_noalloc(const double *A, int64_t lda, const double *X,
                                            int64_t ldx, double *Y, int64_t ldy, int64_t n,
                                            int32_t p, void *stream) {
  using namespace pf;
  if (!A || !X || !Y || X == Y || n < 1 || n > (int64_t)INT32_MAX / 2 || p < 1 || p > kMaxP ||
      lda < n || ldx < p || ldy < p)
    return PF_ERR_INVALID_ARG;
  if (n * (int64_t)p > kStaticScratchDoubles) return PF_ERR_INVALID_ARG;
  // an error left pending by someone else's earlier launch belongs to its
  // owner: report it without clearing it, and launch nothing
  if (cudaPeekAtLastError() != cudaSuccess) return PF_ERR_CUDA;
  double *scratch = nullptr;
  int sms = 0;
  const pf_status st = static_scratch_for_current_device(&scratch, &sms);
  if (st != PF_OK) return st;
  const int ni = (int)n;
  // as many K splits as the workspace path would use, capped by the array
  int kchunk = 0;
  int S = dense_splits(ni, sms, &kchunk);
  const int64_t fit = kStaticScratchDoubles / (n * (int64_t)p);
  if (S > fit) {
    const int ktiles = (ni + BK - 1) / BK;
    const int tiles_per = (int)((ktiles + fit - 1) / fit);
    kchunk = tiles_per * BK;
    S = (ni + kchunk - 1) / kchunk;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 grid((ni + BM - 1) / BM, S);
  if (p <= 16)
    k_gemm_f64_splitk<16><<<grid, NT, 0, s>>>(A, lda, X, ldx, ni, p, kchunk, scratch);
  else if (p <= 32)
    k_gemm_f64_splitk<32><<<grid, NT, 0, s>>>(A, lda, X, ldx, ni, p, kchunk, scratch);
  else
    k_gemm_f64_splitk<64><<<grid, NT, 0, s>>>(A, lda, X, ldx, ni, p, kchunk, scratch);
  if (cudaGetLastError() != cudaSuccess) return PF_ERR_CUDA;
  PF_LAUNCHED();
  const int64_t total = n * p;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4 * sms) blocks = 4 * sms;
  // MODE_PLAIN reads no device parameters
  k_combine<<<blocks, 256, 0, s>>>(scratch, S, ni, p, X, ldx, nullptr, 0, Y, ldy, nullptr,
                                   MODE_PLAIN);
  if (cudaGetLastError() != cudaSuccess) return PF_ERR_CUDA;
  PF_LAUNCHED();
  return PF_OK;
}
