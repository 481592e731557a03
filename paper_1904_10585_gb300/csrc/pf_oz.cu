// FP64-accurate dense filter product on the 5th-generation tensor cores by
// error-free slicing: the splitting idea of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012) with bf16 slices and fp32 accumulation.
//
// One Chebyshev step (Sec. 2.1, Eq. (cheb), by the three-term recurrence in
// the mapped variable (A - cI)/e of Eq. (cheb-linear-map)) with the dense
// FP64 iteration matrix A (n x n) and block X (n x p):
//     Ynext = alpha (A X - c X) - beta Yprev.
//
// Slices.  Row i of A gets the exponent eA_i with |A_ij| < 2^eA_i; each entry
// is rounded to the integer round(A_ij 2^(55 - eA_i)) (|.| <= 2^55), whose
// balanced base-256 digits a_0..a_6 (a_0 in [-128, 128], the rest in
// [-128, 127]) give A_ij ~ 2^(eA_i - 7) sum_s a_s 2^(-8s), error <= 2^(eA_i - 56).
// X is cut the same way per (128-row chunk c, column j) with exponent eX_cj.
// Every digit is an integer of at most 8 significant bits, exact in bf16.
//
// Products.  For a chunk c of 128 values of k, the level sums
//     L_l = sum_{s + t = l} sum_{k in c} a_s(i,k) x_t(k,j),   l = 0..6,
// are integers with |L_l| <= 7 * 128 * 2^14 < 2^24, so the tensor cores'
// fp32 accumulation of the (exact) bf16 products is exact.  Pairs with
// s + t >= 7 are dropped: each weighs <= 2^(eA_i + eX_cj - 56).  The chunk's
// value 2^(eA_i + eX_cj - 14) sum_l L_l 2^(-8l) is folded into one int64 of
// resolution 2^(eA_i + eX_cj - 50) (levels 5 and 6 rounded), shifted to the
// largest exponent of column j in the split, and summed over the split's
// chunks in int64 (exact).  Per output entry the error is a few units of
// 2^(eA_i + max_c eX_cj - 53) per term of the sum, the order of an FP64 dot
// product's rounding bound.
//
// Tensor-core mapping (per CTA: one 128-row block of A, one K split):
//   warp 0, one lane : TMA producer.  Per 64-wide K tile: the 7 digit planes
//                      of X (one stage, 7 x NB rows) and, one stage each,
//                      the 7 digit planes of the A tile (128 x 64 bf16).
//   warp 1, one lane : MMA issuer.  A-plane s times the stacked X planes
//                      0..6-s in one tcgen05.mma of N = (7 - s) NB (split in
//                      runs of N <= 256), accumulating into TMEM columns
//                      [s NB, 7 NB): level l lives at columns l NB.  Two
//                      accumulator sets (one for NB > 32) alternate per chunk.
//   warps 2..        : epilogue.  Per chunk: tcgen05.ld of the 7 levels,
//                      fold to int64, release the accumulator set.  At the
//                      end: the split's FP64 partial; the last CTA of a row
//                      block (atomic ticket, no waiting) sums the partials in
//                      split order, applies the recurrence and, when asked,
//                      cuts the new block's rows into the digit planes of
//                      the next product.
// Every wait is bounded (about 2 s); on expiry the CTA sets flags bit 3 in
// the context parameters, lets its copies and MMAs land, frees its TMEM and
// returns.
#include <climits>
#include <cuda.h>
#include <cuda_bf16.h>

#include "pf_internal.cuh"
#include "pf_sm100.cuh"

namespace pf {

namespace {

constexpr int OZ_BM = 128;               // rows per tile and K per chunk
constexpr int OZ_BK = 64;                // K per TMA tile (128 bytes of bf16)
constexpr int OZ_A_BYTES = OZ_BM * 128;  // one A digit-plane tile
constexpr int OZ_SB = 2;                 // stages of the X planes
constexpr int OZ_FRAC = 8 * (kOzSlices - 1) + 7;  // fractional bits of the rounded entry
constexpr int OZ_FOLD = 36;              // binary point of the int64 fold (level 0)

template <int NB>
struct OzCfg {
  static constexpr int EPI = NB <= 32 ? 4 : 8;   // epilogue warps (two per lane quarter above 32)
  static constexpr int THREADS = 64 + 32 * EPI;
  static constexpr int CW = NB / (EPI / 4);      // columns per epilogue thread
  static constexpr int LEVEL_COLS = kOzSlices * NB;
  static constexpr int NBUF = 2 * LEVEL_COLS <= 512 ? 2 : 1;
  static constexpr uint32_t TMEM_COLS = NBUF * LEVEL_COLS <= 256 ? 256u : 512u;
  static constexpr int SA = NB <= 32 ? 8 : 6;    // A stages
  static constexpr int B_BYTES = kOzSlices * NB * 128;
  static constexpr int MAXRUN = 256 / NB;        // X planes per MMA (N <= 256)
  static constexpr size_t SMEM = 1024 + (size_t)SA * OZ_A_BYTES + (size_t)OZ_SB * B_BYTES;
};

// Biased exponent field of |x|.
__device__ __forceinline__ unsigned oz_exfield(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}
// Exponent e with |x| < 2^e for every x whose exponent field is <= f.
__device__ __forceinline__ int oz_exponent(unsigned f) {
  return f == 0x7FFu ? kOzExpBad : (int)(f > 1u ? f : 1u) - 1022;
}

// Balanced base-256 digits of round(x 2^(OZ_FRAC - e)) for |x| < 2^e:
// x ~ 2^(e - 7) sum_s d[s] 2^(-8s).  Integer arithmetic only.
__device__ __forceinline__ void oz_digits(double x, int e, int *d) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long m = bits & 0xFFFFFFFFFFFFFll;
  if (ex != 0) m |= 1ll << 52;
  // x = m 2^(max(ex,1) - 1075); the scaled value is m 2^sh, sh <= 2
  const int sh = (ex > 1 ? ex : 1) - 1075 + OZ_FRAC - e;
  long long v;
  if (sh >= 0) v = m << sh;
  else if (sh > -60) v = (m + (1ll << (-sh - 1))) >> (-sh);
  else v = 0;
  if (bits < 0) v = -v;
#pragma unroll
  for (int s = kOzSlices - 1; s > 0; --s) {
    const int dd = ((int)(v & 0xFF) ^ 0x80) - 0x80;  // low byte as a value in [-128, 127]
    d[s] = dd;
    v = (v - dd) >> 8;
  }
  d[0] = (int)v;
}

__device__ __forceinline__ __nv_bfloat16 oz_bf16(int d) {
  return __float2bfloat16_rn((float)d);  // exact: |d| <= 128
}

// round(v / 2^s) for s >= 0
__device__ __forceinline__ long long oz_rshift(long long v, int s) {
  if (s <= 0) return v;
  if (s >= 62) return 0;
  return (v + (1ll << (s - 1))) >> s;
}

// Instruction descriptor: fp32 accumulator, bf16 A and B (K-major), M = 128.
__device__ __forceinline__ uint32_t oz_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void epi_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// ---------------------------------------------------------------------------
// A (n x n FP64) -> digit planes zs[s][i][k] (bf16, plane stride slice_rows
// rows of ldk) and row exponents ez[i].  One warp per row.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_oz_zslice(const double *__restrict__ A, int64_t lda,
                                                   int n, __nv_bfloat16 *__restrict__ zs,
                                                   int64_t ldk, int64_t slice_rows,
                                                   int *__restrict__ ez) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= n) return;
  const double *ar = A + (int64_t)row * lda;
  unsigned f = 0;
  for (int k = lane; k < n; k += 32) f = max(f, oz_exfield(ar[k]));
  f = __reduce_max_sync(0xffffffffu, f);
  const int e = oz_exponent(f);
  if (lane == 0) ez[row] = e;
  __nv_bfloat16 *zr = zs + (int64_t)row * ldk;
  for (int k = lane; k < n; k += 32) {
    int d[kOzSlices];
    if (e != kOzExpBad) {
      oz_digits(ar[k], e, d);
    } else {
#pragma unroll
      for (int s = 0; s < kOzSlices; ++s) d[s] = 0;
    }
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s) zr[s * slice_rows * ldk + k] = oz_bf16(d[s]);
  }
}

// ---------------------------------------------------------------------------
// X (n x p FP64) -> digit planes xs[t][j][k] (bf16, plane t of NB rows j,
// ldk) and exponents ex[c * kMaxP + j] of each 128-row chunk c and column j
// (columns p..NB-1 are zero).  One CTA of 128 threads per chunk, thread =
// row.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_oz_xslice(const double *__restrict__ X, int64_t ldx,
                                                   int n, int p, int NB,
                                                   __nv_bfloat16 *__restrict__ xs, int64_t ldk,
                                                   int *__restrict__ ex) {
  __shared__ unsigned qmax[4][kMaxP];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int row = blockIdx.x * OZ_BM + t;
  const bool in = row < n;
  const double *xr = X + (int64_t)row * ldx;
  for (int j = 0; j < NB; ++j) {
    const unsigned f = (in && j < p) ? oz_exfield(xr[j]) : 0u;
    const unsigned m = __reduce_max_sync(0xffffffffu, f);
    if (lane == 0) qmax[w][j] = m;
  }
  __syncthreads();
  for (int j = 0; j < NB; ++j) {
    const unsigned m = max(max(qmax[0][j], qmax[1][j]), max(qmax[2][j], qmax[3][j]));
    const int e = oz_exponent(m);
    if (t == 0) ex[blockIdx.x * kMaxP + j] = e;
    int d[kOzSlices];
    if (in && j < p && e != kOzExpBad) {
      oz_digits(xr[j], e, d);
    } else {
#pragma unroll
      for (int s = 0; s < kOzSlices; ++s) d[s] = 0;
    }
    if (in) {
#pragma unroll
      for (int s = 0; s < kOzSlices; ++s) xs[(int64_t)(s * NB + j) * ldk + row] = oz_bf16(d[s]);
    }
  }
}

// ---------------------------------------------------------------------------
// The sliced product with the recurrence epilogue (see the file comment).
// Grid (row blocks, K splits).
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(OzCfg<NB>::THREADS, 1) k_oz_product(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int n,
    int p, int slice_rows, int nsplit, const int *__restrict__ ez, const int *__restrict__ ex,
    double *__restrict__ part, int *__restrict__ cnt, const double *X, int64_t ldx,
    const double *Yprev, int64_t ldp, double *Ynext, int64_t ldn,
    __nv_bfloat16 *__restrict__ xs_next, int *__restrict__ ex_next, int64_t ldk, Params *prm,
    int mode) {
  using C = OzCfg<NB>;
  constexpr int KS = kOzSlices;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t a_full[C::SA], a_empty[C::SA];
  __shared__ __align__(8) uint64_t b_full[OZ_SB], b_empty[OZ_SB];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int is_last;
  __shared__ int dsh[kOzMaxChunks][NB];  // per chunk and column: shift to the split's exponent
  __shared__ int exmax[NB];
  __shared__ unsigned qmax[4][NB];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.x, split = blockIdx.y;
  const int nchunks = (n + OZ_BM - 1) / OZ_BM;
  const int c0 = (int)((int64_t)split * nchunks / nsplit);
  const int c1 = (int)((int64_t)(split + 1) * nchunks / nsplit);
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sA = base;
  const uint32_t sB = base + C::SA * OZ_A_BYTES;

  for (int j = threadIdx.x; j < NB; j += blockDim.x) {
    int m = INT_MIN;
    for (int c = c0; c < c1; ++c) m = max(m, ex[c * kMaxP + j]);
    exmax[j] = m;
  }
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < C::SA; ++s) {
      mbar_init(smem_u32(&a_full[s]), 1);
      mbar_init(smem_u32(&a_empty[s]), 1);
    }
    for (int s = 0; s < OZ_SB; ++s) {
      mbar_init(smem_u32(&b_full[s]), 1);
      mbar_init(smem_u32(&b_empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&acc_full[s]), 1);
      mbar_init(smem_u32(&acc_empty[s]), C::EPI);
    }
    mbar_init(smem_u32(&mma_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < (c1 - c0) * NB; idx += blockDim.x) {
    const int c = idx / NB, j = idx - c * NB;
    dsh[c][j] = exmax[j] - ex[(c0 + c) * kMaxP + j];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int ia = 0, ib = 0;
      bool ok = true;
      for (int c = c0; c < c1 && ok; ++c) {
        for (int h = 0; h < 2 && ok; ++h) {
          const int kx = (2 * c + h) * OZ_BK;
          const int sb = ib % OZ_SB;
          if (ib >= OZ_SB &&
              !mbar_wait(smem_u32(&b_empty[sb]), ((ib / OZ_SB) - 1) & 1, &abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t fb = smem_u32(&b_full[sb]);
          mbar_expect_tx(fb, C::B_BYTES);
#pragma unroll
          for (int t = 0; t < KS; ++t)
            tma_load_2d(sB + sb * C::B_BYTES + t * NB * 128, &tmB, fb, kx, t * NB);
          ++ib;
          for (int s = 0; s < KS; ++s) {
            const int sa = ia % C::SA;
            if (ia >= C::SA &&
                !mbar_wait(smem_u32(&a_empty[sa]), ((ia / C::SA) - 1) & 1, &abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t fa = smem_u32(&a_full[sa]);
            mbar_expect_tx(fa, OZ_A_BYTES);
            tma_load_2d(sA + sa * OZ_A_BYTES, &tmA, fa, kx, s * slice_rows + rb * OZ_BM);
            ++ia;
          }
        }
      }
      // let every issued copy land before shared memory is released
      for (int s = 0; s < C::SA && s < ia; ++s) {
        const int last = s + ((ia - 1 - s) / C::SA) * C::SA;
        mbar_drain(smem_u32(&a_full[s]), (last / C::SA) & 1);
      }
      for (int s = 0; s < OZ_SB && s < ib; ++s) {
        const int last = s + ((ib - 1 - s) / OZ_SB) * OZ_SB;
        mbar_drain(smem_u32(&b_full[s]), (last / OZ_SB) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int ia = 0, ib = 0, cc = 0;
      bool ok = true;
      for (int c = c0; c < c1 && ok; ++c, ++cc) {
        const int buf = cc % C::NBUF;
        if (cc >= C::NBUF &&
            !mbar_wait(smem_u32(&acc_empty[buf]), ((cc / C::NBUF) - 1) & 1, &abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dbase = tmem + (uint32_t)(buf * C::LEVEL_COLS);
        for (int h = 0; h < 2 && ok; ++h) {
          const int sb = ib % OZ_SB;
          if (!mbar_wait(smem_u32(&b_full[sb]), (ib / OZ_SB) & 1, &abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t bbase = sB + sb * C::B_BYTES;
          for (int s = 0; s < KS; ++s) {
            const int sa = ia % C::SA;
            if (!mbar_wait(smem_u32(&a_full[sa]), (ia / C::SA) & 1, &abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ad = sw128_desc(sA + sa * OZ_A_BYTES);
            for (int r0 = 0; r0 < KS - s; r0 += C::MAXRUN) {
              const int ns = min(C::MAXRUN, KS - s - r0);
              const uint32_t idesc = oz_idesc(ns * NB);
              const uint64_t bd = sw128_desc(bbase + r0 * NB * 128);
              const uint32_t d = dbase + (uint32_t)((s + r0) * NB);
#pragma unroll
              for (int k = 0; k < 4; ++k)  // 16 bf16 of K per instruction: +32 bytes
                mma_issue<false>(d, ad + 2 * k, bd + 2 * k, idesc, (h | s | k) != 0 ? 1u : 0u);
            }
            mma_commit(smem_u32(&a_empty[sa]));
            ++ia;
          }
          if (!ok) break;
          mma_commit(smem_u32(&b_empty[sb]));
          ++ib;
        }
        if (ok) mma_commit(smem_u32(&acc_full[buf]));
      }
      // completion of every MMA issued above, before TMEM is freed
      mma_commit(smem_u32(&mma_done));
      mbar_drain(smem_u32(&mma_done), 0);
    }
  } else {
    // ---------------- epilogue ----------------
    constexpr int CW = C::CW;
    const int ew = warp - 2;
    const int q = warp & 3;           // TMEM lane quarter this warp may read
    const int col0 = (ew >> 2) * CW;  // its columns
    const int rl = q * 32 + lane;
    const int row = rb * OZ_BM + rl;
    long long acc[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) acc[j] = 0;
    int cc = 0;
    for (int c = c0; c < c1; ++c, ++cc) {
      const int buf = cc % C::NBUF;
      if (!mbar_wait(smem_u32(&acc_full[buf]), (cc / C::NBUF) & 1, &abort_flag)) break;
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr =
          tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * C::LEVEL_COLS + col0);
#pragma unroll
      for (int g = 0; g < CW; g += 8) {
        uint32_t L[KS][8];
#pragma unroll
        for (int l = 0; l < KS; ++l) tmem_ld8(taddr + l * NB + g, L[l]);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          long long v = 0;
#pragma unroll
          for (int l = 0; l < KS; ++l) {
            const int li = __float2int_rn(__uint_as_float(L[l][i]));  // exact integer
            const int s = OZ_FOLD - 8 * l;
            if (s >= 0) v += (long long)li << s;
            else v += (long long)((li + (1 << (-s - 1))) >> (-s));
          }
          acc[g + i] += oz_rshift(v, dsh[cc][col0 + g + i]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
    }

    // this split's values: acc 2^(eA_i + exmax_j - 14 - OZ_FOLD)
    const bool in = row < n;
    const int ea = in ? ez[row] : 0;
    double y[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) {
      const int e2 = exmax[col0 + j];
      y[j] = (ea == kOzExpBad || e2 == kOzExpBad)
                 ? __longlong_as_double(0x7FF8000000000000ll)
                 : ldexp((double)acc[j], ea + e2 - 14 - OZ_FOLD);
    }
    bool last = true;
    if (nsplit > 1) {
      if (in) {
        double *pr = part + ((int64_t)split * n + row) * p;
#pragma unroll
        for (int j = 0; j < CW; ++j)
          if (col0 + j < p) pr[col0 + j] = y[j];
      }
      __threadfence();
      epi_sync(32 * C::EPI);
      if (ew == 0 && lane == 0) is_last = atomicAdd(&cnt[rb], 1) == nsplit - 1;
      epi_sync(32 * C::EPI);
      last = is_last != 0;
      if (last) {
        __threadfence();
        if (in) {
#pragma unroll
          for (int j = 0; j < CW; ++j) y[j] = 0.0;
          for (int sp = 0; sp < nsplit; ++sp) {
            const double *pr = part + ((int64_t)sp * n + row) * p;
#pragma unroll
            for (int j = 0; j < CW; ++j)
              if (col0 + j < p) y[j] += __ldcg(pr + col0 + j);
          }
        }
        if (ew == 0 && lane == 0) cnt[rb] = 0;  // ready for the next launch
      }
    }
    if (last) {
      double cval = 0.0, alpha = 1.0;
      if (mode != MODE_PLAIN) {
        cval = prm->c;
        alpha = (mode == MODE_FIRST ? 1.0 : 2.0) / prm->e;
      }
      if (in) {
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          const int jj = col0 + j;
          if (jj >= p) continue;
          double v = y[j];
          if (mode != MODE_PLAIN) {
            v = alpha * (v - cval * X[(int64_t)row * ldx + jj]);
            if (mode == MODE_RECUR) v -= Yprev[(int64_t)row * ldp + jj];
          }
          Ynext[(int64_t)row * ldn + jj] = v;
          y[j] = v;
        }
      }
      if (xs_next != nullptr) {
        // digit planes of the new block's rows for the next product
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          const unsigned f = (in && col0 + j < p) ? oz_exfield(y[j]) : 0u;
          const unsigned m = __reduce_max_sync(0xffffffffu, f);
          if (lane == 0) qmax[q][col0 + j] = m;
        }
        epi_sync(32 * C::EPI);
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          const int jj = col0 + j;
          const int e =
              oz_exponent(max(max(qmax[0][jj], qmax[1][jj]), max(qmax[2][jj], qmax[3][jj])));
          if (rl == 0) ex_next[rb * kMaxP + jj] = e;
          int d[KS];
          if (in && jj < p && e != kOzExpBad) {
            oz_digits(y[j], e, d);
          } else {
#pragma unroll
            for (int s = 0; s < KS; ++s) d[s] = 0;
          }
          if (in) {
#pragma unroll
            for (int s = 0; s < KS; ++s) xs_next[(int64_t)(s * NB + jj) * ldk + row] = oz_bf16(d[s]);
          }
        }
      }
    }
  }

  if (threadIdx.x == 0 && abort_flag) atomicOr(&prm->flags, 8);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}

template <int NB>
cudaError_t oz_set_attr() {
  return cudaFuncSetAttribute(k_oz_product<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)OzCfg<NB>::SMEM);
}

int oz_nb(int p) { return p <= 16 ? 16 : p <= 32 ? 32 : p <= 48 ? 48 : 64; }

}  // namespace

cudaError_t configure_oz() {
  cudaError_t e;
  if ((e = oz_set_attr<16>()) != cudaSuccess) return e;
  if ((e = oz_set_attr<32>()) != cudaSuccess) return e;
  if ((e = oz_set_attr<48>()) != cudaSuccess) return e;
  return oz_set_attr<64>();
}

int oz_splits(int n, int num_sms) {
  const int R = (n + OZ_BM - 1) / OZ_BM;
  int S = num_sms / R;
  if (S > kOzMaxSplits) S = kOzMaxSplits;
  if (S > R) S = R;
  const int need = (R + kOzMaxChunks - 1) / kOzMaxChunks;  // int64 headroom of the fold
  if (S < need) S = need;
  return S < 1 ? 1 : S;
}

cudaError_t launch_oz_zslice(cudaStream_t s, const Workspace &ws, const double *A, int64_t lda,
                             int n) {
  if (ws.oz.zs == nullptr || n > ws.oz.slice_rows) return cudaErrorInvalidValue;
  k_oz_zslice<<<(n + 7) / 8, 256, 0, s>>>(A, lda, n, (__nv_bfloat16 *)ws.oz.zs, ws.oz.ldk,
                                          ws.oz.slice_rows, ws.oz.ez);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_oz_xslice(cudaStream_t s, const Workspace &ws, const double *X, int64_t ldx,
                             int n, int which) {
  if (ws.oz.xs[which] == nullptr || n > ws.oz.ldk) return cudaErrorInvalidValue;
  const int p = ws.p;
  k_oz_xslice<<<(n + OZ_BM - 1) / OZ_BM, OZ_BM, 0, s>>>(
      X, ldx, n, p, oz_nb(p), (__nv_bfloat16 *)ws.oz.xs[which], ws.oz.ldk, ws.oz.ex[which]);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_oz_product(cudaStream_t s, const Workspace &ws, int n, int which,
                              const double *X, int64_t ldx, const double *Yprev, int64_t ldp,
                              double *Ynext, int64_t ldn, int next, int mode) {
  if (ws.oz.zs == nullptr || n > ws.oz.slice_rows) return cudaErrorInvalidValue;
  const int p = ws.p;
  const int NB = oz_nb(p);
  CUtensorMap ma, mb;
  cudaError_t e = encode_tile_map(&ma, ws.oz.zs, false, (int64_t)kOzSlices * ws.oz.slice_rows, n,
                                  ws.oz.ldk, OZ_BM);
  if (e != cudaSuccess) return e;
  e = encode_tile_map(&mb, ws.oz.xs[which], false, (int64_t)kOzSlices * NB, n, ws.oz.ldk, NB);
  if (e != cudaSuccess) return e;
  const int S = oz_splits(n, ws.num_sms);
  const dim3 grid((n + OZ_BM - 1) / OZ_BM, S);
  __nv_bfloat16 *xn = next >= 0 ? (__nv_bfloat16 *)ws.oz.xs[next] : nullptr;
  int *exn = next >= 0 ? ws.oz.ex[next] : nullptr;
#define PF_OZ(NBV)                                                                              \
  k_oz_product<NBV><<<grid, OzCfg<NBV>::THREADS, OzCfg<NBV>::SMEM, s>>>(                       \
      ma, mb, n, p, (int)ws.oz.slice_rows, S, ws.oz.ez, ws.oz.ex[which], ws.oz.part, ws.oz.cnt, \
      X, ldx, Yprev, ldp, Ynext, ldn, xn, exn, ws.oz.ldk, ws.prm, mode)
  switch (NB) {
    case 16: PF_OZ(16); break;
    case 32: PF_OZ(32); break;
    case 48: PF_OZ(48); break;
    default: PF_OZ(64); break;
  }
#undef PF_OZ
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
