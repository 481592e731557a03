// FP64-accurate dense filter product on the 5th-generation tensor cores by
// error-free slicing: the splitting idea of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012) with 8-bit digit slices (stored as bytes,
// multiplied as fp16) and fp32 accumulation.
//
// One Chebyshev step (Sec. 2.1, Eq. (cheb), by the three-term recurrence in
// the mapped variable (A - cI)/e of Eq. (cheb-linear-map)) with the dense
// FP64 iteration matrix A (n x n) and block X (n x p):
//     Ynext = alpha (A X - c X) - beta Yprev.
//
// Slices.  Row i of A gets, per 128-column chunk c, the exponent eA_ic with
// |A_ij| < 2^eA_ic on the chunk; each entry is rounded to the integer
// round(A_ij 2^(55 - eA_ic)) (|.| <= 2^55), whose balanced base-256 digits
// a_0..a_6 (a_0 in [-128, 128], the rest in [-128, 127]) give
// A_ij ~ 2^(eA_ic - 7) sum_s a_s 2^(-8s), error <= 2^(eA_ic - 56).  X is cut
// the same way per (128-row chunk c, column j) with exponent eX_cj.
// Every digit is an integer of at most 8 significant bits, exact in fp16 and
// bf16.  The exponent of A has a margin (oz_exponent_margin: |A_ij| <
// 2^eA_ic (1 - 2^-7)) that keeps a_0 inside [-128, 127], so the planes of A
// are stored as bytes a_s + 128 (7 bytes per entry, against 8 for the FP64
// matrix itself), tile by tile (oz_zs_index): every tile the product reads
// is one contiguous 8 KB block.  The planes of X are fp16.
//
// Products.  For a chunk c of 128 values of k, the level sums
//     L_l = sum_{s + t = l} sum_{k in c} a_s(i,k) x_t(k,j),   l = 0..6,
// are integers with |L_l| <= 7 * 128 * 2^14 < 2^24, so the tensor cores'
// fp32 accumulation of the (exact) bf16 products is exact.  Pairs with
// s + t >= 7 are dropped: each weighs <= 2^(eA_ic + eX_cj - 56).  The chunk's
// value 2^(eA_ic + eX_cj - 14) sum_l L_l 2^(-8l) is folded into one int64 of
// resolution 2^(eA_ic + eX_cj - 50) (levels 5 and 6 rounded), shifted to the
// largest exponents of row i and column j over the split's chunks, and summed
// over those chunks in int64 (exact).  Per output entry the error is a few
// units of 2^(max_c eA_ic + max_c eX_cj - 53) per term of the sum, the order
// of an FP64 dot product's rounding bound.
//
// Tensor-core mapping (per CTA: one 128-row block of A, one K split):
//   warp 0, one lane : producer.  Per 64-wide K tile: the 7 digit planes of
//                      X (TMA, one stage, 7 x NB rows) and, one stage each,
//                      the 7 stored byte tiles of A (bulk copies of 8 KB).
//   widening warps   : each byte tile becomes the fp16 operand tile (128 x 64
//                      fp16, K-major, 128-byte swizzle) in shared memory: a
//                      byte permute and one f16x2 subtraction per two digits.
//   warp 1, one lane : MMA issuer.  A-plane s times the stacked X planes
//                      0..6-s in one tcgen05.mma of N = (7 - s) NB,
//                      accumulating into TMEM columns [s NB, 7 NB): level l
//                      lives at columns l NB.  Two accumulator sets alternate
//                      per chunk.  NB is 16 or 32; a block wider than 32
//                      columns is split over two CTAs per row block (grid z),
//                      each reading the A planes, so that 2 x 7 x NB TMEM
//                      columns always fit.
//   warps 2..        : epilogue, NB / 2 warps, 8 columns per thread (several
//                      warps per lane quarter).  Per chunk: tcgen05.ld of the 7 levels,
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
#include <cuda_fp16.h>

#include "pf_internal.cuh"
#include "pf_sm100.cuh"

namespace pf {

namespace {

constexpr int OZ_BM = 128;               // rows per tile and K per chunk
constexpr int OZ_BK = 64;                // K per TMA tile (128 bytes of bf16)
constexpr int OZ_A_BYTES = OZ_BM * 128;  // one A digit-plane tile as the fp16 MMA operand
constexpr int OZ_S_BYTES = OZ_BM * OZ_BK;  // the same tile as stored: one byte per digit
constexpr int OZ_SB = 2;                 // stages of the X planes
constexpr int OZ_FRAC = 8 * (kOzSlices - 1) + 7;  // fractional bits of the rounded entry
constexpr int OZ_FOLD = 36;              // binary point of the int64 fold (level 0)

template <int NB>
struct OzCfg {
  static_assert(NB == 16 || NB == 32, "columns per CTA");
  // epilogue: 16 columns per thread (NB / 16 warps per TMEM lane quarter);
  // its per-chunk fold is small next to the widening of the A planes, which
  // runs on CONV warps, each widening whole tiles (tile ia on warp ia % CONV),
  // so that several tiles are in flight
  static constexpr int CW = 16;
  static constexpr int EPI = 4 * (NB / CW);      // epilogue warps
  // warps widening the A planes (6, 6 and 6 stages measured fastest at
  // n = 4096: 4 warps with 4 + 12 or 4 + 8 stages, and 2 warps, were slower)
  static constexpr int CONV = 6;
  static constexpr int THREADS = 64 + 32 * EPI + 32 * CONV;
  static constexpr int LEVEL_COLS = kOzSlices * NB;
  static constexpr int NBUF = 2;
  static constexpr uint32_t TMEM_COLS = NBUF * LEVEL_COLS <= 256 ? 256u : 512u;
  static constexpr int SA = 6;                   // A operand stages (fp16, 16 KB)
  static constexpr int SS = 6;                   // A byte-plane stages (8 KB)
  static constexpr int B_BYTES = kOzSlices * NB * 128;
  static constexpr int MAXRUN = 256 / NB;        // X planes per MMA (N <= 256)
  static constexpr size_t SMEM = 1024 + (size_t)SA * OZ_A_BYTES + (size_t)OZ_SB * B_BYTES +
                                 (size_t)SS * OZ_S_BYTES;
  // a stage belongs to one widening warp (tile ia to warp ia % CONV): the
  // warp's parity waits on it then come in phase order
  static_assert(SA % CONV == 0 && SS % CONV == 0, "stages per widening warp");
  static_assert(SMEM + 8192 <= 232448, "shared memory per CTA");
};

// Biased exponent field of |x|.
__device__ __forceinline__ unsigned oz_exfield(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}
// Exponent e with |x| < 2^e for every x whose exponent field is <= f.
__device__ __forceinline__ int oz_exponent(unsigned f) {
  return f == 0x7FFu ? kOzExpBad : (int)(f > 1u ? f : 1u) - 1022;
}

// Exponent of a chunk of A whose largest |x| has the high word `hw` (the
// sign-less top 32 bits of its binary64 pattern): |x| < 2^e (1 - 2^-7) for
// every x of the chunk, one more than oz_exponent when the largest mantissa
// is within 2^-6 of the next power of two.  The margin keeps the leading
// digit inside [-128, 127], so every digit of A fits one byte.
__device__ __forceinline__ int oz_exponent_margin(unsigned hw) {
  const int e = oz_exponent(hw >> 20);
  if (e == kOzExpBad) return e;
  return ((hw >> 14) & 0x3Fu) == 0x3Fu ? e + 1 : e;
}
__device__ __forceinline__ unsigned oz_highword(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7FFFFFFFu;
}
// The 7 balanced base-256 digits of v (|v| <= 2^55 (1 - 2^-7)) as bytes
// d_s + 128: byte 6 - s of v + 128 (1 + 256 + ... + 256^6) (no carry runs
// between digits, each digit plus 128 lies in [0, 255]).
__device__ __forceinline__ unsigned long long oz_digit_word(long long v) {
  return (unsigned long long)v + 0x0080808080808080ull;
}
// Plane s's bytes of four digit words as one 32-bit word (column i in byte i).
__device__ __forceinline__ uint32_t oz_plane_bytes4(const unsigned long long *u, int s) {
  const int k = 6 - s;  // byte of the word holding plane s
  const uint32_t a0 = (uint32_t)(u[0] >> (k < 4 ? 0 : 32)), a1 = (uint32_t)(u[1] >> (k < 4 ? 0 : 32));
  const uint32_t a2 = (uint32_t)(u[2] >> (k < 4 ? 0 : 32)), a3 = (uint32_t)(u[3] >> (k < 4 ? 0 : 32));
  const unsigned kk = (unsigned)(k & 3);
  const uint32_t lo = __byte_perm(a0, a1, kk | ((kk + 4) << 4));
  const uint32_t hi = __byte_perm(a2, a3, kk | ((kk + 4) << 4));
  return __byte_perm(lo, hi, 0x5410);
}
// fp16 pattern of a digit given as its exact fp32 pattern (oz_digit_bits).
__device__ __forceinline__ unsigned short oz_f16_of(uint32_t f) {
  return __half_as_ushort(__float2half_rn(__uint_as_float(f)));
}

// round(x 2^(OZ_FRAC - e)) for |x| < 2^e (|result| <= 2^55).  Integer
// arithmetic only.
__device__ __forceinline__ long long oz_fixed(double x, int e) {
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
  return bits < 0 ? -v : v;
}

// The 7 balanced base-256 digits of v (|v| <= 2^55), v = sum_s d[s] 256^(6-s)
// with d[1..6] in [-128, 127] and d[0] in [-128, 128], as the fp32 bit
// patterns of the digits; each is exact in bf16 (at most 8 significant bits),
// so its high half is the digit's bf16 pattern and its low half is zero.
// Adding 128 (1 + 256 + ... + 256^6) makes the digits, plus 128, the bytes
// of u (the top one, up to 256, is u >> 48): no carry runs from one digit to
// the next.  A byte permute drops byte k into the mantissa of 1.5 2^23, and
// one exact fp32 subtraction of 1.5 2^23 + 128 leaves the digit.
__device__ __forceinline__ void oz_digit_bits(long long v, uint32_t *f) {
  const unsigned long long u = (unsigned long long)v + 0x0080808080808080ull;
  const uint32_t lo = (uint32_t)u, hi = (uint32_t)(u >> 32);
  constexpr uint32_t kM = 0x4B400000u;  // 1.5 2^23
  constexpr float kB = 12583040.0f;     // 1.5 2^23 + 128
  f[6] = __float_as_uint(__uint_as_float(__byte_perm(lo, kM, 0x7650)) - kB);
  f[5] = __float_as_uint(__uint_as_float(__byte_perm(lo, kM, 0x7651)) - kB);
  f[4] = __float_as_uint(__uint_as_float(__byte_perm(lo, kM, 0x7652)) - kB);
  f[3] = __float_as_uint(__uint_as_float(__byte_perm(lo, kM, 0x7653)) - kB);
  f[2] = __float_as_uint(__uint_as_float(__byte_perm(hi, kM, 0x7650)) - kB);
  f[1] = __float_as_uint(__uint_as_float(__byte_perm(hi, kM, 0x7651)) - kB);
  f[0] = __float_as_uint(__uint_as_float(kM + (hi >> 16)) - kB);
}

__device__ __forceinline__ __nv_bfloat16 oz_bf16_of(uint32_t f) {
  return __ushort_as_bfloat16((unsigned short)(f >> 16));
}

// round(v / 2^s) for s >= 0
__device__ __forceinline__ long long oz_rshift(long long v, int s) {
  if (s <= 0) return v;
  if (s >= 62) return 0;
  return (v + (1ll << (s - 1))) >> s;
}

// (double)v 2^k: the conversion rounds to nearest even, the scaling is done
// on the exponent field when the result stays normal (ldexp otherwise).  The
// conversion is built with integer operations from the binary64 format: |v|
// normalised by its leading-zero count, its top 53 bits rounded to nearest
// even on the 11 bits below, the exponent set from the shift (a rounding
// carry into bit 53 moves into the exponent by the addition).  GB300 runs
// the int64 -> FP64 conversion instruction on its slow FP64 pipe.
__device__ __forceinline__ double oz_scale(long long v, int k) {
  if (v == 0) return 0.0;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  const unsigned long long m = a << lz;  // bit 63 set
  unsigned long long r = m >> 11;         // 53 bits
  const unsigned rem = (unsigned)(m & 0x7FF);
  r += (rem > 0x400u || (rem == 0x400u && (r & 1ull))) ? 1ull : 0ull;
  const long long bits =
      (long long)((((unsigned long long)(63 - lz + 1022)) << 52) + r) |
      (v < 0 ? (long long)0x8000000000000000ull : 0ll);
  const double d = __longlong_as_double(bits);
  const int ex = (int)((bits >> 52) & 0x7FF) + k;
  if (ex > 0 && ex < 0x7FF) return __longlong_as_double(bits + ((long long)k << 52));
  return ldexp(d, k);
}

// Instruction descriptor: fp32 accumulator, bf16 A and B (K-major), M = 128.
// The same with fp16 A and B (the product's widened byte planes and X planes).
__device__ __forceinline__ uint32_t oz_idesc_f16(int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}
// Four stored digit bytes (d + 128) -> two fp16x2 words (d exactly).
__device__ __forceinline__ void oz_widen4(uint32_t w, uint32_t &lo, uint32_t &hi) {
  constexpr uint32_t k1024 = 0x64646464u;   // bytes 0x64: exponent of 1024 in each half
  constexpr uint32_t k1152 = 0x64806480u;   // 1024 + 128 in both halves
  lo = __byte_perm(w, k1024, 0x4140);
  hi = __byte_perm(w, k1024, 0x4342);
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(lo) : "r"(lo), "r"(k1152));
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(hi) : "r"(hi), "r"(k1152));
}
__device__ __forceinline__ uint32_t oz_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(OZ_BM >> 4) << 24);
}

// Digit planes of A are stored tile by tile: plane s, 128-row block, 64-wide
// K tile, then the 128 x 64 tile row-major (128 bytes per row), so that one
// TMA box of the product is 16 KB of contiguous memory.  rb_n = row blocks
// per plane, kt_n = K tiles per row (the buffer's capacity, not n).
__host__ __device__ __forceinline__ int64_t oz_zs_index(int s, int row, int col, int rb_n,
                                                         int kt_n) {
  return ((((int64_t)s * rb_n + (row >> 7)) * kt_n + (col >> 6)) * OZ_BM + (row & 127)) * OZ_BK +
         (col & 63);
}

__device__ __forceinline__ void epi_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// 32-byte global vector access (p 32-byte aligned): a full sector per lane
__device__ __forceinline__ void ld_v4_f64(const double *p, double *v) {
  asm("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
      : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
      : "l"(p)
      : "memory");
}
__device__ __forceinline__ void st_v4_b32(void *p, uint32_t a, uint32_t b, uint32_t c,
                                          uint32_t d) {
  asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
__device__ __forceinline__ void st_v4_f64(double *p, const double *v) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
               "d"(v[2]), "d"(v[3])
               : "memory");
}

// ---------------------------------------------------------------------------
// A (n x n FP64) -> digit planes of A (one byte per digit, d + 128,
// tile-contiguous, oz_zs_index) and exponents ez[i * nzc + c] of each row
// and 128-column chunk (oz_exponent_margin).  One warp per row, four entries
// per lane and chunk.
// ---------------------------------------------------------------------------
// One 128-column chunk of one row: its exponent and its 7 digit-plane
// segments, by one warp (four entries per lane).
__device__ __forceinline__ void oz_slice_chunk(const double *__restrict__ ar, int n, int row,
                                               int c0, int lane, uint8_t *__restrict__ zs,
                                               int rb_n, int kt_n, int nzc,
                                               int *__restrict__ ez) {
  double v[4];
  unsigned hw = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = c0 + 32 * q + lane;
    v[q] = k < n ? ar[k] : 0.0;
    hw = max(hw, oz_highword(v[q]));
  }
  hw = __reduce_max_sync(0xffffffffu, hw);
  const int e = oz_exponent_margin(hw);
  if (lane == 0) ez[(int64_t)row * nzc + c0 / OZ_BM] = e;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = c0 + 32 * q + lane;
    if (k >= n) continue;
    const unsigned long long u = oz_digit_word(e != kOzExpBad ? oz_fixed(v[q], e) : 0ll);
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s)
      zs[oz_zs_index(s, row, k, rb_n, kt_n)] = (uint8_t)(u >> (8 * (6 - s)));
  }
}

__global__ void __launch_bounds__(256) k_oz_zslice(const double *__restrict__ A, int64_t lda,
                                                   int n, uint8_t *__restrict__ zs,
                                                   int rb_n, int kt_n, int nzc,
                                                   int *__restrict__ ez) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= n) return;
  const double *ar = A + (int64_t)row * lda;
  for (int c0 = 0; c0 < n; c0 += OZ_BM) oz_slice_chunk(ar, n, row, c0, lane, zs, rb_n, kt_n, nzc, ez);
}

// The same for only the chunk that holds each row's diagonal entry: the
// planes of a matrix whose other entries have not changed since it was
// sliced (the nearest-correlation iteration matrix G + Diag(x)).
__global__ void __launch_bounds__(256) k_oz_zslice_diag(const double *__restrict__ A,
                                                        int64_t lda, int n,
                                                        uint8_t *__restrict__ zs, int rb_n,
                                                        int kt_n, int nzc, int *__restrict__ ez) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= n) return;
  oz_slice_chunk(A + (int64_t)row * lda, n, row, (row / OZ_BM) * OZ_BM, lane, zs, rb_n, kt_n,
                 nzc, ez);
}

// ---------------------------------------------------------------------------
// X (n x p FP64) -> digit planes xs[t][j][k] (fp16, plane t of NB rows j,
// ldk) and exponents ex[c * kMaxP + j] of each 128-row chunk c and column j
// (columns p..NB-1 are zero).  Grid (128-row chunks, groups of 8 columns),
// thread = row: each thread reads the 8 entries of its row in the group
// (two 32-byte vectors where X allows), so that the grid covers the SMs and
// each row segment leaves HBM in whole sectors.
__global__ void __launch_bounds__(128) k_oz_xslice(const double *__restrict__ X, int64_t ldx,
                                                   int n, int p, int NB,
                                                   __half *__restrict__ xs, int64_t ldk,
                                                   int *__restrict__ ex, int xvec) {
  __shared__ unsigned qmax[4][8];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int row = blockIdx.x * OZ_BM + t, j0 = blockIdx.y * 8;
  const bool in = row < n;
  const double *xr = X + (int64_t)(in ? row : 0) * ldx + j0;
  double v[8];
  if (in && xvec && j0 + 8 <= p) {
    ld_v4_f64(xr, v);
    ld_v4_f64(xr + 4, v + 4);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = (in && j0 + j < p) ? xr[j] : 0.0;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const unsigned f = (in && j0 + j < p) ? oz_exfield(v[j]) : 0u;
    const unsigned m = __reduce_max_sync(0xffffffffu, f);
    if (lane == 0) qmax[w][j] = m;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int jj = j0 + j;
    if (jj >= NB) break;
    const int e = oz_exponent(max(max(qmax[0][j], qmax[1][j]), max(qmax[2][j], qmax[3][j])));
    if (t == 0) ex[blockIdx.x * kMaxP + jj] = e;
    uint32_t d[kOzSlices];
    oz_digit_bits((in && jj < p && e != kOzExpBad) ? oz_fixed(v[j], e) : 0ll, d);
    if (in) {
#pragma unroll
      for (int s2 = 0; s2 < kOzSlices; ++s2)
        xs[(int64_t)(s2 * NB + jj) * ldk + row] = __ushort_as_half(oz_f16_of(d[s2]));
    }
  }
}

// ---------------------------------------------------------------------------
// The sliced product with the recurrence epilogue (see the file comment).
// Grid (row blocks, K splits).
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(OzCfg<NB>::THREADS, 1) k_oz_product(
    const uint8_t *__restrict__ zs, const __grid_constant__ CUtensorMap tmB, int n,
    int p, int nbt, int rb_n, int kt_n, int nzc, int nsplit, const int *__restrict__ ez,
    const int *__restrict__ ex, double *__restrict__ part, Params *prm) {
  using C = OzCfg<NB>;
  constexpr int KS = kOzSlices;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t a_full[C::SA], a_empty[C::SA];
  __shared__ __align__(8) uint64_t s_full[C::SS], s_empty[C::SS];
  __shared__ __align__(8) uint64_t b_full[OZ_SB], b_empty[OZ_SB];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int dsh[kOzMaxChunks][NB];  // per chunk and column: shift to the split's exponent
  __shared__ int exmax[NB];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rb = blockIdx.x, split = blockIdx.y;
  const int jh = blockIdx.z * NB;  // first column of this CTA (planes hold nbt rows each)
  const int nchunks = (n + OZ_BM - 1) / OZ_BM;
  const int c0 = (int)((int64_t)split * nchunks / nsplit);
  const int c1 = (int)((int64_t)(split + 1) * nchunks / nsplit);
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sA = base;                            // fp16 operand ring
  const uint32_t sB = base + C::SA * OZ_A_BYTES;       // X planes
  const uint32_t sS = sB + OZ_SB * C::B_BYTES;         // byte planes of A as stored
  uint8_t *const gbase = smem_raw + (base - smem_u32(smem_raw));  // generic view of base

  for (int j = threadIdx.x; j < NB; j += blockDim.x) {
    int m = INT_MIN;
    for (int c = c0; c < c1; ++c) m = max(m, ex[c * kMaxP + jh + j]);
    exmax[j] = m;
  }
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < C::SA; ++s) {
      mbar_init(smem_u32(&a_full[s]), 32);  // the 32 threads of the widening warp
      mbar_init(smem_u32(&a_empty[s]), 1);
    }
    for (int s = 0; s < C::SS; ++s) {
      mbar_init(smem_u32(&s_full[s]), 1);
      mbar_init(smem_u32(&s_empty[s]), 32);
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
    dsh[c][j] = exmax[j] - ex[(c0 + c) * kMaxP + jh + j];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int is = 0, ib = 0;
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
            tma_load_2d(sB + sb * C::B_BYTES + t * NB * 128, &tmB, fb, kx, t * nbt + jh);
          ++ib;
          for (int s = 0; s < KS; ++s) {
            // the A tile of plane s as stored (8 KB of bytes, contiguous)
            const int ss = is % C::SS;
            if (is >= C::SS &&
                !mbar_wait(smem_u32(&s_empty[ss]), ((is / C::SS) - 1) & 1, &abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t fs = smem_u32(&s_full[ss]);
            mbar_expect_tx(fs, OZ_S_BYTES);
            const int64_t tile = ((int64_t)s * rb_n + rb) * kt_n + 2 * c + h;
            bulk_load(sS + ss * OZ_S_BYTES, zs + tile * OZ_S_BYTES, OZ_S_BYTES, fs);
            ++is;
          }
        }
      }
      // let every issued copy land before shared memory is released
      for (int s = 0; s < C::SS && s < is; ++s) {
        const int last = s + ((is - 1 - s) / C::SS) * C::SS;
        mbar_drain(smem_u32(&s_full[s]), (last / C::SS) & 1);
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
              const uint32_t idesc = oz_idesc_f16(ns * NB);
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
  } else if (warp >= 2 + C::EPI) {
    // ---------------- widening of the A planes ----------------
    // Each stored tile (128 rows x 64 bytes, the digits plus 128) becomes the
    // fp16 MMA operand (128 rows x 128 bytes, K-major, 128-byte swizzle: the
    // 16-byte chunk c of row r sits at chunk c ^ (r mod 8)).  Two bytes at a
    // time: a byte permute puts them into the mantissas of 1024 + b in two
    // fp16 halves, and one f16x2 subtraction of 1152 leaves b - 128 (exact).
    // Warp cw widens the tiles ia = cw, cw + CONV, ...; each lane the same
    // sixteen 16-byte pieces of every tile (piece q = lane + 32 i: row q / 4,
    // bytes 16 (q % 4) of the stored row).
    constexpr int NP = OZ_BM * 4 / 32;  // pieces per lane and tile
    const int cw = warp - 2 - C::EPI;
    const int total = (c1 - c0) * 2 * KS;
    for (int ia = cw; ia < total; ia += C::CONV) {
      const int ss = ia % C::SS, sa = ia % C::SA;
      if (!mbar_wait(smem_u32(&s_full[ss]), (ia / C::SS) & 1, &abort_flag)) break;
      if (ia >= C::SA &&
          !mbar_wait(smem_u32(&a_empty[sa]), ((ia / C::SA) - 1) & 1, &abort_flag))
        break;
      const uint8_t *src = gbase + (sS - base) + ss * OZ_S_BYTES;
      uint8_t *dst = gbase + sa * OZ_A_BYTES;
#pragma unroll 4
      for (int i = 0; i < NP; ++i) {
        const int q = lane + 32 * i, r = q >> 2, g = q & 3;
        const uint4 w = *reinterpret_cast<const uint4 *>(src + r * OZ_BK + g * 16);
        uint32_t o[8];
        oz_widen4(w.x, o[0], o[1]);
        oz_widen4(w.y, o[2], o[3]);
        oz_widen4(w.z, o[4], o[5]);
        oz_widen4(w.w, o[6], o[7]);
        uint8_t *row = dst + (r >> 3) * 1024 + (r & 7) * 128;
        *reinterpret_cast<uint4 *>(row + (((2 * g) ^ (r & 7)) << 4)) =
            make_uint4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<uint4 *>(row + (((2 * g + 1) ^ (r & 7)) << 4)) =
            make_uint4(o[4], o[5], o[6], o[7]);
      }
      fence_proxy_async_smem();
      mbar_arrive(smem_u32(&s_empty[ss]));
      mbar_arrive(smem_u32(&a_full[sa]));
    }
  } else {
    // ---------------- epilogue ----------------
    constexpr int CW = C::CW;
    const int ew = warp - 2;
    const int q = warp & 3;           // TMEM lane quarter this warp may read
    const int col0 = (ew >> 2) * CW;  // its columns (of this CTA's NB)
    const int gc0 = jh + col0;        // the same, in the block
    const int rl = q * 32 + lane;
    const int row = rb * OZ_BM + rl;
    const bool in = row < n;
    // the row's exponents over the split's chunks
    const int *ezr = ez + (int64_t)(in ? row : 0) * nzc;
    int ea = INT_MIN;
#pragma unroll 4
    for (int c = c0; c < c1; ++c) ea = max(ea, ezr[c]);
    long long acc[CW];
#pragma unroll
    for (int j = 0; j < CW; ++j) acc[j] = 0;
    int cc = 0;
    int ez_next = ezr[c0];
    for (int c = c0; c < c1; ++c, ++cc) {
      const int buf = cc % C::NBUF;
      // the row's exponent of this chunk, and the next one's load in flight
      const int da = ea - ez_next;
      if (c + 1 < c1) ez_next = ezr[c + 1];
      // one lane waits on the accumulator, the warp follows it
      int ok = 1;
      if (lane == 0) ok = mbar_wait(smem_u32(&acc_full[buf]), (cc / C::NBUF) & 1, &abort_flag);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
      if (!ok) break;
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
          acc[g + i] += oz_rshift(v, da + dsh[cc][col0 + g + i]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
    }

    // this split's values, acc 2^(max_c eA_ic + exmax_j - 14 - OZ_FOLD), to
    // the partials (summed with the recurrence by k_oz_finish)
    if (in) {
      double *pr = part + ((int64_t)split * n + row) * p;
      double y[CW];
#pragma unroll
      for (int j = 0; j < CW; ++j) {
        const int e2 = exmax[col0 + j];
        y[j] = (ea == kOzExpBad || e2 == kOzExpBad)
                   ? __longlong_as_double(0x7FF8000000000000ll)
                   : oz_scale(acc[j], ea + e2 - 14 - OZ_FOLD);
      }
      if ((p & 3) == 0 && gc0 + CW <= p) {  // 32-byte aligned: whole sectors
#pragma unroll
        for (int j = 0; j < CW; j += 4) st_v4_f64(pr + gc0 + j, y + j);
      } else {
#pragma unroll
        for (int j = 0; j < CW; ++j)
          if (gc0 + j < p) pr[gc0 + j] = y[j];
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

// ===========================================================================
// Max-cut DRS update (Eq. (PFAM1), prox of G with the minus sign) with the
// rank-r+ expansion X~ = W V^T, W = V diag(max(theta, 0)), on the tensor
// cores, producing the new Z = X~ - tC - Diag(lam) in FP64 together with its
// digit planes for the next step's products:
//   k_oz_maxcut_rows : lam of the DRS update, the report's row sums, the
//                  next interval's row bounds, and the digit planes of the
//                  rows of W and V (K = 64, zero beyond p and for
//                  theta_l <= 0) with their row exponents, sqrt(X~_ii) and
//                  per 128-row chunk the largest sqrt(X~_jj);
//   k_oz_expand  : persistent over 128 x 64 output tiles (row block by row
//                  block).  One MMA round per tile (K = 64, one exact chunk:
//                  |level sums| <= 7 * 64 * 2^14), the 7 levels in 448 TMEM
//                  columns; the epilogue folds them, scales to FP64, applies
//                  -tC and -lam on the diagonal, accumulates <C, X~>,
//                  stores Z and its digit planes (the old Z is not read: the
//                  dual residual ||Z_old - Z|| comes from the factors).
// The exponent of a (row i, 128-column chunk c) of the new Z comes from a
// bound known before the product: X~ is PSD, so |X~_ij| <= sqrt(X~_ii X~_jj),
// and |Z_ij| <= sqrt(X~_ii) max_{j in c} sqrt(X~_jj) + t max_{j in c} |C_ij|
// + [i in c] |lam_i| (times 1 + 2^-20 for rounding).  A loose bound costs
// accuracy bits of the planes, never correctness.
// ===========================================================================
// epilogue warps: 4 per TMEM lane quarter, 16 columns each (18 warps in all:
// at 96 registers a thread with a few spills they still hide more latency
// than 8 warps at 160 registers; measured 471 vs 547 us at n = 4096)
constexpr int XP_EPI = 16;
constexpr int XP_THREADS = 64 + 32 * XP_EPI;
constexpr int XP_CW = 16;                     // columns per epilogue thread
constexpr int XP_G = 8;                       // columns folded together (TMEM load width)
constexpr int XP_TN = 64;                     // output columns per tile
constexpr int XP_W_BYTES = kOzSlices * OZ_A_BYTES;         // 7 W planes of a row block
constexpr int XP_V_BYTES = kOzSlices * XP_TN * 128;        // 7 V planes of a column tile
constexpr size_t XP_SMEM = 1024 + (size_t)XP_W_BYTES + XP_V_BYTES;

// One warp per row of the sliced max-cut update (Eq. (PFAM1)), from the
// Ritz pairs (V, theta) of the step:
//   X~_ii = sum_l theta+_l V_il^2 and lam'_i = 2 X~_ii - Z_ii - t C_ii - 1
//   (lam' replaces lam; Z_ii is the current iteration matrix's diagonal);
//   the report's partial sums per block: ||diag X~ - 1||^2, sum lam', and the
//   diagonal terms of ||Z_k - Z_{k+1}||^2 (Z_k = X~_{k-1} - tC - Diag(lam),
//   so X~_{k-1,ii} = Z_ii + t C_ii + lam_i);
//   the Gershgorin bounds of the next step's sparse part -tC - Diag(lam')
//   (Sec. 4.1, reading R4; C_ii and the off-diagonal |C| row sums come
//   precomputed);
//   sqrt(X~_ii) and, per 128-row chunk, its maximum (for the expansion's
//   exponent bound; the chunk maxima are zeroed at the start of the step);
//   the digit planes of the rows of W = V diag(theta+) and V (K = 64, zero
//   beyond p and where theta_l <= 0) with their row exponents.
// Each warp accumulates its rows' sums in a fixed order; the block adds its
// eight warps in order (no atomics on sums: the result is reproducible).
__global__ void __launch_bounds__(256) k_oz_maxcut_rows(
    int n, int p, const double *__restrict__ V, int64_t ldv, const double *__restrict__ theta,
    const double *__restrict__ Z, int64_t ldz, double *__restrict__ lam,
    const double *__restrict__ cdiag, const double *__restrict__ crsum,
    const Params *__restrict__ prm, double *__restrict__ xdiag,
    unsigned long long *__restrict__ mchunk_bits, __nv_bfloat16 *__restrict__ wp,
    __nv_bfloat16 *__restrict__ vp, int64_t plane_rows, int *__restrict__ ew,
    int *__restrict__ ev, double *__restrict__ red_lam, double *__restrict__ red_ivl) {
  __shared__ double th[kMaxP];
  __shared__ double acc[8][6];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < kMaxP)
    th[threadIdx.x] = (threadIdx.x < p && theta[threadIdx.x] > 0.0) ? theta[threadIdx.x] : 0.0;
  __syncthreads();
  const double t = prm->t;
  const double t0 = th[lane], t1 = th[lane + 32];
  const bool on0 = t0 > 0.0, on1 = t1 > 0.0;  // implies column < p
  double spinf = 0.0, slam = 0.0, sdl2 = 0.0, sxl = 0.0, lo = INFINITY, hi = -INFINITY;
  const int warps = gridDim.x * 8;
  for (int row = blockIdx.x * 8 + w; row < n; row += warps) {
    const double *vr = V + (int64_t)row * ldv;
    const double v0 = lane < p ? vr[lane] : 0.0;
    const double v1 = lane + 32 < p ? vr[lane + 32] : 0.0;
    const double w0 = v0 * t0, w1 = v1 * t1;
    const double dx = warp_sum(fma(w1, v1, w0 * v0));
    unsigned fw = max(on0 ? oz_exfield(w0) : 0u, on1 ? oz_exfield(w1) : 0u);
    unsigned fv = max(on0 ? oz_exfield(v0) : 0u, on1 ? oz_exfield(v1) : 0u);
    fw = __reduce_max_sync(0xffffffffu, fw);
    fv = __reduce_max_sync(0xffffffffu, fv);
    const int e_w = oz_exponent(fw), e_v = oz_exponent(fv);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e_q = q == 0 ? e_w : e_v;
      __nv_bfloat16 *dst = (q == 0 ? wp : vp) + (int64_t)row * 64 + lane;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double x = q == 0 ? (h ? w1 : w0) : (h ? v1 : v0);
        const bool on = (h ? on1 : on0) && e_q != kOzExpBad;
        uint32_t d[kOzSlices];
        oz_digit_bits(on ? oz_fixed(x, e_q) : 0ll, d);
#pragma unroll
        for (int s2 = 0; s2 < kOzSlices; ++s2)
          dst[(int64_t)s2 * plane_rows * 64 + 32 * h] = oz_bf16_of(d[s2]);
      }
    }
    if (lane == 0) {
      ew[row] = e_w;
      ev[row] = e_v;
      const double zii = Z[(int64_t)row * ldz + row];
      const double cii = cdiag[row];
      const double l_old = lam[row];
      const double l_new = 2.0 * dx - zii - t * cii - 1.0;
      const double dl = l_old - l_new;
      const double dxx = (zii + t * cii + l_old) - dx;
      lam[row] = l_new;
      const double r = sqrt(fmax(dx, 0.0));
      xdiag[row] = r;
      atomicMax(mchunk_bits + row / OZ_BM, (unsigned long long)__double_as_longlong(r));
      spinf = fma(dx - 1.0, dx - 1.0, spinf);
      slam += l_new;
      sdl2 = fma(dl, dl, sdl2);
      sxl = fma(dxx, dl, sxl);
      const double dg = -t * cii - l_new, o = t * crsum[row];
      lo = fmin(lo, dg - o);
      hi = fmax(hi, dg + o);
    }
  }
  if (lane == 0) {
    acc[w][0] = spinf;
    acc[w][1] = slam;
    acc[w][2] = sdl2;
    acc[w][3] = sxl;
    acc[w][4] = lo;
    acc[w][5] = hi;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    double v = acc[0][k];
    for (int q = 1; q < 8; ++q) v = k == 4 ? fmin(v, acc[q][k]) : (k == 5 ? fmax(v, acc[q][k]) : v + acc[q][k]);
    if (k < 4) red_lam[blockIdx.x * kRedWidth + k] = v;
    else red_ivl[blockIdx.x * kRedWidth + (k - 4)] = v;
  }
}

__global__ void __launch_bounds__(XP_THREADS, 1) k_oz_expand(
    const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmV, int n,
    int plane_rows, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colind,
    const double *__restrict__ cvals, const double *__restrict__ lam,
    const double *__restrict__ xdiag, const double *__restrict__ mchunk,
    const int *__restrict__ ew, const int *__restrict__ ev, double *__restrict__ Z, int64_t ldz,
    int zvec, int small_k, uint8_t *__restrict__ zs, int rb_n, int kt_n,
    int *__restrict__ ez,
    int nzc, const Params *__restrict__ prm, Params *__restrict__ prm_flags,
    double *__restrict__ red) {
  constexpr int KS = kOzSlices;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t w_full, w_empty, v_full, v_empty, acc_full, acc_empty,
      mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ double rsum[XP_EPI][2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = (n + OZ_BM - 1) / OZ_BM, TCN = (n + XP_TN - 1) / XP_TN;
  const int64_t T = (int64_t)R * TCN;
  const int64_t t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sW = base, sV = base + XP_W_BYTES;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&w_full), 1);
    mbar_init(smem_u32(&w_empty), 1);
    mbar_init(smem_u32(&v_full), 1);
    mbar_init(smem_u32(&v_empty), 1);
    mbar_init(smem_u32(&acc_full), 1);
    mbar_init(smem_u32(&acc_empty), XP_EPI);
    mbar_init(smem_u32(&mma_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmW) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmV) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int cur = -1, nw = 0, nv = 0;
      bool ok = true;
      for (int64_t t = t0; t < t1 && ok; ++t) {
        const int rb = (int)(t / TCN), ct = (int)(t - (int64_t)rb * TCN);
        if (rb != cur) {
          if (nw > 0 && !mbar_wait(smem_u32(&w_empty), (nw - 1) & 1, &abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&w_full), XP_W_BYTES);
#pragma unroll
          for (int s2 = 0; s2 < KS; ++s2)
            tma_load_2d(sW + s2 * OZ_A_BYTES, &tmW, smem_u32(&w_full), 0,
                        s2 * plane_rows + rb * OZ_BM);
          ++nw;
          cur = rb;
        }
        if (nv > 0 && !mbar_wait(smem_u32(&v_empty), (nv - 1) & 1, &abort_flag)) {
          ok = false;
          break;
        }
        mbar_expect_tx(smem_u32(&v_full), XP_V_BYTES);
#pragma unroll
        for (int s2 = 0; s2 < KS; ++s2)
          tma_load_2d(sV + s2 * XP_TN * 128, &tmV, smem_u32(&v_full), 0,
                      s2 * plane_rows + ct * XP_TN);
        ++nv;
      }
      if (nw > 0) mbar_drain(smem_u32(&w_full), (nw - 1) & 1);
      if (nv > 0) mbar_drain(smem_u32(&v_full), (nv - 1) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int cur = -1, nw = 0, nt = 0;
      for (int64_t t = t0; t < t1; ++t, ++nt) {
        const int rb = (int)(t / TCN);
        if (rb != cur) {
          if (!mbar_wait(smem_u32(&w_full), nw & 1, &abort_flag)) break;
          ++nw;
          cur = rb;
        }
        if (!mbar_wait(smem_u32(&v_full), nt & 1, &abort_flag)) break;
        if (nt > 0 && !mbar_wait(smem_u32(&acc_empty), (nt - 1) & 1, &abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int s2 = 0; s2 < KS; ++s2) {
          const uint64_t ad = sw128_desc(sW + s2 * OZ_A_BYTES);
          for (int r0 = 0; r0 < KS - s2; r0 += 4) {  // N = 64 x planes <= 256
            const int ns = min(4, KS - s2 - r0);
            const uint32_t idesc = oz_idesc(ns * XP_TN);
            const uint64_t bd = sw128_desc(sV + r0 * XP_TN * 128);
            const uint32_t d = tmem + (uint32_t)((s2 + r0) * XP_TN);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              mma_issue<false>(d, ad + 2 * k, bd + 2 * k, idesc, (s2 | k) != 0 ? 1u : 0u);
          }
        }
        mma_commit(smem_u32(&v_empty));
        mma_commit(smem_u32(&acc_full));
        const bool last_of_block = t + 1 >= t1 || (int)((t + 1) / TCN) != rb;
        if (last_of_block) mma_commit(smem_u32(&w_empty));
      }
      mma_commit(smem_u32(&mma_done));
      mbar_drain(smem_u32(&mma_done), 0);
    }
  } else {
    // ---------------- epilogue ----------------
    const int ew_ = warp - 2;
    const int q = warp & 3;
    const int col0 = (ew_ >> 2) * XP_CW;  // columns of the 64-wide tile
    const double tt = prm->t;
    double dsum = 0.0, cx = 0.0;
    int nt = 0;
    for (int64_t t = t0; t < t1; ++t, ++nt) {
      const int rb = (int)(t / TCN), ct = (int)(t - (int64_t)rb * TCN);
      const int row = rb * OZ_BM + q * 32 + lane;
      const bool in = row < n;
      const int j0 = ct * XP_TN + col0;      // first column of this thread
      const int c = (ct * XP_TN) / OZ_BM;    // 128-column chunk
      // exponent of (row, chunk) from the bound; the CSR cursor at column j0
      int ez_rc = 0, ewr = 0;
      int e_lo = 0, e_hi = 0;
      double lam_r = 0.0;
      if (in) {
        ewr = ew[row];
        lam_r = lam[row];
        const int cb = c * OZ_BM, ce = min(n, cb + OZ_BM);
        int lo = rowptr[row], hi = rowptr[row + 1];
        e_hi = hi;
        while (lo < hi) {  // first entry with column >= cb
          const int mid = (lo + hi) >> 1;
          if (colind[mid] < cb) lo = mid + 1;
          else hi = mid;
        }
        double cmax = 0.0;
        e_lo = e_hi;
        for (int e = lo; e < e_hi; ++e) {
          const int col = colind[e];
          if (col >= ce) break;
          cmax = fmax(cmax, fabs(cvals[e]));
          if (col >= j0 && e_lo == e_hi) e_lo = e;
        }
        // the factor 1 + 2^-6 covers rounding and keeps |Z_ij| < 2^e (1 - 2^-7),
        // so that the leading digit fits its byte (oz_exponent_margin)
        const double bound =
            (xdiag[row] * mchunk[c] + tt * cmax +
             ((row >= cb && row < ce) ? fabs(lam_r) : 0.0)) *
            (1.0 + 0x1p-6);
        ez_rc = oz_exponent(oz_exfield(bound));
        if (col0 == 0 && (ct * XP_TN) % OZ_BM == 0) ez[(int64_t)row * nzc + c] = ez_rc;
      }
      int ok = 1;
      if (lane == 0) ok = mbar_wait(smem_u32(&acc_full), nt & 1, &abort_flag);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col0;
      int e = e_lo;
      int ncol = e < e_hi ? colind[e] : INT_MAX;  // column of the next entry of C
      static_assert(XP_G == 8 && XP_CW == 2 * XP_G, "two 8-column groups per thread");
      static_assert(OZ_FOLD == 36 && KS == 7, "the fold below is written out for 7 levels");
      // the first group's plane bytes, stored with the second group's: 16
      // bytes of each plane row per store (columns j0 .. j0 + 15)
      uint32_t pk0[KS][XP_G / 4];
#pragma unroll
      for (int g = 0; g < XP_CW; g += XP_G) {
        // the group's new Z values, stored together: whole groups of an
        // aligned Z leave as two 32-byte vectors (a full sector per access:
        // each lane of the warp holds another row).  The old Z is not read:
        // the dual residual comes from the factors (k_maxcut_kkt)
        double zo[XP_G];
        double *zrow = Z + (int64_t)(in ? row : 0) * ldz;
        const bool vec = zvec && j0 + g + XP_G <= n;  // the same for the whole warp
        // v = sum_l L_l 2^(36 - 8l), levels 5 and 6 rounded together, folded
        // in pairs of levels as they leave TMEM.  With K <= 64,
        // |L_l| <= (l + 1) 2^20, so L_0 2^8 + L_1, L_2 2^8 + L_3 and
        // L_5 2^8 + L_6 stay inside int32
        int hi[XP_G], mid[XP_G], lo[XP_G];
        {
          uint32_t A[XP_G], B[XP_G], C[XP_G];
          // exact integers in fp32; with p <= 32, |L_l| <= 7 32 2^14 < 2^22, and
          // adding 1.5 2^23 leaves L_l in the low mantissa bits (an FMA-pipe
          // add instead of a conversion)
          auto f2i = [small_k](uint32_t u) {
            return small_k ? __float_as_int(__uint_as_float(u) + 12582912.0f) - 0x4B400000
                           : __float2int_rn(__uint_as_float(u));
          };
          tmem_ld8(taddr + 0 * XP_TN + g, A);
          tmem_ld8(taddr + 1 * XP_TN + g, B);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < XP_G; ++i) hi[i] = f2i(A[i]) * 256 + f2i(B[i]);
          tmem_ld8(taddr + 2 * XP_TN + g, A);
          tmem_ld8(taddr + 3 * XP_TN + g, B);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < XP_G; ++i) mid[i] = f2i(A[i]) * 256 + f2i(B[i]);
          tmem_ld8(taddr + 4 * XP_TN + g, A);
          tmem_ld8(taddr + 5 * XP_TN + g, B);
          tmem_ld8(taddr + 6 * XP_TN + g, C);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < XP_G; ++i)
            lo[i] = f2i(A[i]) * 16 + ((f2i(B[i]) * 256 + f2i(C[i]) + 2048) >> 12);
        }
        uint32_t pk[KS][XP_G / 4];
        unsigned long long uw[XP_G];  // digit words (oz_digit_word) of the group
#pragma unroll
        for (int i = 0; i < XP_G; ++i) {
          const int col = j0 + g + i;
          const long long v = (long long)lo[i] + (long long)mid[i] * 4096 +
                              (long long)hi[i] * 268435456;
          long long zf = 0;  // round(Z_ij 2^(OZ_FRAC - e)) for the planes
          if (in && col < n) {
            const int evc = ev[col];
            double xt = (ewr == kOzExpBad || evc == kOzExpBad)
                            ? __longlong_as_double(0x7FF8000000000000ll)
                            : oz_scale(v, ewr + evc - 14 - OZ_FOLD);
            double z = xt;
            if (ncol == col) {
              const double cij = cvals[e];
              z = fma(-tt, cij, z);
              cx = fma(cij, xt, cx);
              ++e;
              ncol = e < e_hi ? colind[e] : INT_MAX;
            }
            if (col == row) z -= lam_r;
            zo[i] = z;  // the new value, stored with the group
            if (!vec) zrow[col] = z;
            if (ez_rc != kOzExpBad) zf = oz_fixed(z, ez_rc);
          }
          uw[i] = oz_digit_word(zf);
        }
#pragma unroll
        for (int s2 = 0; s2 < KS; ++s2) {
          pk[s2][0] = oz_plane_bytes4(uw, s2);
          pk[s2][1] = oz_plane_bytes4(uw + 4, s2);
        }
        if (vec && in) {
          st_v4_f64(zrow + j0 + g, zo);
          st_v4_f64(zrow + j0 + g + 4, zo + 4);
        }
        if (g == 0) {
#pragma unroll
          for (int s2 = 0; s2 < KS; ++s2)
#pragma unroll
            for (int w2 = 0; w2 < XP_G / 4; ++w2) pk0[s2][w2] = pk[s2][w2];
        } else if (in) {
          // columns j0 .. j0 + 15 of each plane row: 16 bytes at a 16-byte
          // boundary (j0 is a multiple of 16, plane rows are 64 bytes)
#pragma unroll
          for (int s2 = 0; s2 < KS; ++s2)
            st_v4_b32(zs + oz_zs_index(s2, row, j0, rb_n, kt_n), pk0[s2][0], pk0[s2][1],
                      pk[s2][0], pk[s2][1]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty));
    }
    // per-CTA sums in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      cx += __shfl_xor_sync(0xffffffffu, cx, o);
    }
    if (lane == 0) {
      rsum[ew_][0] = dsum;
      rsum[ew_][1] = cx;
    }
    epi_sync(32 * XP_EPI);
    if (ew_ == 0 && lane == 0) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < XP_EPI; ++k) {
        a += rsum[k][0];
        b += rsum[k][1];
      }
      red[blockIdx.x * kRedWidth + 0] = a;
      red[blockIdx.x * kRedWidth + 1] = b;
    }
  }

  if (threadIdx.x == 0 && abort_flag) atomicOr(&prm_flags->flags, 8);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// The sum of the K splits in split order, the recurrence, and the digit
// planes of the new block for the next product.  Grid (128-row blocks,
// 8-column groups), thread = row: the FP64 work of the combine spreads over
// many SMs instead of one CTA per row block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_BM) k_oz_finish(
    const double *__restrict__ part, int nsplit, int n, int p, const double *X, int64_t ldx,
    const double *Yprev, int64_t ldp, double *Ynext, int64_t ldn,
    __half *__restrict__ xs_next, int *__restrict__ ex_next, int64_t ldk, int nbt,
    const Params *__restrict__ prm, int mode, int vmask) {
  __shared__ unsigned qmax[4][8];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int rb = blockIdx.x, j0 = blockIdx.y * 8;
  const int row = rb * OZ_BM + t;
  const bool in = row < n;
  double cval = 0.0, alpha = 1.0;
  if (mode != MODE_PLAIN) {
    cval = prm->c;
    alpha = (mode == MODE_FIRST ? 1.0 : 2.0) / prm->e;
  }
  double y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) y[j] = 0.0;
  // a whole group of 8 columns moves as two 32-byte vectors per row where
  // the array allows it (vmask bits: partials, X, Y_prev, Y_next)
  const bool full = j0 + 8 <= p;
  if (in) {
    for (int sp = 0; sp < nsplit; ++sp) {
      const double *pr = part + ((int64_t)sp * n + row) * p + j0;
      if (full && (vmask & 1)) {
        double a[8];
        ld_v4_f64(pr, a);
        ld_v4_f64(pr + 4, a + 4);
#pragma unroll
        for (int j = 0; j < 8; ++j) y[j] += a[j];
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j0 + j < p) y[j] += __ldcg(pr + j);
      }
    }
    if (mode != MODE_PLAIN) {
      double xv[8], yp[8];
      const double *xr = X + (int64_t)row * ldx + j0;
      const double *pr = Yprev + (int64_t)row * ldp + j0;
      if (full && (vmask & 2)) {
        ld_v4_f64(xr, xv);
        ld_v4_f64(xr + 4, xv + 4);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) xv[j] = j0 + j < p ? xr[j] : 0.0;
      }
      if (mode == MODE_RECUR) {
        if (full && (vmask & 4)) {
          ld_v4_f64(pr, yp);
          ld_v4_f64(pr + 4, yp + 4);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) yp[j] = j0 + j < p ? pr[j] : 0.0;
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        double v = alpha * (y[j] - cval * xv[j]);
        if (mode == MODE_RECUR) v -= yp[j];
        y[j] = v;
      }
    }
    double *yn = Ynext + (int64_t)row * ldn + j0;
    if (full && (vmask & 8)) {
      st_v4_f64(yn, y);
      st_v4_f64(yn + 4, y + 4);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j0 + j < p) yn[j] = y[j];
    }
  }
  if (xs_next == nullptr) return;  // uniform over the grid
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const unsigned f = (in && j0 + j < p) ? oz_exfield(y[j]) : 0u;
    const unsigned mx = __reduce_max_sync(0xffffffffu, f);
    if (lane == 0) qmax[w][j] = mx;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int jj = j0 + j;
    const int e = oz_exponent(max(max(qmax[0][j], qmax[1][j]), max(qmax[2][j], qmax[3][j])));
    if (t == 0 && jj < nbt) ex_next[rb * kMaxP + jj] = e;
    uint32_t d[kOzSlices];
    oz_digit_bits((in && jj < p && e != kOzExpBad) ? oz_fixed(y[j], e) : 0ll, d);
    if (in && jj < nbt) {
#pragma unroll
      for (int s2 = 0; s2 < kOzSlices; ++s2)
        xs_next[(int64_t)(s2 * nbt + jj) * ldk + row] = __ushort_as_half(oz_f16_of(d[s2]));
    }
  }
}

template <int NB>
cudaError_t oz_set_attr() {
  return cudaFuncSetAttribute(k_oz_product<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)OzCfg<NB>::SMEM);
}

// columns per CTA, column halves (grid z) and rows per digit plane of X
int oz_nb(int p) { return p <= 16 ? 16 : 32; }
int oz_halves(int p) { return p <= 32 ? 1 : 2; }
int oz_nbt(int p) { return oz_halves(p) == 1 ? oz_nb(p) : 64; }

}  // namespace

// Limit of the bounded pipeline waits of this file's kernels (current device).
cudaError_t set_wait_limit_oz(uint64_t ns) { return set_wait_limit_here(ns); }

cudaError_t configure_oz() {
  cudaError_t e;
  if ((e = oz_set_attr<16>()) != cudaSuccess) return e;
  if ((e = oz_set_attr<32>()) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_oz_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)XP_SMEM);
}

int oz_splits(int n, int p, int num_sms) {
  const int R = (n + OZ_BM - 1) / OZ_BM;
  int S = num_sms / (R * oz_halves(p));
  if (S > kOzMaxSplits) S = kOzMaxSplits;
  if (S > R) S = R;
  const int need = (R + kOzMaxChunks - 1) / kOzMaxChunks;  // int64 headroom of the fold
  if (S < need) S = need;
  return S < 1 ? 1 : S;
}

cudaError_t launch_oz_zslice(cudaStream_t s, const Workspace &ws, const double *A, int64_t lda,
                             int n) {
  if (ws.oz.zs == nullptr || n > ws.oz.slice_rows) return cudaErrorInvalidValue;
  k_oz_zslice<<<(n + 7) / 8, 256, 0, s>>>(A, lda, n, (uint8_t *)ws.oz.zs,
                                          (int)(ws.oz.slice_rows / OZ_BM),
                                          (int)(ws.oz.ldk / OZ_BK),
                                          (int)(ws.oz.slice_rows / OZ_BM), ws.oz.ez);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_oz_zslice_diag(cudaStream_t s, const Workspace &ws, const double *A,
                                  int64_t lda, int n) {
  if (ws.oz.zs == nullptr || n > ws.oz.slice_rows) return cudaErrorInvalidValue;
  k_oz_zslice_diag<<<(n + 7) / 8, 256, 0, s>>>(A, lda, n, (uint8_t *)ws.oz.zs,
                                               (int)(ws.oz.slice_rows / OZ_BM),
                                               (int)(ws.oz.ldk / OZ_BK),
                                               (int)(ws.oz.slice_rows / OZ_BM), ws.oz.ez);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_oz_xslice(cudaStream_t s, const Workspace &ws, const double *X, int64_t ldx,
                             int n, int which) {
  if (ws.oz.xs[which] == nullptr || n > ws.oz.ldk) return cudaErrorInvalidValue;
  const int p = ws.p;
  const int nb = oz_nbt(p);
  const int xvec = ((reinterpret_cast<uintptr_t>(X) & 31) == 0 && (ldx & 3) == 0) ? 1 : 0;
  k_oz_xslice<<<dim3((n + OZ_BM - 1) / OZ_BM, (nb + 7) / 8), OZ_BM, 0, s>>>(
      X, ldx, n, p, nb, (__half *)ws.oz.xs[which], ws.oz.ldk, ws.oz.ex[which], xvec);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_oz_product(cudaStream_t s, const Workspace &ws, int n, int which,
                              const double *X, int64_t ldx, const double *Yprev, int64_t ldp,
                              double *Ynext, int64_t ldn, int next, int mode) {
  if (ws.oz.zs == nullptr || n > ws.oz.slice_rows) return cudaErrorInvalidValue;
  const int p = ws.p;
  const int NB = oz_nb(p), H = oz_halves(p), nbt = oz_nbt(p);
  CUtensorMap mb;
  // the X planes (fp16 digits, 2-byte elements like bf16 for the copy)
  cudaError_t e = encode_tile_map(&mb, ws.oz.xs[which], false, (int64_t)kOzSlices * nbt, n,
                                  ws.oz.ldk, NB);
  if (e != cudaSuccess) return e;
  const int S = oz_splits(n, p, ws.num_sms);
  const int R = (n + OZ_BM - 1) / OZ_BM;
  const dim3 grid(R, S, H);
#define PF_OZ(NBV)                                                                              \
  k_oz_product<NBV><<<grid, OzCfg<NBV>::THREADS, OzCfg<NBV>::SMEM, s>>>(                       \
      (const uint8_t *)ws.oz.zs, mb, n, p, nbt, (int)(ws.oz.slice_rows / OZ_BM),               \
      (int)(ws.oz.ldk / OZ_BK),                                                                   \
      (int)(ws.oz.slice_rows / OZ_BM), S, ws.oz.ez, ws.oz.ex[which], ws.oz.part, ws.prm)
  if (NB == 16) PF_OZ(16);
  else PF_OZ(32);
#undef PF_OZ
  PF_LAUNCHED();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  __half *xn = next >= 0 ? (__half *)ws.oz.xs[next] : nullptr;
  int *exn = next >= 0 ? ws.oz.ex[next] : nullptr;
  auto vec_ok = [](const double *a, int64_t ld) {
    return a != nullptr && (reinterpret_cast<uintptr_t>(a) & 31) == 0 && (ld & 3) == 0;
  };
  const int vmask = ((p & 3) == 0 ? 1 : 0) | (vec_ok(X, ldx) ? 2 : 0) |
                    (vec_ok(Yprev, ldp) ? 4 : 0) | (vec_ok(Ynext, ldn) ? 8 : 0);
  k_oz_finish<<<dim3(R, (nbt + 7) / 8), OZ_BM, 0, s>>>(ws.oz.part, S, n, p, X, ldx, Yprev, ldp,
                                                      Ynext, ldn, xn, exn, ws.oz.ldk, nbt,
                                                      ws.prm, mode, vmask);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_oz_expand(cudaStream_t s, const Workspace &ws, const int32_t *rowptr,
                             const int32_t *colind, const double *vals, int n, int p,
                             const double *V, int64_t ldv, const double *theta, const double *lam,
                             double *Z, int64_t ldz, double *red, int *nblocks) {
  const OzBuffers &oz = ws.oz;
  if (oz.zs == nullptr || oz.wp == nullptr || n > oz.slice_rows) return cudaErrorInvalidValue;
  const int R = (n + OZ_BM - 1) / OZ_BM;
  cudaError_t e;
  CUtensorMap mw, mv;
  if ((e = encode_tile_map(&mw, oz.wp, false, (int64_t)kOzSlices * oz.slice_rows, 64, 64,
                           OZ_BM)) != cudaSuccess)
    return e;
  if ((e = encode_tile_map(&mv, oz.vp, false, (int64_t)kOzSlices * oz.slice_rows, 64, 64,
                           XP_TN)) != cudaSuccess)
    return e;
  const int64_t T = (int64_t)R * ((n + XP_TN - 1) / XP_TN);
  const int grid = (int)(T < ws.num_sms ? T : ws.num_sms);
  // 32-byte vector access to Z: 32-byte aligned rows
  const int zvec = ((reinterpret_cast<uintptr_t>(Z) & 31) == 0 && (ldz & 3) == 0) ? 1 : 0;
  k_oz_expand<<<grid, XP_THREADS, XP_SMEM, s>>>(
      mw, mv, n, (int)oz.slice_rows, rowptr, colind, vals, lam, oz.xdiag, oz.mchunk, oz.ew,
      oz.ev, Z, ldz, zvec, p <= 32 ? 1 : 0, (uint8_t *)oz.zs,
      (int)(oz.slice_rows / OZ_BM),
      (int)(oz.ldk / OZ_BK), oz.ez, (int)(oz.slice_rows / OZ_BM), ws.prm, ws.prm, red);
  PF_LAUNCHED();
  *nblocks = grid;
  return cudaGetLastError();
}

cudaError_t launch_oz_maxcut_rows(cudaStream_t s, const Workspace &ws, int n, int p,
                                  const double *V, int64_t ldv, const double *theta,
                                  const double *Z, int64_t ldz, double *lam, int nb,
                                  double *red_lam, double *red_ivl) {
  const OzBuffers &oz = ws.oz;
  if (oz.wp == nullptr || n > oz.slice_rows) return cudaErrorInvalidValue;
  k_oz_maxcut_rows<<<nb, 256, 0, s>>>(n, p, V, ldv, theta, Z, ldz, lam, oz.cdiag, oz.crsum,
                                      ws.prm, oz.xdiag, (unsigned long long *)oz.mchunk,
                                      (__nv_bfloat16 *)oz.wp, (__nv_bfloat16 *)oz.vp,
                                      oz.slice_rows, oz.ew, oz.ev, red_lam, red_ivl);
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
