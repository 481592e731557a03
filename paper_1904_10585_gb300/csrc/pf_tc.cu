// Low-precision dense filter product on the 5th-generation tensor cores.
//
// One Chebyshev step (Sec. 2.1, Eq. (cheb) by the three-term recurrence in
// the mapped variable of Eq. (cheb-linear-map)) with the dense iteration
// matrix held as a low-precision shadow A_lp = A / s (bf16, or fp32 read as
// tf32), scaled into [-1, 1]:
//     Ynext = alpha (s * A_lp Xlp - c Ycur) - beta Yprev
// Xlp is the current block in the same low precision, stored transposed
// (p x n, K-major); Ycur / Yprev / Ynext are fp32 row-major n x p.  The
// epilogue also writes Ynext transposed in low precision, the B operand of
// the next product.
//
// Kernel structure (one CTA per 128-row block, 128 threads):
//   warp 0, one lane : TMA producer, 128B-swizzled A and B tiles into a ring
//                      of shared-memory stages (mbarrier complete_tx);
//   warp 1, one lane : MMA issuer, tcgen05.mma (kind::f16 or kind::tf32,
//                      M = 128, N = p, K = 32 bytes per instruction) into a
//                      TMEM accumulator; tcgen05.commit frees each stage;
//   all 4 warps      : epilogue, tcgen05.ld of the 128 x p fp32 accumulator
//                      (warp w owns TMEM lanes 32w..32w+31 = its rows).
// Every wait is bounded (about 2 s of %globaltimer); on expiry the CTA sets
// flags bit 3 in the context parameters, skips the rest and frees its TMEM.
#include <climits>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "pf_internal.cuh"
#include "pf_sm100.cuh"

namespace pf {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_STAGES = 6;
constexpr int TC_ROWB = 128;                       // bytes of K per tile row (one swizzle row)
constexpr int TC_A_BYTES = TC_BM * TC_ROWB;        // 16 KB per stage

// Instruction descriptor: fp32 accumulator, A/B K-major, M = 128, N = NB.
template <bool TF32, int NB>
__host__ __device__ constexpr uint32_t make_idesc() {
  return (1u << 4)                              // D format fp32
         | ((TF32 ? 2u : 1u) << 7)              // A format: bf16 (kind::f16) / tf32
         | ((TF32 ? 2u : 1u) << 10)             // B format
         | ((uint32_t)(NB >> 3) << 17)          // N >> 3
         | ((uint32_t)(TC_BM >> 4) << 24);      // M >> 4
}

template <int NB, bool TF32>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_filter(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                int n, int p, int num_kb, const float *Ycur, const float *Yprev,
                float *Ynext, void *Xt_next, int64_t ldxt, Params *prm, int mode) {
  constexpr int B_BYTES = NB * TC_ROWB;
  constexpr int STAGE_TX = TC_A_BYTES + B_BYTES;
  constexpr uint32_t TMEM_COLS = NB <= 32 ? 32 : (NB <= 64 ? 64 : 128);
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sA = base;
  const uint32_t sB = base + TC_STAGES * TC_A_BYTES;
  const int row0 = blockIdx.x * TC_BM;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&acc_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < num_kb; ++kb) {
      const int s = kb % TC_STAGES;
      if (kb >= TC_STAGES) {
        if (!mbar_wait(smem_u32(&empty_bar[s]), ((kb / TC_STAGES) - 1) & 1, &abort_flag)) break;
      }
      const uint32_t fb = smem_u32(&full_bar[s]);
      mbar_expect_tx(fb, STAGE_TX);
      const int kx = kb * (TC_ROWB / (TF32 ? 4 : 2));
      tma_load_2d(sA + s * TC_A_BYTES, &tmA, fb, kx, row0);
      tma_load_2d(sB + s * B_BYTES, &tmB, fb, kx, 0);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = make_idesc<TF32, NB>();
    bool ok = true;
    for (int kb = 0; kb < num_kb; ++kb) {
      const int s = kb % TC_STAGES;
      if (!mbar_wait(smem_u32(&full_bar[s]), (kb / TC_STAGES) & 1, &abort_flag)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = sw128_desc(sA + s * TC_A_BYTES);
      const uint64_t bd = sw128_desc(sB + s * B_BYTES);
#pragma unroll
      for (int k = 0; k < TC_ROWB / 32; ++k) {
        // advance 32 bytes along K inside the swizzled row: +2 in the >>4 field
        mma_issue<TF32>(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
      }
      mma_commit(smem_u32(&empty_bar[s]));
    }
    if (ok) mma_commit(smem_u32(&acc_bar));
  }
  __syncwarp();

  // epilogue: warp w owns TMEM lanes / rows 32w .. 32w+31
  const bool have_acc = mbar_wait(smem_u32(&acc_bar), 0, &abort_flag);
  __syncwarp();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (have_acc) {
    const float scale = (float)prm->lp_scale;
    double c = 0.0, alpha = 1.0;
    if (mode != MODE_PLAIN) {
      c = prm->c;
      alpha = (mode == MODE_FIRST ? 1.0 : 2.0) / prm->e;
    }
    const float cf = (float)c, af = (float)alpha;
    const int row = row0 + warp * 32 + lane;
    const bool in = row < n;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c0 = 0; c0 < NB; c0 += 16) {
      float v[16];
      tmem_ld16(taddr + c0, v);
      if (!in) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int j = c0 + i;
        if (j >= p) break;
        const int64_t idx = (int64_t)row * p + j;
        const float prod = scale * v[i];
        float y;
        if (mode == MODE_PLAIN) {
          y = prod;
        } else {
          y = af * (prod - cf * Ycur[idx]);
          if (mode == MODE_RECUR) y -= Yprev[idx];
        }
        Ynext[idx] = y;
        if (Xt_next != nullptr) {
          if (TF32)
            reinterpret_cast<float *>(Xt_next)[(int64_t)j * ldxt + row] = y;
          else
            reinterpret_cast<__nv_bfloat16 *>(Xt_next)[(int64_t)j * ldxt + row] =
                __float2bfloat16_rn(y);
        }
      }
    }
  }
  if (threadIdx.x == 0 && (abort_flag || !have_acc)) atomicOr(&prm->flags, 8);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// U (fp64, ldu) -> Y32 (fp32 n x p) and the transposed low-precision operand.
template <bool TF32>
__global__ void k_prep_lp(const double *__restrict__ U, int64_t ldu, int n, int p,
                          float *__restrict__ U32, void *__restrict__ Xt, int64_t ldxt) {
  const int64_t total = (int64_t)n * p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    // column-major walk so that the transposed write is coalesced
    const int j = (int)(idx / n);
    const int i = (int)(idx - (int64_t)j * n);
    const float v = (float)U[(int64_t)i * ldu + j];
    U32[(int64_t)i * p + j] = v;
    if (TF32) reinterpret_cast<float *>(Xt)[(int64_t)j * ldxt + i] = v;
    else reinterpret_cast<__nv_bfloat16 *>(Xt)[(int64_t)j * ldxt + i] = __float2bfloat16_rn(v);
  }
}

__global__ void k_f32_to_f64(const float *__restrict__ src, int64_t total, double *__restrict__ dst) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x)
    dst[idx] = (double)src[idx];
}

// ---------------------------------------------------------------------------
// Low-precision shadow of the max-cut iteration matrix (Eq. (PFAM1)):
//     Z_lp[i][j] = ( sum_l W[i][l] V[j][l] - t C_ij - [i == j] lam_i ) / s
// with W = V diag(max(theta, 0)) (fp32, K-padded to KP columns, zero beyond
// r+).  The write of Z_lp (n^2 elements) bounds the kernel.  The grid is
// persistent (two CTAs per SM); the 128 x 128 output tiles, numbered row
// block by row block, are split into equal contiguous ranges, one per CTA:
//   warp 0 (one lane): TMA of the W tile of the current row block (reloaded
//                      when the range crosses into the next row block, once
//                      the MMAs that read the old one have completed), and of
//                      the V tiles through a 2-stage ring;
//   warp 1 (one lane): tcgen05.mma kind::tf32 (M = N = 128, K = KP) into one
//                      of two 128-column TMEM accumulators;
//   warps 2-9        : epilogue of the previous tile, two warps per TMEM lane
//                      quarter (rows), each taking 64 of the 128 columns:
//                      sparse and diagonal parts, bf16/fp32 stores; they
//                      release the accumulator through an mbarrier.
// ---------------------------------------------------------------------------
constexpr int EX_TILE = 128;
constexpr int EX_EPI_WARPS = 8;
constexpr int EX_THREADS = 64 + 32 * EX_EPI_WARPS;
constexpr int EX_VST = 2;

template <int KP, bool F32OUT>
__global__ void __launch_bounds__(EX_THREADS, 2)
    k_tc_expand(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmV,
                int n, const int32_t *__restrict__ rowptr,
                const int32_t *__restrict__ colind, const double *__restrict__ vals,
                const double *__restrict__ lam, void *Zlp, int64_t ldz, Params *prm) {
  constexpr int KB = KP / 32;                    // 128-byte k-blocks of tf32
  constexpr int TILE_BYTES = EX_TILE * TC_ROWB;  // 16 KB per operand per k-block
  constexpr int OP_BYTES = KB * TILE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t w_full, w_empty;
  __shared__ __align__(8) uint64_t v_full[EX_VST], v_empty[EX_VST];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sW = base, sV = base + OP_BYTES;
  const int T = (n + EX_TILE - 1) / EX_TILE;
  const int64_t ntiles = (int64_t)T * T;
  const int64_t g_begin = ntiles * blockIdx.x / gridDim.x;
  const int64_t g_end = ntiles * (blockIdx.x + 1) / gridDim.x;
  const int cnt = (int)(g_end - g_begin);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&w_full), 1);
    mbar_init(smem_u32(&w_empty), 1);
    for (int s = 0; s < EX_VST; ++s) {
      mbar_init(smem_u32(&v_full[s]), 1);
      mbar_init(smem_u32(&v_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), EX_EPI_WARPS);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0 && cnt > 0) {
      int cur_rb = -1, wloads = 0;
      for (int t = 0; t < cnt; ++t) {
        const int64_t g = g_begin + t;
        const int rb = (int)(g / T), ct = (int)(g - (int64_t)rb * T);
        if (rb != cur_rb) {
          // the MMAs that read the previous W tile have completed
          if (wloads > 0 && !mbar_wait(smem_u32(&w_empty), (wloads - 1) & 1, &abort_flag)) break;
          const uint32_t wb = smem_u32(&w_full);
          mbar_expect_tx(wb, OP_BYTES);
#pragma unroll
          for (int kb = 0; kb < KB; ++kb)
            tma_load_2d(sW + kb * TILE_BYTES, &tmW, wb, kb * 32, rb * EX_TILE);
          ++wloads;
          cur_rb = rb;
        }
        const int s = t % EX_VST;
        if (t >= EX_VST && !mbar_wait(smem_u32(&v_empty[s]), ((t / EX_VST) - 1) & 1, &abort_flag))
          break;
        const uint32_t vb = smem_u32(&v_full[s]);
        mbar_expect_tx(vb, OP_BYTES);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb)
          tma_load_2d(sV + s * OP_BYTES + kb * TILE_BYTES, &tmV, vb, kb * 32, ct * EX_TILE);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && cnt > 0) {
      constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                 ((uint32_t)(EX_TILE >> 3) << 17) | ((uint32_t)(EX_TILE >> 4) << 24);
      int cur_rb = -1, wloads = 0;
      for (int t = 0; t < cnt; ++t) {
        const int64_t g = g_begin + t;
        const int rb = (int)(g / T);
        if (rb != cur_rb) {
          if (!mbar_wait(smem_u32(&w_full), wloads & 1, &abort_flag)) break;
          ++wloads;
          cur_rb = rb;
        }
        const int s = t % EX_VST, b = t & 1;
        if (!mbar_wait(smem_u32(&v_full[s]), (t / EX_VST) & 1, &abort_flag)) break;
        if (t >= 2 && !mbar_wait(smem_u32(&acc_empty[b]), ((t >> 1) - 1) & 1, &abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * EX_TILE);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
          const uint64_t ad = sw128_desc(sW + kb * TILE_BYTES);
          const uint64_t bd = sw128_desc(sV + s * OP_BYTES + kb * TILE_BYTES);
#pragma unroll
          for (int k = 0; k < TC_ROWB / 32; ++k)
            mma_issue<true>(d, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
        }
        mma_commit(smem_u32(&v_empty[s]));
        mma_commit(smem_u32(&acc_full[b]));
        const bool last_of_rb = t + 1 == cnt || (int)((g + 1) / T) != rb;
        if (last_of_rb) mma_commit(smem_u32(&w_empty));
      }
    }
  } else {
    // epilogue warps 2..9: TMEM lane quarter (warp % 4) = rows of the block,
    // column half (warp - 2) / 4 of every tile
    const int quarter = warp & 3;
    const int chalf = (warp - 2) >> 2;
    const float ts = (float)(prm->t / prm->lp_scale);
    const double inv_s = 1.0 / prm->lp_scale;
    int cur_rb = -1, row = 0;
    bool in = false;
    float ls = 0.f;
    // the row's next four sparse entries (column, t C / s), prefetched so that
    // consuming one issues the load of the entry three places later
    int e = 0, e_end = 0;
    int rc[4];
    float rv[4];
    auto fetch = [&](int idx, int &c, float &v) {
      if (idx < e_end) {
        c = colind[idx];
        v = ts * (float)vals[idx];
      } else {
        c = INT_MAX;
        v = 0.f;
      }
    };
    auto advance = [&]() {
      rc[0] = rc[1]; rv[0] = rv[1];
      rc[1] = rc[2]; rv[1] = rv[2];
      rc[2] = rc[3]; rv[2] = rv[3];
      ++e;
      fetch(e + 3, rc[3], rv[3]);
    };
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      rc[q] = INT_MAX;
      rv[q] = 0.f;
    }
    for (int tt = 0; tt < cnt; ++tt) {
      const int64_t g = g_begin + tt;
      const int rb = (int)(g / T), ct = (int)(g - (int64_t)rb * T);
      const int j0 = ct * EX_TILE + chalf * 64;  // first column of this warp's half
      if (rb != cur_rb) {
        // new row block: row state and the first sparse entry at or after j0
        cur_rb = rb;
        row = rb * EX_TILE + quarter * 32 + lane;
        in = row < n;
        ls = in ? (float)(lam[row] * inv_s) : 0.f;
        e_end = 0;
        e = 0;
        if (in) {
          int lo = rowptr[row], hi = rowptr[row + 1];
          e_end = hi;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (colind[mid] < j0) lo = mid + 1;
            else hi = mid;
          }
          e = lo;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) fetch(e + q, rc[q], rv[q]);
      }
      const int b = tt & 1;
      const bool have = mbar_wait(smem_u32(&acc_full[b]), (tt >> 1) & 1, &abort_flag);
      __syncwarp();
      if (!have) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + (uint32_t)(b * EX_TILE + chalf * 64) +
                             ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < 64; c0 += 32) {
        float v[32];
        tmem_ld32(taddr + c0, v);
        const int jc = j0 + c0;
        if (!in || jc >= n) continue;
        // sparse entries before this chunk belong to the other column half
        while (rc[0] < jc) advance();
        while (rc[0] < jc + 32) {
          const int q = rc[0] - jc;
          const float tc = rv[0];
#pragma unroll
          for (int k = 0; k < 32; ++k) v[k] -= (k == q) ? tc : 0.f;
          advance();
        }
        const int dj = row - jc;
        if (dj >= 0 && dj < 32) {
#pragma unroll
          for (int k = 0; k < 32; ++k) v[k] -= (k == dj) ? ls : 0.f;
        }
        const int64_t off = (int64_t)row * ldz + jc;
        const int valid = min(32, n - jc);
        if (F32OUT) {
          float *zp = reinterpret_cast<float *>(Zlp) + off;
          if (valid == 32 && ((off & 3) == 0)) {
            float4 *dst = reinterpret_cast<float4 *>(zp);
#pragma unroll
            for (int q = 0; q < 8; ++q)
              dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (q < valid) zp[q] = v[q];
          }
        } else {
          __nv_bfloat16 *zp = reinterpret_cast<__nv_bfloat16 *>(Zlp) + off;
          if (valid == 32 && ((off & 7) == 0)) {
            uint32_t w[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
              w[q] = *reinterpret_cast<const uint32_t *>(&h2);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(zp);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (q < valid) zp[q] = __float2bfloat16_rn(v[q]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b]))
                     : "memory");
      }
    }
  }
  __syncwarp();
  if (threadIdx.x == 0 && abort_flag) atomicOr(&prm->flags, 8);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u)
                 : "memory");
  }
}

// W = V diag(max(theta,0)) and V in fp32, K-padded to KP (zero beyond r+).
__global__ void k_expand_prep(const double *__restrict__ V, int64_t ldv,
                              const double *__restrict__ theta, int n, int p, int KP,
                              float *__restrict__ Wf, float *__restrict__ Vf,
                              const Params *__restrict__ prm) {
  const double inv_s = 1.0 / prm->lp_scale;  // the shadow's scale folded into W
  const int64_t total = (int64_t)n * KP;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / KP;
    const int l = (int)(idx - i * KP);
    float w = 0.f, v = 0.f;
    if (l < p) {
      const double th = theta[l];
      if (th > 0.0) {
        const double x = V[i * ldv + l];
        w = (float)(x * th * inv_s);
        v = (float)x;
      }
    }
    Wf[idx] = w;
    Vf[idx] = v;
  }
}

size_t expand_smem_bytes(int KP) {
  return 1024 + (size_t)(1 + EX_VST) * (KP / 32) * EX_TILE * TC_ROWB;
}

size_t tc_smem_bytes(int NB) { return 1024 + (size_t)TC_STAGES * (TC_A_BYTES + NB * TC_ROWB); }

template <int NB, bool TF32>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(k_tc_filter<NB, TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes(NB));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

// Limit of the bounded pipeline waits of this file's kernels (current device).
cudaError_t set_wait_limit_tc(uint64_t ns) { return set_wait_limit_here(ns); }

cudaError_t configure_tc() {
  if (g_encode == nullptr) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  cudaError_t e;
#define PF_TC_ATTR(NB)                          \
  if ((e = set_attr<NB, false>()) != cudaSuccess) return e; \
  if ((e = set_attr<NB, true>()) != cudaSuccess) return e;
  PF_TC_ATTR(16)
  PF_TC_ATTR(32)
  PF_TC_ATTR(48)
  PF_TC_ATTR(64)
#undef PF_TC_ATTR
#define PF_EX_ATTR(KPV, F32)                                                                 \
  if ((e = cudaFuncSetAttribute(k_tc_expand<KPV, F32>,                                       \
                                cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                                (int)expand_smem_bytes(KPV))) != cudaSuccess)                \
    return e;
  PF_EX_ATTR(32, false)
  PF_EX_ATTR(64, false)
  PF_EX_ATTR(32, true)
  PF_EX_ATTR(64, true)
#undef PF_EX_ATTR
  return cudaSuccess;
}

cudaError_t encode_tile_map(CUtensorMap *m, const void *ptr, bool f32, int64_t rows, int64_t cols,
                            int64_t ld, int box_rows) {
  if (g_encode == nullptr) return cudaErrorNotSupported;
  const int esz = f32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {(cuuint32_t)(TC_ROWB / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        2, const_cast<void *>(ptr), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int tc_nb(int p) { return p <= 16 ? 16 : p <= 32 ? 32 : p <= 48 ? 48 : 64; }

cudaError_t launch_tc_product(cudaStream_t s, const Workspace &ws, bool tf32, const void *A_lp,
                              int64_t lda_lp, int n, const void *Xt,
                              const float *Ycur, const float *Yprev, float *Ynext, void *Xt_next,
                              int mode) {
  const int p = ws.p;
  const int NB = tc_nb(p);
  CUtensorMap ma, mb;
  cudaError_t e = encode_tile_map(&ma, A_lp, tf32, n, n, lda_lp, TC_BM);
  if (e != cudaSuccess) return e;
  e = encode_tile_map(&mb, Xt, tf32, p, n, ws.ldxt, NB);
  if (e != cudaSuccess) return e;
  const int kel = TC_ROWB / (tf32 ? 4 : 2);
  const int num_kb = (n + kel - 1) / kel;
  const dim3 grid((n + TC_BM - 1) / TC_BM);
  const size_t smem = tc_smem_bytes(NB);
#define PF_TC_LAUNCH(NBV, TFV)                                                                    \
  k_tc_filter<NBV, TFV><<<grid, TC_THREADS, smem, s>>>(ma, mb, n, p, num_kb, Ycur, Yprev,       \
                                                       Ynext, Xt_next, ws.ldxt, ws.prm, mode)
  if (tf32) {
    switch (NB) {
      case 16: PF_TC_LAUNCH(16, true); break;
      case 32: PF_TC_LAUNCH(32, true); break;
      case 48: PF_TC_LAUNCH(48, true); break;
      default: PF_TC_LAUNCH(64, true); break;
    }
  } else {
    switch (NB) {
      case 16: PF_TC_LAUNCH(16, false); break;
      case 32: PF_TC_LAUNCH(32, false); break;
      case 48: PF_TC_LAUNCH(48, false); break;
      default: PF_TC_LAUNCH(64, false); break;
    }
  }
#undef PF_TC_LAUNCH
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_prep_lp(cudaStream_t s, const Workspace &ws, bool tf32, const double *U,
                           int64_t ldu, int n, float *U32, void *Xt) {
  const int64_t total = (int64_t)n * ws.p;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  if (tf32) k_prep_lp<true><<<(int)blocks, 256, 0, s>>>(U, ldu, n, ws.p, U32, Xt, ws.ldxt);
  else k_prep_lp<false><<<(int)blocks, 256, 0, s>>>(U, ldu, n, ws.p, U32, Xt, ws.ldxt);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(cudaStream_t s, const Workspace &ws, const float *src, int64_t total,
                              double *dst) {
  int64_t blocks = (total + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  if (blocks < 1) blocks = 1;
  k_f32_to_f64<<<(int)blocks, 256, 0, s>>>(src, total, dst);
  PF_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_tc_expand(cudaStream_t s, const Workspace &ws, bool f32out, const int32_t *rowptr,
                             const int32_t *colind, const double *vals, int n, const double *V,
                             int64_t ldv, const double *theta, const double *lam, void *Zlp,
                             int64_t ldz) {
  const int p = ws.p;
  const int KP = p <= 32 ? 32 : 64;
  int64_t blocks = ((int64_t)n * KP + 255) / 256;
  if (blocks > 4 * ws.num_sms) blocks = 4 * ws.num_sms;
  k_expand_prep<<<(int)blocks, 256, 0, s>>>(V, ldv, theta, n, p, KP, ws.Wf, ws.Vf, ws.prm);
  PF_LAUNCHED();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mw, mv;
  if ((e = encode_tile_map(&mw, ws.Wf, true, n, KP, KP, EX_TILE)) != cudaSuccess) return e;
  if ((e = encode_tile_map(&mv, ws.Vf, true, n, KP, KP, EX_TILE)) != cudaSuccess) return e;
  // persistent: two CTAs per SM over equal contiguous ranges of the T x T tiles
  const int T = (n + EX_TILE - 1) / EX_TILE;
  const int64_t ntiles = (int64_t)T * T;
  const int grid = (int)(ntiles < 2 * ws.num_sms ? ntiles : 2 * ws.num_sms);
  const size_t smem = expand_smem_bytes(KP);
#define PF_EX_LAUNCH(KPV, F32)                                                                  \
  k_tc_expand<KPV, F32><<<grid, EX_THREADS, smem, s>>>(mw, mv, n, rowptr, colind, vals, lam,  \
                                                       Zlp, ldz, ws.prm)
  if (KP == 32) {
    if (f32out) PF_EX_LAUNCH(32, true);
    else PF_EX_LAUNCH(32, false);
  } else {
    if (f32out) PF_EX_LAUNCH(64, true);
    else PF_EX_LAUNCH(64, false);
  }
#undef PF_EX_LAUNCH
  PF_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace pf
