// contrastive.cu -- InfoNCE-style contrastive join: forward and backward on
// sm_103a tensor cores.
//
// S = A B^T / T over N paired rows (positives on the diagonal), BF16 operands
// (round-to-nearest-even of the float32 inputs), FP32 accumulation in TMEM.
//   forward : l_i = logsumexp_j S_ij, loss = (1/N) sum_i (l_i - S_ii)
//             (symmetric flag: also the column term, averaged)
//   backward: G_ij = dloss/dS_ij = (g/N) (P_ij - [i == j]) (+ column term),
//             dA = G B / T,  dB = G^T A / T.
//
// One persistent kernel template, one CTA per SM, warp-specialised:
//   warp 0: TMA producer, warp 1: TMEM allocator + MMA issuer,
//   warps 2-9: epilogue (two per TMEM lane quarter, one row per thread, each
//   owning half of a tile's columns).
//   FWD : 128 x 256 score tiles double-buffered in TMEM; units = (128-row
//         block, column split); the epilogue keeps an online (max, sum) per
//         row and column half, written as partial states that a second
//         launch merges into l_i and the loss terms.
//   GP  : the G pass of the materialised backward: the same tiles turned into
//         G' = w_r (P - I) + w_c (Q - I) in BF16 and written to memory
//         (through a shared-memory staging tile and TMA stores); two GEMM
//         launches (contrastive_gemm_kernel) then form dA = G' B and
//         dB = G'^T A (G' read as an MN-major operand), scaled by g / (N T).
//   BWD : the fused backward for when G' does not fit in memory: unit =
//         (128-row block of X, chunk of <= 384 output dimensions); per
//         128-column tile t, S_t = X_blk Y_t^T (TMEM cols 0..127), G'_t in
//         shared memory, and the MMA warp adds G'_t Z_t^T to the chunk
//         accumulator (TMEM cols 128..511), Z^T being a transposed BF16 copy
//         of the other side.  The same kernel gives dA (X = A, Y = B, Z^T =
//         B^T) and dB (X = B, Y = A, Z^T = A^T, the softmax terms swapped
//         between rows and columns).  A 128 x 768 FP32 block would exceed
//         tensor memory (512 columns), hence the chunks.
// Every wait is bounded (globaltimer); a wait that gives up flags
// SJ_ERR_TIMEOUT and the CTA drains its copies and MMAs before freeing TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "../../include/sj.h"
#include "contrastive.h"
#include "tc_common.cuh"

namespace sj {
namespace {

using namespace tc;

constexpr int TM = 128;             // rows per tile (TMEM lanes)
constexpr int BK = 64;              // k-block (128 bytes of BF16)
constexpr int kMaxChunk = 384;      // output dimensions per fused-backward unit
constexpr int kPiece = 192;         // N of one backward MMA
constexpr int kZBox = 64;           // rows of one Z^T TMA box
constexpr uint32_t kOpBytes = TM * BK * 2;  // one 128-row operand k-block (16 KB)
constexpr uint32_t kGBytes = TM * 128 * 2;  // one 128 x 128 G' tile (32 KB)
constexpr float kLog2e = 1.4426950408889634f;

// Kernel modes: the forward; the fused backward (G' recomputed per output
// chunk and consumed in shared memory); the G' pass of the materialised
// backward (G' written to global memory).
constexpr int kModeFwd = kContrastiveFwd, kModeBwd = kContrastiveBwdFused,
              kModeGp = kContrastiveGprime;

// Per-mode shapes.  Score tiles are 128 x TN.  The operand stream bounds
// these kernels (one k-block of a 128 x 256 tile is ~540 tensor-core cycles,
// one L2 round trip several times that), so the forward and the G' pass use
// 256-column tiles (a third fewer operand bytes per flop than 128) with S
// double-buffered in TMEM (2 x 256 columns).  The fused backward keeps
// 128-column tiles: its chunk accumulator takes the other 384 TMEM columns.
// Ring slots hold one k-block of the X row block and of the Y tile, or (fused
// backward) a Z^T slice of up to 192 rows, in the order the MMA warp consumes
// them: S(0), then for t >= 1 S(t) and Z^T(t-1), then Z^T(last).
// Epilogue: 8 warps, two per TMEM lane quarter, each owning half of a tile's
// columns (NC chunks of 32).
template <int MODE>
struct CCfg {
  static constexpr int TN = MODE == kModeBwd ? 128 : 256;
  static constexpr uint32_t kSlot = kOpBytes + TN * BK * 2;
  static constexpr int kStages = MODE == kModeBwd ? 6 : 4;
  static constexpr int NC = TN / 64;
};
constexpr int kEpiWarps = 8;
constexpr int kCThreads = 64 + 32 * kEpiWarps;

template <int MODE>
struct alignas(1024) CSmem {
  using C = CCfg<MODE>;
  unsigned char slot[C::kStages][C::kSlot];
  // fused backward: the G' operand tile; G' pass: staging of one 128 x 128
  // half of a G' tile for the TMA stores
  unsigned char g[MODE == kModeFwd ? 1024 : kGBytes];
  uint64_t full[C::kStages], empty[C::kStages];
  uint64_t s_full[2], s_empty[2];
  uint64_t g_full, g_empty;
  uint64_t st_full[2], st_free[2];  // G' pass: staging written / free, per column half
  uint64_t acc_full, acc_empty;
  uint64_t drain, never;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename SM>
__device__ __forceinline__ void flag_timeout(SM &sm, unsigned *err) {
  *(volatile int *)&sm.abort = 1;
  atomicOr(err, 4u);  // kErrTimeout
}

// fence the generic-proxy shared-memory writes before the async proxy
// (tensor core, TMA store) reads them
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int MODE>
__global__ void __launch_bounds__(kCThreads, 1)
    contrastive_kernel(const __grid_constant__ CUtensorMap tmX,
                       const __grid_constant__ CUtensorMap tmY,
                       const __grid_constant__ CUtensorMap tmZ, ContrastiveArgs a) {
  constexpr bool BWD = MODE == kModeBwd;
  constexpr bool GP = MODE == kModeGp;
  using C = CCfg<MODE>;
  constexpr int TN = C::TN, NC = C::NC, kStages = C::kStages;
  constexpr int kEpi = kEpiWarps * 32;
  extern __shared__ unsigned char smem_raw[];
  using Smem = CSmem<MODE>;
  Smem &sm = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                       ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t limit_ns = 4000000000ull;
  volatile int *abort = &sm.abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&sm.s_full[q], 1);
      mbar_init(&sm.s_empty[q], kEpi);
      mbar_init(&sm.st_full[q], kEpi / 2);
      mbar_init(&sm.st_free[q], 1);
    }
    mbar_init(&sm.g_full, kEpi);
    mbar_init(&sm.g_empty, 1);
    mbar_init(&sm.acc_full, 1);
    mbar_init(&sm.acc_empty, kEpi);
    mbar_init(&sm.drain, 1);
    mbar_init(&sm.never, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&sm.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  const int nkb = (int)(a.dp / BK);
  const int n_tiles = (int)(a.npy / TN);  // column tiles (rows of Y)
  const int n_rb = (int)(a.np / TM);      // row blocks (rows of X)
  const int n_chunks = BWD ? a.n_chunks : 1;
  // the forward and the G' pass also split a row block's column tiles
  const int n_splits = BWD ? 1 : a.n_splits;
  const int tps = BWD ? n_tiles : a.tiles_per_split;
  const int64_t n_units = (int64_t)n_rb * n_chunks * n_splits;
  const uint32_t idesc_s = idesc_bf16(TM, TN);
  // unit u: row block, output chunk, split, column tiles [t0, t1)
  auto unit_of = [&](int64_t u, int &rb, int &ch, int &sp, int &t0, int &t1) {
    const int64_t per_rb = (int64_t)n_chunks * n_splits;
    rb = (int)(u / per_rb);
    const int rem = (int)(u % per_rb);
    ch = rem / n_splits;
    sp = rem % n_splits;
    t0 = sp * tps;
    t1 = min(n_tiles, t0 + tps);
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint64_t it = 0;
      bool ok = true;
      auto take = [&](uint32_t bytes) -> int {  // next slot, armed for `bytes`
        const int s = (int)(it % kStages);
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        if (!mbar_wait(&sm.empty[s], ph ^ 1, limit_ns, abort)) {
          flag_timeout(sm, &a.ctr->err_flags);
          ok = false;
          return -1;
        }
        ++it;
        mbar_arrive_expect_tx(&sm.full[s], bytes);
        return s;
      };
      for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        int rb, ch, sp, t0, t1;
        unit_of(u, rb, ch, sp, t0, t1);
        const int c0 = ch * kMaxChunk;
        const int cw = (int)min64(kMaxChunk, a.dp - c0);
        auto push_s = [&](int t) {
          for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = take(C::kSlot);
            if (s < 0) break;
            tma_load_2d(sm.slot[s], &tmX, kb * BK, rb * TM, &sm.full[s]);
            for (int y = 0; y < TN; y += 128)
              tma_load_2d(sm.slot[s] + kOpBytes + y * BK * 2, &tmY, kb * BK, t * TN + y,
                          &sm.full[s]);
          }
        };
        // Z^T(t): per 64-wide k-block kz of the tile's columns, slices of up
        // to kPiece output dimensions (rows of Z^T), kZBox rows per TMA box
        auto push_z = [&](int t) {
          for (int kz = 0; kz < 2 && ok; ++kz)
            for (int p = 0; p < cw && ok; p += kPiece) {
              const int pw = min(kPiece, cw - p);
              const int s = take((uint32_t)pw * BK * 2);
              if (s < 0) break;
              for (int b = 0; b < pw; b += kZBox)
                tma_load_2d(sm.slot[s] + b * BK * 2, &tmZ, t * TN + kz * BK, c0 + p + b,
                            &sm.full[s]);
            }
        };
        for (int t = t0; t < t1 && ok; ++t) {
          push_s(t);
          if (BWD && t > t0) push_z(t - 1);
        }
        if (BWD && ok && t1 > t0) push_z(t1 - 1);
      }
      // drain: the last copy into each slot must have landed
      for (uint64_t q = (it > kStages ? it - kStages : 0); q < it; ++q) {
        const uint64_t t0 = now_ns();
        while (!mbar_try(&sm.full[q % kStages], (uint32_t)((q / kStages) & 1)) &&
               now_ns() - t0 < limit_ns) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint64_t it = 0, tile = 0, unit_n = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++unit_n) {
        int rb, ch, sp, t0, t1;
        unit_of(u, rb, ch, sp, t0, t1);
        const int cw = (int)min64(kMaxChunk, a.dp - ch * kMaxChunk);
        // S tiles use TMEM buffer (tile & 1), at column buf * TN; the fused
        // backward has one buffer (its accumulator takes the rest)
        auto issue_s = [&](uint64_t tl) -> bool {
          const int buf = BWD ? 0 : (int)(tl & 1);
          const uint32_t ph = BWD ? (uint32_t)(tl & 1) : (uint32_t)((tl >> 1) & 1);
          if (!mbar_wait(&sm.s_empty[buf], ph ^ 1, limit_ns, abort)) return false;
          fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * TN);
          for (int kb = 0; kb < nkb; ++kb, ++it) {
            const int s = (int)(it % kStages);
            const uint32_t spar = (uint32_t)((it / kStages) & 1);
            if (!mbar_wait(&sm.full[s], spar, limit_ns, abort)) return false;
            fence_after();
            const uint32_t x0 = su32(sm.slot[s]), y0 = x0 + kOpBytes;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_bf16(d, sdesc(x0 + kk * 32), sdesc(y0 + kk * 32), idesc_s,
                       (kb > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&sm.empty[s]);
          }
          mma_commit(&sm.s_full[buf]);
          return true;
        };
        // fused backward, tile tl: acc += G'_tl Z_tl^T
        auto issue_g = [&](uint64_t tl, bool first) -> bool {
          const uint32_t gph = (uint32_t)(tl & 1);
          if (!mbar_wait(&sm.g_full, gph, limit_ns, abort)) return false;
          if (first && unit_n > 0) {
            if (!mbar_wait(&sm.acc_empty, (uint32_t)((unit_n - 1) & 1), limit_ns, abort))
              return false;
          }
          fence_after();
          for (int kz = 0; kz < 2; ++kz) {
            const uint32_t g0 = su32(sm.g) + kz * (TM * BK * 2);
            for (int p = 0; p < cw; p += kPiece, ++it) {
              const int pw = min(kPiece, cw - p);
              const int s = (int)(it % kStages);
              const uint32_t spar = (uint32_t)((it / kStages) & 1);
              if (!mbar_wait(&sm.full[s], spar, limit_ns, abort)) return false;
              fence_after();
              const uint32_t z0 = su32(sm.slot[s]);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem + TN + (uint32_t)p, sdesc(g0 + kk * 32), sdesc(z0 + kk * 32),
                         idesc_bf16(TM, pw), (first && kz == 0 && kk == 0) ? 0u : 1u);
              mma_commit(&sm.empty[s]);
            }
          }
          mma_commit(&sm.g_empty);
          return true;
        };
        for (int t = t0; t < t1 && ok; ++t, ++tile) {
          if (!issue_s(tile)) {
            ok = false;
            break;
          }
          if (BWD && t > t0 && !issue_g(tile - 1, t == t0 + 1)) {
            ok = false;
            break;
          }
        }
        if (BWD && ok && t1 > t0) {
          if (!issue_g(tile - 1, t1 - t0 == 1)) ok = false;
          else mma_commit(&sm.acc_full);
        }
        if (!ok) flag_timeout(sm, &a.ctr->err_flags);
      }
      mma_commit(&sm.drain);
      const uint64_t t0 = now_ns();
      while (!mbar_try(&sm.drain, 0) && now_ns() - t0 < limit_ns) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;      // row within the tile
    const int half = (warp - 2) >> 2;       // column half of the tile
    const int cb = half * NC;               // first 32-column chunk of this warp
    uint64_t tile = 0, unit_n = 0;
    bool ok = true;
    if (a.debug_timeout) {
      const bool w = mbar_wait(&sm.never, 0, 1000000ull, abort);
      if (!__all_sync(0xffffffffu, w)) {
        flag_timeout(sm, &a.ctr->err_flags);
        ok = false;
      }
    }
    const float c1 = kLog2e / a.T;
    for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++unit_n) {
      int rb, ch, sp, t0, t1;
      unit_of(u, rb, ch, sp, t0, t1);
      const int64_t row = (int64_t)rb * TM + r;
      const bool valid = row < a.n;
      // forward state of this row over this warp's columns of the unit's
      // tiles (log2 domain); the running sum is compensated (TwoSum), so its
      // error does not grow with N
      float m = -INFINITY, l = 0.f, lc = 0.f;
      // backward: this row's own-term log-sum-exp (log2 domain)
      const float lr2 = (MODE != kModeFwd && valid && a.wr != 0.f) ? a.lse_r[row] * kLog2e : 0.f;
      for (int t = t0; t < t1; ++t, ++tile) {
        const int buf = BWD ? 0 : (int)(tile & 1);
        const uint32_t ph = BWD ? (uint32_t)(tile & 1) : (uint32_t)((tile >> 1) & 1);
        const bool w = mbar_wait(&sm.s_full[buf], ph, limit_ns, abort);
        if (!__all_sync(0xffffffffu, w)) {
          flag_timeout(sm, &a.ctr->err_flags);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * TN);
        float v[NC][32];
#pragma unroll
        for (int c = 0; c < NC; ++c) tmem_ld32_nowait(taddr + (cb + c) * 32, v[c]);
        if constexpr (NC == 2) tmem_wait_ld(v[0], v[1]);
        else tmem_wait_ld4(v);
        fence_before();
        mbar_arrive(&sm.s_empty[buf]);  // S buffer free for the next tile
        const int64_t col0 = (int64_t)t * TN;
        if constexpr (MODE == kModeFwd) {
          const bool cols_full = col0 + TN <= a.ny;
          const int64_t pos = row + a.diag_off;  // the row's positive column
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            // in place: scores -> log2-domain logits -> exponentials -> sum
            const int64_t jb = col0 + (cb + c) * 32;
            if (valid && pos >= jb && pos < jb + 32) {
#pragma unroll
              for (int q = 0; q < 32; ++q)
                if (jb + q == pos) a.diag_out[row] = v[c][q];
            }
            float cm = -INFINITY;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              float x = v[c][q] * c1;
              if (!cols_full && jb + q >= a.ny) x = -INFINITY;
              v[c][q] = x;
              cm = fmaxf(cm, x);
            }
            if (cm > m) {
              const float sc = (m == -INFINITY) ? 0.f : ex2(m - cm);
              l *= sc;
              lc *= sc;
              m = cm;
            }
            if (m == -INFINITY) continue;  // no valid column seen yet (padding)
            // pairwise sum of the chunk, then a compensated add into l
#pragma unroll
            for (int q = 0; q < 32; ++q) v[c][q] = ex2(v[c][q] - m);
#pragma unroll
            for (int w2 = 16; w2 >= 1; w2 >>= 1)
#pragma unroll
              for (int q = 0; q < w2; ++q) v[c][q] += v[c][q + w2];
            {
              const float e0 = v[c][0];
              const float tt = __fadd_rn(l, e0);
              const float bp = __fsub_rn(tt, l);
              lc = __fadd_rn(lc, __fadd_rn(__fsub_rn(l, __fsub_rn(tt, bp)), __fsub_rn(e0, bp)));
              l = tt;
            }
          }
        } else {
          // G'_t = w_r (P - I) + w_c (Q - I), computed in place: one ex2 per
          // term and element; the column log-sum-exp (log2 domain) comes one
          // value per lane and is broadcast by shuffles; the diagonal and the
          // ragged last tile are fixed up apart from the element loop
          const float wr = a.wr, wc = a.wc;
          const bool cols_full = col0 + TN <= a.ny;
          const int64_t dr = row + a.diag_off - col0;  // the positive's column in the tile
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            float lcq = INFINITY;
            if (wc != 0.f) {
              const int64_t jj = col0 + (cb + c) * 32 + lane;
              if (jj < a.ny) lcq = __ldg(a.lse_c + jj) * kLog2e;
            }
            const int dq = (int)(dr - (cb + c) * 32);  // 0..31 when the diagonal is in this chunk
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              const float x = v[c][q] * c1;
              float gv = 0.f;
              if (wr != 0.f) gv = wr * ex2(x - lr2);
              if (wc != 0.f) gv = fmaf(wc, ex2(x - __shfl_sync(0xffffffffu, lcq, q)), gv);
              if (q == dq) gv -= wr + wc;
              v[c][q] = gv;
            }
          }
          if (!valid || !cols_full) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
              for (int q = 0; q < 32; ++q)
                if (!valid || col0 + (cb + c) * 32 + q >= a.ny) v[c][q] = 0.f;
          }
          // G' into the shared tile (128B-swizzled K-major k-blocks of 64
          // columns): the fused backward's MMA operand, or the G' pass's
          // staging of this warp's column half (the two halves take turns)
          const uint32_t gph = (uint32_t)(tile & 1);
          bool we;
          if constexpr (GP) {
            // half 0 of tile t waits for half 1 of tile t - 1, half 1 for half 0 of tile t
            const uint32_t par = half == 0 ? gph ^ 1u : gph;
            we = mbar_wait(&sm.st_free[half], par, limit_ns, abort);
          } else {
            we = mbar_wait(&sm.g_empty, gph ^ 1, limit_ns, abort);
          }
          if (!__all_sync(0xffffffffu, we)) {
            flag_timeout(sm, &a.ctr->err_flags);
            ok = false;
            break;
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const float *gq = v[c];
            const int cc = GP ? c : cb + c;  // chunk within the shared 128-column tile
            // 32 columns = 4 chunks of 16 bytes in k-block (cc >> 1)
            unsigned char *kbase = sm.g + (cc >> 1) * (TM * BK * 2) + r * 128;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int l16 = (cc & 1) * 4 + h;  // logical 16-byte chunk in the 128-byte row
              __nv_bfloat162 p0 = __floats2bfloat162_rn(gq[h * 8 + 0], gq[h * 8 + 1]);
              __nv_bfloat162 p1 = __floats2bfloat162_rn(gq[h * 8 + 2], gq[h * 8 + 3]);
              __nv_bfloat162 p2 = __floats2bfloat162_rn(gq[h * 8 + 4], gq[h * 8 + 5]);
              __nv_bfloat162 p3 = __floats2bfloat162_rn(gq[h * 8 + 6], gq[h * 8 + 7]);
              uint4 pk;
              pk.x = *reinterpret_cast<uint32_t *>(&p0);
              pk.y = *reinterpret_cast<uint32_t *>(&p1);
              pk.z = *reinterpret_cast<uint32_t *>(&p2);
              pk.w = *reinterpret_cast<uint32_t *>(&p3);
              *reinterpret_cast<uint4 *>(kbase + ((l16 ^ (r & 7)) * 16)) = pk;
            }
          }
          fence_proxy_async_smem();
          if constexpr (GP) {
            mbar_arrive(&sm.st_full[half]);
            if (((warp - 2) & 3) == 0 && lane == 0) {
              // the half's first warp stores its two 64-column boxes once the
              // half's four warps have written them
              if (!mbar_wait(&sm.st_full[half], gph, limit_ns, abort)) {
                flag_timeout(sm, &a.ctr->err_flags);
              } else {
                const int y0 = rb * TM, x0 = (int)col0 + half * 128;
                const uint64_t pol = l2_policy_evict_first();
                tma_store_2d_hint(&tmZ, sm.g, x0, y0, pol);
                tma_store_2d_hint(&tmZ, sm.g + TM * BK * 2, x0 + BK, y0, pol);
                bulk_commit();
                bulk_wait_read_all();
                mbar_arrive(&sm.st_free[half ^ 1]);
              }
            }
          } else {
            mbar_arrive(&sm.g_full);
          }
        }
      }
      if (!ok) break;
      if constexpr (MODE == kModeFwd) {
        if (valid) {
          // partial state of (row, split, half): merged by the finishing kernel
          const int64_t pi = (int64_t)(sp * 2 + half) * a.np + row;
          a.part_m[pi] = m;
          a.part_l[pi] = l;
          a.part_c[pi] = lc;
        }
      } else if constexpr (BWD) {
        // chunk accumulator -> dX[row, chunk] * (g / (N T))
        const bool w = mbar_wait(&sm.acc_full, (uint32_t)(unit_n & 1), limit_ns, abort);
        if (!__all_sync(0xffffffffu, w)) {
          flag_timeout(sm, &a.ctr->err_flags);
          ok = false;
          break;
        }
        fence_after();
        const float scale = __ldg(a.grad_loss) / ((float)a.n_norm * a.T);
        const int c0 = ch * kMaxChunk;
        const int cw = (int)min64(kMaxChunk, a.dp - c0);
        // each epilogue warp of a lane quarter stores its half of the chunk
        const int hw = cw / 2;
        for (int c = half * hw; c < (half + 1) * hw; c += 32) {
          float o[32];
          tmem_ld32_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(TN + c), o);
          tmem_wait_ld1(o);
          if (valid) {
            float *dst = a.dX + row * a.d + c0 + c;
            const int64_t lim = a.d - (c0 + c);
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (q < lim) dst[q] = o[q] * scale;
          }
        }
        fence_before();
        mbar_arrive(&sm.acc_empty);
      }
    }
    // G' pass: the last stores must complete before the CTA's shared memory goes
    if (GP && ((warp - 2) & 3) == 0 && lane == 0) bulk_wait_all();
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Forward finish: lse_i from the partial (max, sum) of every (split, half)
// of row i (sums in double), and the loss term lse_i - S_ii / T.
__global__ void contrastive_merge_kernel(ContrastiveArgs a, int n_parts) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= a.n) return;
  float M = -INFINITY;
  for (int p = 0; p < n_parts; ++p) M = fmaxf(M, a.part_m[(int64_t)p * a.np + row]);
  double s = 0.0;
  for (int p = 0; p < n_parts; ++p) {
    const int64_t pi = (int64_t)p * a.np + row;
    const float mp = a.part_m[pi];
    if (mp == -INFINITY) continue;  // no valid column in this part
    s += ((double)a.part_l[pi] + (double)a.part_c[pi]) * (double)exp2f(mp - M);
  }
  const float lse = (M + (float)log2(s)) * 0.69314718055994531f;  // natural log
  a.lse_out[row] = lse;
  a.term_out[row] = lse - a.diag_out[row] / a.T;
}

// ---------------------------------------------------------------------------
// Materialised backward, second half: dX = (g / (N T)) P Z with P = G or
// P = G^T, for G (np x np, BF16, row-major) and Z (np x d) given as Z^T
// (dp x np, BF16).  Unit = (128-row block of P, chunk of <= 384 output
// dimensions), accumulated over K = np in 64-wide k-blocks; a ring slot holds
// one k-block of P (16 KB) and of the chunk's Z^T rows (<= 48 KB).  P = G is
// read K-major (box of 64 columns x 128 rows); P = G^T is read from G itself
// as an MN-major operand: two boxes of 64 columns (the output rows) x 64 rows
// (the k-block), 8 KB apart.  Warp 0: TMA, warp 1: MMA, warps 2-5: readout
// (one TMEM lane quarter each).
constexpr int kGemmStages = 3;
constexpr uint32_t kGemmSlot = kOpBytes + kMaxChunk * BK * 2;  // 64 KB
constexpr int kGemmThreads = 64 + 4 * 32;

struct alignas(1024) GSmem {
  unsigned char slot[kGemmStages][kGemmSlot];
  uint64_t full[kGemmStages], empty[kGemmStages];
  uint64_t acc_full, acc_empty, drain;
  uint32_t tmem_base;
  int abort;
};

template <bool TRANS>
__global__ void __launch_bounds__(kGemmThreads, 1)
    contrastive_gemm_kernel(const __grid_constant__ CUtensorMap tmG,
                            const __grid_constant__ CUtensorMap tmZ, ContrastiveGemmArgs a) {
  extern __shared__ unsigned char smem_raw[];
  GSmem &sm = *reinterpret_cast<GSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                         ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t limit_ns = 4000000000ull;
  volatile int *abort = &sm.abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGemmStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    mbar_init(&sm.acc_full, 1);
    mbar_init(&sm.acc_empty, 4 * 32);
    mbar_init(&sm.drain, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&sm.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  const int nkb = (int)(a.kp / BK);
  const int64_t n_units = (a.np / TM) * a.n_chunks;

  if (warp == 0) {
    if (lane == 0) {
      uint64_t it = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
        const int rb = (int)(u / a.n_chunks), ch = (int)(u % a.n_chunks);
        const int c0 = ch * kMaxChunk;
        const int cw = (int)min64(kMaxChunk, a.dp - c0);
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = (int)(it % kGemmStages);
          const uint32_t ph = (uint32_t)((it / kGemmStages) & 1);
          if (!mbar_wait(&sm.empty[s], ph ^ 1, limit_ns, abort)) {
            flag_timeout(sm, &a.ctr->err_flags);
            ok = false;
            break;
          }
          ++it;
          mbar_arrive_expect_tx(&sm.full[s], kOpBytes + (uint32_t)cw * BK * 2);
          if (TRANS) {
            tma_load_2d(sm.slot[s], &tmG, rb * TM, kb * BK, &sm.full[s]);
            tma_load_2d(sm.slot[s] + kOpBytes / 2, &tmG, rb * TM + 64, kb * BK, &sm.full[s]);
          } else {
            tma_load_2d(sm.slot[s], &tmG, kb * BK, rb * TM, &sm.full[s]);
          }
          for (int b = 0; b < cw; b += kZBox)
            tma_load_2d(sm.slot[s] + kOpBytes + b * BK * 2, &tmZ, kb * BK, c0 + b, &sm.full[s]);
        }
      }
      for (uint64_t q = (it > kGemmStages ? it - kGemmStages : 0); q < it; ++q) {
        const uint64_t t0 = now_ns();
        while (!mbar_try(&sm.full[q % kGemmStages], (uint32_t)((q / kGemmStages) & 1)) &&
               now_ns() - t0 < limit_ns) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint64_t it = 0, unit_n = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++unit_n) {
        const int ch = (int)(u % a.n_chunks);
        const int cw = (int)min64(kMaxChunk, a.dp - ch * kMaxChunk);
        if (unit_n > 0 &&
            !mbar_wait(&sm.acc_empty, (uint32_t)((unit_n - 1) & 1), limit_ns, abort)) {
          ok = false;
          break;
        }
        fence_after();
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % kGemmStages);
          if (!mbar_wait(&sm.full[s], (uint32_t)((it / kGemmStages) & 1), limit_ns, abort)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t g0 = su32(sm.slot[s]), z0 = g0 + kOpBytes;
          for (int p = 0; p < cw; p += kPiece) {
            const int pw = min(kPiece, cw - p);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              // K = 16 per MMA: 32 bytes along a K-major row, or 16 rows of
              // 128 bytes (two 8-row atoms) of the MN-major tile
              const uint64_t ad = TRANS ? sdesc_mn(g0 + kk * 2048, kOpBytes / 2, 1024)
                                        : sdesc(g0 + kk * 32);
              mma_bf16(tmem + (uint32_t)p, ad, sdesc(z0 + (uint32_t)p * BK * 2 + kk * 32),
                       TRANS ? idesc_bf16_amn(TM, pw) : idesc_bf16(TM, pw),
                       (kb > 0 || kk > 0) ? 1u : 0u);
            }
          }
          mma_commit(&sm.empty[s]);
        }
        if (ok) mma_commit(&sm.acc_full);
      }
      if (!ok) flag_timeout(sm, &a.ctr->err_flags);
      mma_commit(&sm.drain);
      const uint64_t t0 = now_ns();
      while (!mbar_try(&sm.drain, 0) && now_ns() - t0 < limit_ns) {
      }
    }
  } else {
    const int quarter = warp & 3;
    const float scale = __ldg(a.grad_loss) / ((float)a.n_norm * a.T);
    uint64_t unit_n = 0;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x, ++unit_n) {
      const int rb = (int)(u / a.n_chunks), ch = (int)(u % a.n_chunks);
      const int c0 = ch * kMaxChunk;
      const int cw = (int)min64(kMaxChunk, a.dp - c0);
      const bool w = mbar_wait(&sm.acc_full, (uint32_t)(unit_n & 1), limit_ns, abort);
      if (!__all_sync(0xffffffffu, w)) {
        flag_timeout(sm, &a.ctr->err_flags);
        break;
      }
      fence_after();
      const int64_t row = (int64_t)rb * TM + quarter * 32 + lane;
      for (int c = 0; c < cw; c += 32) {
        float o[32];
        tmem_ld32_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, o);
        tmem_wait_ld1(o);
        if (row < a.n) {
          float *dst = a.dX + row * a.d + c0 + c;
          const int64_t lim = a.d - (c0 + c);
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (q < lim) dst[q] = o[q] * scale;
        }
      }
      fence_before();
      mbar_arrive(&sm.acc_empty);
    }
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Round float32 rows to BF16 (RNE) into a zero-padded row-major copy
// (np x dp) and a transposed copy (dp x np); flags non-finite input.
__global__ void contrastive_pack_kernel(const float *__restrict__ X, int64_t n, int64_t d,
                                        __nv_bfloat16 *__restrict__ Xp,
                                        __nv_bfloat16 *__restrict__ XT, int64_t np, int64_t dp,
                                        unsigned *err) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t r = r0 + yy, k = k0 + tx;
    float x = (r < n && k < d) ? X[r * d + k] : 0.f;
    if (!isfinite(x)) {
      atomicOr(err, 1u);  // kErrNonFinite
      x = 0.f;
    }
    const __nv_bfloat16 q = __float2bfloat16_rn(x);
    Xp[r * dp + k] = q;
    tile[yy][tx] = q;
  }
  __syncthreads();
  if (XT) {
    for (int yy = ty; yy < 32; yy += 8) XT[(k0 + yy) * np + r0 + tx] = tile[tx][yy];
  }
}

// loss = (w1 sum term1 + w2 sum term2) / N, compensated summation, one block.
__global__ void contrastive_loss_kernel(const float *t1, const float *t2, int64_t n,
                                        int64_t n_norm, float w1, float w2, float *loss) {
  __shared__ float sh_s[32];
  float s = 0.f, c = 0.f;  // Kahan-compensated per-thread partial sum
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    float v = w1 * t1[i] + (t2 ? w2 * t2[i] : 0.f);
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  s -= c;
  for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh_s[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh_s[w];
    *loss = tot / (float)n_norm;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side

size_t contrastive_smem_bytes(int mode) {
  const size_t b = mode == kModeFwd ? sizeof(CSmem<kModeFwd>)
                   : mode == kModeBwd ? sizeof(CSmem<kModeBwd>)
                                      : sizeof(CSmem<kModeGp>);
  return b + 1024;
}

void contrastive_splits(int64_t np, int *n_splits, int *tiles_per_split) {
  const int64_t n_tiles = np / CCfg<kModeFwd>::TN;
  const int64_t want = std::max<int64_t>(1, (n_tiles + 31) / 32);
  const int64_t tps = (n_tiles + want - 1) / want;
  *tiles_per_split = (int)tps;
  *n_splits = (int)((n_tiles + tps - 1) / tps);
}

cudaError_t launch_contrastive_pack(const float *X, int64_t n, int64_t d, void *Xp, void *XT,
                                    int64_t np, int64_t dp, unsigned *err, cudaStream_t st) {
  dim3 grid((unsigned)(dp / 32), (unsigned)(np / 32)), block(32, 8);
  contrastive_pack_kernel<<<grid, block, 0, st>>>(X, n, d, static_cast<__nv_bfloat16 *>(Xp),
                                                  static_cast<__nv_bfloat16 *>(XT), np, dp, err);
  return cudaGetLastError();
}

cudaError_t launch_contrastive_loss(const float *t1, const float *t2, int64_t n, int64_t n_norm,
                                    float w1, float w2, float *loss, cudaStream_t st) {
  contrastive_loss_kernel<<<1, 1024, 0, st>>>(t1, t2, n, n_norm, w1, w2, loss);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const CUtensorMap &mx, const CUtensorMap &my, const CUtensorMap &mz,
                               const ContrastiveArgs &a, int grid, cudaStream_t st) {
  const size_t smem = contrastive_smem_bytes(MODE);
  cudaError_t e = cudaFuncSetAttribute(contrastive_kernel<MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  contrastive_kernel<MODE><<<grid, kCThreads, smem, st>>>(mx, my, mz, a);
  return cudaGetLastError();
}

cudaError_t launch_contrastive(int mode, const void *tmX, const void *tmY, const void *tmZ,
                               const ContrastiveArgs &a, int grid, cudaStream_t st) {
  CUtensorMap mx, my, mz;
  std::memcpy(&mx, tmX, sizeof mx);
  std::memcpy(&my, tmY, sizeof my);
  std::memcpy(&mz, tmZ ? tmZ : tmX, sizeof mz);
  cudaError_t e;
  switch (mode) {
    case kModeFwd:
      e = launch_mode<kModeFwd>(mx, my, mz, a, grid, st);
      if (e != cudaSuccess) return e;
      contrastive_merge_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, st>>>(a, 2 * a.n_splits);
      return cudaGetLastError();
    case kModeBwd: return launch_mode<kModeBwd>(mx, my, mz, a, grid, st);
    case kModeGp: return launch_mode<kModeGp>(mx, my, mz, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t contrastive_gemm_smem_bytes() { return sizeof(GSmem) + 1024; }

cudaError_t launch_contrastive_gemm(bool trans, const void *tmG, const void *tmZ,
                                    const ContrastiveGemmArgs &a, int grid, cudaStream_t st) {
  CUtensorMap mg, mz;
  std::memcpy(&mg, tmG, sizeof mg);
  std::memcpy(&mz, tmZ, sizeof mz);
  const size_t smem = contrastive_gemm_smem_bytes();
  auto kern = trans ? contrastive_gemm_kernel<true> : contrastive_gemm_kernel<false>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kGemmThreads, smem, st>>>(mg, mz, a);
  return cudaGetLastError();
}

}  // namespace sj
