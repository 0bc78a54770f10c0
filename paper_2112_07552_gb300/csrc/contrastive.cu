// contrastive.cu -- InfoNCE-style contrastive join: forward and backward on
// sm_103a tensor cores, recomputing score tiles instead of storing S.
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
//   warps 2-5: epilogue (one TMEM lane quarter each, one row per thread).
// Tiles are 128 rows x 128 columns.
//   FWD  : S tiles double-buffered in TMEM; epilogue keeps an online
//          (max, sum) per row with exp2 and records the diagonal.
//   BWD  : unit = (128-row block of X, chunk of <= 384 output dimensions).
//          Per column tile t: S_t = X_blk Y_t^T (TMEM cols 0..127); the
//          epilogue turns S_t into G'_t = w_r (P - I) + w_c (Q - I) in BF16,
//          written 128B-swizzled into shared memory; the MMA warp then adds
//          G'_t Z_t^T to the chunk accumulator (TMEM cols 128..511), Z^T being
//          a transposed BF16 copy of the other side.  The same kernel gives dA
//          (X = A, Y = B, Z^T = B^T) and dB (X = B, Y = A, Z^T = A^T, the
//          softmax terms swapped between rows and columns).  A 128 x 768 FP32
//          block would exceed tensor memory (512 columns), hence the chunks.
// Every wait is bounded (globaltimer); a wait that gives up flags
// SJ_ERR_TIMEOUT and the CTA drains its copies and MMAs before freeing TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "../../include/sj.h"
#include "contrastive.h"
#include "tc_common.cuh"

namespace sj {
namespace {

using namespace tc;

constexpr int TM = 128;             // rows per tile (TMEM lanes)
constexpr int TN = 128;             // columns per tile
constexpr int BK = 64;              // k-block (128 bytes of BF16)
// Operand ring of 32 KB slots: the bytes in flight bound the operand stream
// (one 64-wide k-block of a 128 x 128 tile is ~270 tensor-core cycles, one L2
// round trip several times that).  A slot holds an S k-block (X and Y, 16 KB
// each) or, in the backward, a Z^T slice (up to 192 rows of a 64-wide
// k-block, 24 KB), in the order the MMA warp consumes them: S(0), then for
// t >= 1 S(t) and Z^T(t-1), then Z^T(last).  Six slots and one G' tile; the
// G' pass has five slots and two staging tiles (G' and its transpose).
constexpr int kMaxChunk = 384;      // output dimensions per backward unit
constexpr int kPiece = 192;         // N of one backward MMA
constexpr int kZBox = 64;           // rows of one Z^T TMA box
// Kernel modes: the forward; the fused backward (G' recomputed per output
// chunk and consumed in shared memory); the G' pass of the materialised
// backward (G' and its transpose written to global memory).
constexpr int kModeFwd = kContrastiveFwd, kModeBwd = kContrastiveBwdFused,
              kModeGp = kContrastiveGprime;
// Producer and MMA warps, then the epilogue: 4 warps (one TMEM lane quarter
// each, all 128 columns of a tile) in the forward, 8 in the other modes (two
// per lane quarter, one 64-column half each: one k-block of the G' tile).
__host__ __device__ constexpr int epi_warps(int mode) { return mode == kModeFwd ? 4 : 8; }
__host__ __device__ constexpr int cthreads(int mode) { return 64 + 32 * epi_warps(mode); }
constexpr uint32_t kOpBytes = TM * BK * 2;  // one operand k-block (16 KB)
constexpr uint32_t kGBytes = TM * TN * 2;         // one G tile (32 KB)
constexpr float kLog2e = 1.4426950408889634f;

template <int MODE>
struct alignas(1024) CSmem {
  static constexpr int kSStages = MODE == kModeGp ? 5 : 6;
  static constexpr int kGTiles = MODE == kModeGp ? 2 : 1;
  unsigned char slot[kSStages][2 * kOpBytes];
  unsigned char g[kGTiles][MODE == kModeFwd ? 1024 : kGBytes];  // G' tile(s)
  uint64_t full[kSStages], empty[kSStages];
  uint64_t st_full, st_free;  // G' pass: staging tiles written / read by the stores
  uint64_t s_full[2], s_empty[2];
  uint64_t g_full[2], g_empty[2];
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

// fence the generic-proxy shared-memory writes before the tensor core reads them
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int MODE>
__global__ void __launch_bounds__(cthreads(MODE), 1)
    contrastive_kernel(const __grid_constant__ CUtensorMap tmX,
                       const __grid_constant__ CUtensorMap tmY,
                       const __grid_constant__ CUtensorMap tmZ,
                       const __grid_constant__ CUtensorMap tmW, ContrastiveArgs a) {
  constexpr bool BWD = MODE == kModeBwd;
  constexpr bool GP = MODE == kModeGp;
  constexpr int kEpi = epi_warps(MODE) * 32;
  extern __shared__ unsigned char smem_raw[];
  using Smem = CSmem<MODE>;
  constexpr int kSStages = Smem::kSStages;
  Smem &sm = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                       ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t limit_ns = 4000000000ull;
  volatile int *abort = &sm.abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&sm.s_full[q], 1);
      mbar_init(&sm.s_empty[q], kEpi);
      mbar_init(&sm.g_full[q], kEpi);
      mbar_init(&sm.g_empty[q], 1);
    }
    mbar_init(&sm.acc_full, 1);
    mbar_init(&sm.acc_empty, kEpi);
    mbar_init(&sm.st_full, kEpi);
    mbar_init(&sm.st_free, 1);
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
  const int n_tiles = (int)(a.np / TN);
  const int n_rb = (int)(a.np / TM);
  const int n_chunks = BWD ? a.n_chunks : 1;
  // G' pass: units also split the column tiles (no state crosses tiles there)
  const int n_splits = GP ? a.n_splits : 1;
  const int tps = GP ? a.tiles_per_split : n_tiles;
  const int64_t n_units = (int64_t)n_rb * n_chunks * n_splits;
  // unit u: row block, output chunk, column tiles [t0, t1)
  auto unit_of = [&](int64_t u, int &rb, int &ch, int &t0, int &t1) {
    const int64_t per_rb = (int64_t)n_chunks * n_splits;
    rb = (int)(u / per_rb);
    const int rem = (int)(u % per_rb);
    ch = rem / n_splits;
    t0 = (rem % n_splits) * tps;
    t1 = min(n_tiles, t0 + tps);
  };
  const uint32_t idesc_s = idesc_bf16(TM, TN);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint64_t it = 0;
      bool ok = true;
      auto take = [&](uint32_t bytes) -> int {  // next slot, armed for `bytes`
        const int s = (int)(it % kSStages);
        const uint32_t ph = (uint32_t)((it / kSStages) & 1);
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
        int rb, ch, t0, t1;
        unit_of(u, rb, ch, t0, t1);
        const int c0 = ch * kMaxChunk;
        const int cw = (int)min64(kMaxChunk, a.dp - c0);
        auto push_s = [&](int t) {
          for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = take(2 * kOpBytes);
            if (s < 0) break;
            tma_load_2d(sm.slot[s], &tmX, kb * BK, rb * TM, &sm.full[s]);
            tma_load_2d(sm.slot[s] + kOpBytes, &tmY, kb * BK, t * TN, &sm.full[s]);
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
      for (uint64_t q = (it > kSStages ? it - kSStages : 0); q < it; ++q) {
        const uint64_t t0 = now_ns();
        while (!mbar_try(&sm.full[q % kSStages], (uint32_t)((q / kSStages) & 1)) &&
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
        int rb, ch, t0, t1;
        unit_of(u, rb, ch, t0, t1);
        const int cw = (int)min64(kMaxChunk, a.dp - ch * kMaxChunk);
        // S tiles use TMEM buffer (tile & 1) in the forward, buffer 0 in the backward
        auto issue_s = [&](uint64_t tl) -> bool {
          const int buf = BWD ? 0 : (int)(tl & 1);
          const uint32_t ph = BWD ? (uint32_t)(tl & 1) : (uint32_t)((tl >> 1) & 1);
          if (!mbar_wait(&sm.s_empty[buf], ph ^ 1, limit_ns, abort)) return false;
          fence_after();
          const uint32_t d = tmem + (uint32_t)(buf * TN);
          for (int kb = 0; kb < nkb; ++kb, ++it) {
            const int s = (int)(it % kSStages);
            const uint32_t sp = (uint32_t)((it / kSStages) & 1);
            if (!mbar_wait(&sm.full[s], sp, limit_ns, abort)) return false;
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
        // backward product of tile tl: acc += G'_tl Z_tl^T
        auto issue_g = [&](uint64_t tl, bool first) -> bool {
          const int gb = 0;
          const uint32_t gph = (uint32_t)(tl & 1);
          if (!mbar_wait(&sm.g_full[gb], gph, limit_ns, abort)) return false;
          if (first && unit_n > 0) {
            if (!mbar_wait(&sm.acc_empty, (uint32_t)((unit_n - 1) & 1), limit_ns, abort))
              return false;
          }
          fence_after();
          for (int kz = 0; kz < 2; ++kz) {
            const uint32_t g0 = su32(sm.g[gb]) + kz * (TM * BK * 2);
            for (int p = 0; p < cw; p += kPiece, ++it) {
              const int pw = min(kPiece, cw - p);
              const int s = (int)(it % kSStages);
              const uint32_t sp = (uint32_t)((it / kSStages) & 1);
              if (!mbar_wait(&sm.full[s], sp, limit_ns, abort)) return false;
              fence_after();
              const uint32_t z0 = su32(sm.slot[s]);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem + TN + (uint32_t)p, sdesc(g0 + kk * 32), sdesc(z0 + kk * 32),
                         idesc_bf16(TM, pw), (first && kz == 0 && kk == 0) ? 0u : 1u);
              mma_commit(&sm.empty[s]);
            }
          }
          mma_commit(&sm.g_empty[gb]);
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
    // ---------------- epilogue (warps 2 and up) ----------------
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;  // row within the tile
    constexpr int NC = MODE == kModeFwd ? 4 : 2;  // 32-column chunks of a tile per warp
    const int cb = MODE == kModeFwd ? 0 : ((warp - 2) >> 2) * 2;  // first chunk of this warp
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
      int rb, ch, t0, t1;
      unit_of(u, rb, ch, t0, t1);
      const int64_t row = (int64_t)rb * TM + r;
      const bool valid = row < a.n;
      // forward state (log2 domain); the running sum is compensated (TwoSum),
      // so its error does not grow with N
      float m = -INFINITY, l = 0.f, lc = 0.f, diag = 0.f;
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
          const bool cols_full = col0 + TN <= a.n;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float x[32];
            float cm = -INFINITY;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              x[q] = v[c][q] * c1;
              if (!cols_full && col0 + c * 32 + q >= a.n) x[q] = -INFINITY;
              cm = fmaxf(cm, x[q]);
            }
            if (cm > m) {
              const float sc = (m == -INFINITY) ? 0.f : ex2(m - cm);
              l *= sc;
              lc *= sc;
              m = cm;
            }
            // pairwise sum of the chunk, then a compensated add into l
            float e[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) e[q] = ex2(x[q] - m);
#pragma unroll
            for (int w2 = 16; w2 >= 1; w2 >>= 1)
#pragma unroll
              for (int q = 0; q < w2; ++q) e[q] += e[q + w2];
            {
              const float t = __fadd_rn(l, e[0]);
              const float bp = __fsub_rn(t, l);
              lc = __fadd_rn(lc, __fadd_rn(__fsub_rn(l, __fsub_rn(t, bp)), __fsub_rn(e[0], bp)));
              l = t;
            }
            const int64_t jb = col0 + c * 32;
            if (row >= jb && row < jb + 32) {
#pragma unroll
              for (int q = 0; q < 32; ++q)
                if (jb + q == row) diag = v[c][q];
            }
          }
        } else {
          // G'_t = w_r (P - I) + w_c (Q - I), computed in place: one ex2 per
          // term and element; the column log-sum-exp (log2 domain) comes one
          // value per lane and is broadcast by shuffles; the diagonal and the
          // ragged last tile are fixed up apart from the element loop
          const float wr = a.wr, wc = a.wc;
          const bool cols_full = col0 + TN <= a.n;
          const int64_t dr = row - col0;  // position of the diagonal in the tile
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            float lcq = INFINITY;
            if (wc != 0.f) {
              const int64_t jj = col0 + (cb + c) * 32 + lane;
              if (jj < a.n) lcq = __ldg(a.lse_c + jj) * kLog2e;
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
                if (!valid || col0 + (cb + c) * 32 + q >= a.n) v[c][q] = 0.f;
          }
          // the G' tile buffer is free once the MMA warp (fused backward) or
          // the stores of the previous tile (G' pass) have read it
          const uint32_t gph = (uint32_t)(tile & 1);
          const bool we = mbar_wait(GP ? &sm.st_free : &sm.g_empty[0], gph ^ 1, limit_ns, abort);
          if (!__all_sync(0xffffffffu, we)) {
            flag_timeout(sm, &a.ctr->err_flags);
            ok = false;
            break;
          }
          unsigned char *gt = sm.g[0];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const float *gq = v[c];
            const int cc = cb + c;  // chunk of the tile
            // 32 columns = 4 chunks of 16 bytes in k-block (cc >> 1)
            unsigned char *kbase = gt + (cc >> 1) * (TM * BK * 2) + r * 128;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int lc = (cc & 1) * 4 + h;  // logical 16-byte chunk in the 128-byte row
              __nv_bfloat162 p0 = __floats2bfloat162_rn(gq[h * 8 + 0], gq[h * 8 + 1]);
              __nv_bfloat162 p1 = __floats2bfloat162_rn(gq[h * 8 + 2], gq[h * 8 + 3]);
              __nv_bfloat162 p2 = __floats2bfloat162_rn(gq[h * 8 + 4], gq[h * 8 + 5]);
              __nv_bfloat162 p3 = __floats2bfloat162_rn(gq[h * 8 + 6], gq[h * 8 + 7]);
              uint4 pk;
              pk.x = *reinterpret_cast<uint32_t *>(&p0);
              pk.y = *reinterpret_cast<uint32_t *>(&p1);
              pk.z = *reinterpret_cast<uint32_t *>(&p2);
              pk.w = *reinterpret_cast<uint32_t *>(&p3);
              *reinterpret_cast<uint4 *>(kbase + ((lc ^ (r & 7)) * 16)) = pk;
            }
          }
          if constexpr (GP) {
            // the transposed tile (row j, column i), same swizzled layout:
            // lanes 2m and 2m + 1 swap one value per column pair, then each
            // stores two adjacent i of one j as a 32-bit word
            unsigned char *tt = sm.g[1];
            const int ic = r & ~1;  // even i of the lane pair
            unsigned char *tbase = tt + (ic >> 6) * (TM * BK * 2) + (ic & 7) * 2;
            const int ichunk = (ic & 63) >> 3;
            const bool odd = (lane & 1) != 0;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
#pragma unroll
              for (int q = 0; q < 32; q += 2) {
                const float send = odd ? v[c][q] : v[c][q + 1];
                const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                const __nv_bfloat162 pr = odd ? __floats2bfloat162_rn(recv, v[c][q + 1])
                                              : __floats2bfloat162_rn(v[c][q], recv);
                const int j = (cb + c) * 32 + q + (odd ? 1 : 0);
                *reinterpret_cast<__nv_bfloat162 *>(tbase + j * 128 + ((ichunk ^ (j & 7)) << 4)) =
                    pr;
              }
            }
          }
          fence_proxy_async_smem();
          if constexpr (GP) {
            mbar_arrive(&sm.st_full);
            if (threadIdx.x == 64) {
              // one thread stores both tiles (two 64-column boxes each) once
              // every epilogue thread has written its part
              if (!mbar_wait(&sm.st_full, gph, limit_ns, abort)) {
                flag_timeout(sm, &a.ctr->err_flags);
              } else {
                const int y0 = rb * TM, x0 = (int)col0;
                tma_store_2d(&tmZ, sm.g[0], x0, y0);
                tma_store_2d(&tmZ, sm.g[0] + TM * BK * 2, x0 + BK, y0);
                tma_store_2d(&tmW, sm.g[1], y0, x0);
                tma_store_2d(&tmW, sm.g[1] + TM * BK * 2, y0 + BK, x0);
                bulk_commit();
                bulk_wait_read_all();
                mbar_arrive(&sm.st_free);
              }
            }
          } else {
            mbar_arrive(&sm.g_full[0]);
          }
        }
      }
      if (!ok) break;
      if constexpr (MODE == kModeFwd) {
        if (valid) {
          const float lse = (m + log2f(__fadd_rn(l, lc))) * 0.69314718055994531f;  // natural log
          a.lse_out[row] = lse;
          a.term_out[row] = lse - diag / a.T;
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
        const float scale = __ldg(a.grad_loss) / ((float)a.n * a.T);
        const int c0 = ch * kMaxChunk;
        const int cw = (int)min64(kMaxChunk, a.dp - c0);
        // each epilogue warp of a lane quarter stores its half of the chunk
        const int hw = cw / 2;
        for (int c = (cb / 2) * hw; c < (cb / 2 + 1) * hw; c += 32) {
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
    if (GP && threadIdx.x == 64) bulk_wait_all();
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------------------
// Materialised backward, second half: dX = (g / (N T)) G Z for G (np x np,
// BF16, row-major) and Z (np x d) given as Z^T (dp x np, BF16).  Unit =
// (128-row block, chunk of <= 384 output dimensions), accumulated over
// K = np in 64-wide k-blocks; a ring slot holds one k-block of G (16 KB) and
// of the chunk's Z^T rows (<= 48 KB).  Warp 0: TMA, warp 1: MMA, warps 2-5:
// readout (one TMEM lane quarter each).
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
  const int nkb = (int)(a.np / BK);
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
          tma_load_2d(sm.slot[s], &tmG, kb * BK, rb * TM, &sm.full[s]);
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
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_bf16(tmem + (uint32_t)p, sdesc(g0 + kk * 32),
                       sdesc(z0 + (uint32_t)p * BK * 2 + kk * 32), idesc_bf16(TM, pw),
                       (kb > 0 || kk > 0) ? 1u : 0u);
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
    const float scale = __ldg(a.grad_loss) / ((float)a.n * a.T);
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
__global__ void contrastive_loss_kernel(const float *t1, const float *t2, int64_t n, float w1,
                                        float w2, float *loss) {
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
    *loss = tot / (float)n;
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

cudaError_t launch_contrastive_pack(const float *X, int64_t n, int64_t d, void *Xp, void *XT,
                                    int64_t np, int64_t dp, unsigned *err, cudaStream_t st) {
  dim3 grid((unsigned)(dp / 32), (unsigned)(np / 32)), block(32, 8);
  contrastive_pack_kernel<<<grid, block, 0, st>>>(X, n, d, static_cast<__nv_bfloat16 *>(Xp),
                                                  static_cast<__nv_bfloat16 *>(XT), np, dp, err);
  return cudaGetLastError();
}

cudaError_t launch_contrastive_loss(const float *t1, const float *t2, int64_t n, float w1, float w2,
                                    float *loss, cudaStream_t st) {
  contrastive_loss_kernel<<<1, 1024, 0, st>>>(t1, t2, n, w1, w2, loss);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_mode(const CUtensorMap &mx, const CUtensorMap &my, const CUtensorMap &mz,
                               const CUtensorMap &mw, const ContrastiveArgs &a, int grid,
                               cudaStream_t st) {
  const size_t smem = contrastive_smem_bytes(MODE);
  cudaError_t e = cudaFuncSetAttribute(contrastive_kernel<MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  contrastive_kernel<MODE><<<grid, cthreads(MODE), smem, st>>>(mx, my, mz, mw, a);
  return cudaGetLastError();
}

cudaError_t launch_contrastive(int mode, const void *tmX, const void *tmY, const void *tmZ,
                               const void *tmW, const ContrastiveArgs &a, int grid,
                               cudaStream_t st) {
  CUtensorMap mx, my, mz, mw;
  std::memcpy(&mx, tmX, sizeof mx);
  std::memcpy(&my, tmY, sizeof my);
  std::memcpy(&mz, tmZ ? tmZ : tmX, sizeof mz);
  std::memcpy(&mw, tmW ? tmW : tmX, sizeof mw);
  switch (mode) {
    case kModeFwd: return launch_mode<kModeFwd>(mx, my, mz, mw, a, grid, st);
    case kModeBwd: return launch_mode<kModeBwd>(mx, my, mz, mw, a, grid, st);
    case kModeGp: return launch_mode<kModeGp>(mx, my, mz, mw, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t contrastive_gemm_smem_bytes() { return sizeof(GSmem) + 1024; }

cudaError_t launch_contrastive_gemm(const void *tmG, const void *tmZ, const ContrastiveGemmArgs &a,
                                    int grid, cudaStream_t st) {
  CUtensorMap mg, mz;
  std::memcpy(&mg, tmG, sizeof mg);
  std::memcpy(&mz, tmZ, sizeof mz);
  const size_t smem = contrastive_gemm_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(contrastive_gemm_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  contrastive_gemm_kernel<<<grid, kGemmThreads, smem, st>>>(mg, mz, a);
  return cudaGetLastError();
}

}  // namespace sj
