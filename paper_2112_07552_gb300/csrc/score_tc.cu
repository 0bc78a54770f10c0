// score_tc.cu -- tensor-core scoring pass for sm_103a (tcgen05 + TMA + TMEM).
//
// s~ = a~ . b~ for bfloat16 operands, products exact and accumulated in FP32
// in tensor memory.  The score matrix is a dense contraction (Sec. 3.1:
// C = mat(A) mat(B)^T), so it runs on the 5th-generation tensor cores; the
// paper's own kernels (WMMA on Ampere/Turing) are prior art only.
//
// Persistent kernel, one CTA per SM, warp-specialised (320 threads):
//   warp 0     TMA producer: 128x64 A tile + 256x64 B tile per k-block into a
//              4-stage ring of 128B-swizzled shared memory buffers;
//   warp 1     TMEM allocator + MMA issuer: tcgen05.mma kind::f16, M=128,
//              N=256, K=16, into one of two 256-column TMEM accumulators;
//   warps 2-9  epilogue: two warps per 32-lane TMEM quarter (the quarter a
//              warp may access is its index mod 4), each taking one half of
//              the tile's columns; tcgen05.ld (one left row per thread),
//              fused top-k / threshold filter (epilogue.cuh) with one band
//              list and register top-k per (row, column half): passing
//              scores are queued while the accumulator is held and visited
//              after it is released to the MMA warp.
// Work unit = (128-row block of A, column split of B); CTAs take units
// round-robin.  Every wait is bounded (globaltimer); a wait that gives up
// flags SJ_ERR_TIMEOUT, the CTA drains its in-flight copies and MMAs,
// frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>

#include "epilogue.cuh"
#include "tc_common.cuh"
#include "tc_host.h"

namespace sj {

namespace {

using namespace tc;

constexpr int BM = kTcBM;       // 128 rows of A per tile (TMEM lanes)
constexpr int BN = kTcBN;       // 256 columns of B per tile (TMEM columns)
constexpr int kRowBytes = 128;  // k-block: one 128-byte swizzle row per tile row
constexpr int BK = 64;          // k-block elements, BF16 (E4M3: 128)
constexpr int STAGES = 4;
constexpr int kEpiChunks = 1;  // 32-column chunks per TMEM round trip (1: no spills)
constexpr int kRegsSmallK = 16;  // k <= 16: 16 register slots; 16 < k <= kTcExactMaxK: 32
static_assert(kTcExactMaxK <= kTopKRegs, "register top-k size");
constexpr int kEpiWarps = 8;    // two per TMEM lane quarter
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;
constexpr int kQueueFlush = 2;  // a warp drains once one of its lanes holds this many
constexpr uint32_t kTileABytes = BM * BK * 2;
constexpr uint32_t kTileBBytes = BN * BK * 2;
constexpr uint32_t kTmemCols = 2 * BN;  // two accumulators
constexpr uint32_t kIdesc = idesc_bf16(BM, BN);
constexpr uint32_t kIdescNarrow = idesc_bf16(BM, kTcBNNarrow);
constexpr uint32_t kIdesc8 = idesc_e4m3(BM, BN);
constexpr uint32_t kIdesc8Narrow = idesc_e4m3(BM, kTcBNNarrow);
constexpr int kMmaPerStage = 4;  // 32 bytes of K per instruction (16 BF16 or 32 E4M3)

struct alignas(1024) TcSmem {
  unsigned char a[STAGES][kTileABytes];  // each 1024-byte aligned
  unsigned char b[STAGES][kTileBBytes];
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tmem_full[2];
  uint64_t tmem_empty[2];
  uint64_t drain;
  uint64_t never;  // debug-timeout hook: nothing ever arrives here
  // per-thread visit queues (score, column): entry e of epilogue thread t at
  // [e][t], so a warp's lanes fall in distinct banks
  float qv[kTcQueue][kEpiThreads];
  int32_t qj[kTcQueue][kEpiThreads];
  // each (column half, tile row)'s latest theta, tagged with its unit:
  // (tag << 32) | float bits
  unsigned long long kpub[2][BM];
  uint32_t tmem_base;
  int abort;
};

// The two column halves of a row share their thresholds.  Each half's theta
// is at most (k-th best of the columns it has seen) - 2m, and the k-th best
// of any subset of a row's columns is at most the row's, so either half may
// filter with the larger of the two: its band list still holds every final
// candidate of its columns, and the row's top-k members it holds are among
// its k best visited scores, so the finaliser's k-th (from the lists' top-k
// or by bisection over the lists) is unchanged.  The tag (unit + 1) keeps a
// half from adopting a value its partner published for the previous unit's
// row; an overflowed list (theta = +inf) publishes nothing.
__device__ __forceinline__ void theta_publish(TcSmem &sm, int half, int r, uint32_t tag,
                                              const RowCtx &rc) {
  if (rc.overflow || !(rc.theta > -INFINITY)) return;
  *reinterpret_cast<volatile unsigned long long *>(&sm.kpub[half][r]) =
      ((unsigned long long)tag << 32) | __float_as_uint(rc.theta);
}
__device__ __forceinline__ void theta_adopt(TcSmem &sm, int half, int r, uint32_t tag,
                                            RowCtx &rc) {
  const unsigned long long p =
      *reinterpret_cast<volatile unsigned long long *>(&sm.kpub[half ^ 1][r]);
  if ((uint32_t)(p >> 32) == tag && !rc.overflow)
    rc.theta = fmaxf(rc.theta, __uint_as_float((uint32_t)p));
}

// One visit of a score that passed min(theta, tau_lo): band list, running
// top-k (KM > 0 register slots; KM == 0: lazy theta) and threshold list.
template <int KM>
__device__ __forceinline__ void visit(RowCtx &rc, float (&h)[KM > 0 ? KM : 1], const ScoreArgs &a,
                                      float v, int32_t j) {
  if constexpr (KM > 0) row_push_regs<KM>(rc, h, a, v, j);
  else row_push(rc, a, v, j);
}

// The thread's queued visits, in arrival order, against the current theta.
template <int KM>
__device__ __forceinline__ void drain_queue(RowCtx &rc, float (&h)[KM > 0 ? KM : 1],
                                            const ScoreArgs &a, const float *qv,
                                            const int32_t *qj, int &qn) {
#pragma unroll 1
  for (int e = 0; e < qn; ++e) visit<KM>(rc, h, a, qv[e * kEpiThreads], qj[e * kEpiThreads]);
  qn = 0;
}

// Fused filter over 32 scores of the thread's row, columns jb .. jb+31.
// Scores >= min(theta, tau_lo) are appended to the thread's queue; a full
// queue is drained on the spot.  theta only rises, so a queued score that a
// later theta would reject is rejected when it is drained, and filtering
// with the theta of the chunk start keeps a superset.
template <int KM>
__device__ __forceinline__ void epilogue_chunk(RowCtx &rc, float (&h)[KM > 0 ? KM : 1],
                                               const ScoreArgs &a, const float (&v)[32],
                                               int64_t jb, int64_t nB, float *qv, int32_t *qj,
                                               int &qn) {
  // fast path: one compare per 32 scores (balanced max tree)
  float p16[16], q8[8];
#pragma unroll
  for (int q = 0; q < 16; ++q) p16[q] = fmaxf(v[2 * q], v[2 * q + 1]);
#pragma unroll
  for (int q = 0; q < 8; ++q) q8[q] = fmaxf(p16[2 * q], p16[2 * q + 1]);
  const float mx = fmaxf(fmaxf(fmaxf(q8[0], q8[1]), fmaxf(q8[2], q8[3])),
                         fmaxf(fmaxf(q8[4], q8[5]), fmaxf(q8[6], q8[7])));
  const float tmin = fminf(rc.theta, rc.tau_lo);
  if (mx >= tmin) {
    // loop over the passing quads; the quad's registers are picked by a
    // select tree on the bits of its index (static register indices, no
    // indirect branch: lanes with different quads do not serialise)
    uint32_t qm = 0;
#pragma unroll
    for (int g = 0; g < 8; ++g) qm |= (q8[g] >= tmin ? 1u : 0u) << g;
    while (qm) {
      const int g = __ffs(qm) - 1;
      qm &= qm - 1;
      float xs[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool g0 = (g & 1) != 0, g1 = (g & 2) != 0, g2 = (g & 4) != 0;
        const float s0 = g0 ? v[4 + e] : v[e], s1 = g0 ? v[12 + e] : v[8 + e];
        const float s2 = g0 ? v[20 + e] : v[16 + e], s3 = g0 ? v[28 + e] : v[24 + e];
        const float t0 = g1 ? s1 : s0, t1 = g1 ? s3 : s2;
        xs[e] = g2 ? t1 : t0;
      }
      const int64_t jq = jb + 4 * g;
      // room for the quad first, then four predicated appends
      if (qn > kTcQueue - 4) drain_queue<KM>(rc, h, a, qv, qj, qn);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float x = xs[e];
        if (x >= tmin && jq + e < nB) {
          qv[qn * kEpiThreads] = x;
          qj[qn * kEpiThreads] = (int32_t)(jq + e);
          ++qn;
        }
      }
    }
  }
}

// The k-blocks of one score tile, in increasing order, handed to f (which
// returns false to stop): every k-block when scoring dense; with occupancy
// bitmaps, the k-blocks nonzero in the A row group and in one of the B tile's
// row groups.  A skipped k-block contributes exactly 0 to every score of the
// tile, so the accumulators equal the dense ones; a tile with no k-block left
// is all zeros (the epilogue then reads no accumulator).  Returns the count,
// -1 when f stopped.
template <bool SPARSE, class F>
__device__ __forceinline__ int tile_kblocks(const ScoreArgs &a, int64_t nkb, int64_t arow,
                                            int64_t brow, int bn, F &&f) {
  if constexpr (!SPARSE) {
    for (int64_t kb = 0; kb < nkb; ++kb)
      if (!f(kb)) return -1;
    return (int)nkb;
  }
  const uint32_t *oa = a.occ + (arow / 128) * a.occ_words;
  const uint32_t *ob0 = a.occ + (brow / 128) * a.occ_words;
  const uint32_t *ob1 = bn > 128 ? ob0 + a.occ_words : ob0;
  int n = 0;
  for (int w = 0; w < a.occ_words; ++w) {
    uint32_t m = __ldg(oa + w) & (__ldg(ob0 + w) | __ldg(ob1 + w));
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      if (!f((int64_t)w * 32 + b)) return -1;
      ++n;
    }
  }
  return n;
}

__device__ __forceinline__ void flag_timeout(TcSmem &sm, Counters *ctr) {
  *(volatile int *)&sm.abort = 1;
  atomicOr(&ctr->err_flags, kErrTimeout);
}

// The epilogue warps' share of one unit: the row's running top-k in
// registers (KM > 0 slots) or none (KM == 0: lazy theta), every tile of the
// unit's column range from tensor memory through the fused filter, then the
// row's band count and exact top-k values.  While a tile's accumulator is
// held, passing scores only go to the thread's queue; the warp drains its
// queues after releasing the accumulator, so the visits (band and threshold
// pushes, top-k inserts) overlap the next tiles' MMAs and run on all lanes
// with queued visits at once.
template <int KM, bool FP8, bool SPARSE>
__device__ __forceinline__ void epilogue_unit(TcSmem &sm, const ScoreArgs &a, const UnitDev &un,
                                              const JobDev &jb, int64_t row, bool owner,
                                              int list, uint32_t tmem, int quarter, int half,
                                              uint64_t limit_ns, uint64_t &tile, bool &ok,
                                              uint32_t tag) {
  volatile int *abort = &sm.abort;
  const int rt = quarter * 32 + (int)(threadIdx.x & 31);  // row within the tile
  const int kj = jb.k;
  // Band room: before a chunk, for its 32 visits plus a full queue; before a
  // drain, for the queue alone.  (A list whose entries at or above theta do
  // not fit in that room is marked overflowed and goes to the fallback.)
  const int limit = jb.cap - 32 - kTcQueue;
  const int limit_drain = jb.cap - kTcQueue;
  static_assert(32 + kTcQueue <= 64, "band room of the lists (capacity plan)");
  const int64_t nB = jb.nB;
  RowCtx rc;
  rc.cnt = 0;
  rc.overflow = 0;
  rc.k = kj;
  rc.theta = INFINITY;
  rc.tau_lo = INFINITY;
  rc.exact = KM != 0;
  float h[KM > 0 ? KM : 1];
  const int et = (int)threadIdx.x - 64;  // epilogue thread index
  float *qv = &sm.qv[0][et];
  int32_t *qj = &sm.qj[0][et];
  int qn = 0;
  if constexpr (KM > 0) topk_regs_init<KM>(h, kj);
  if (owner) row_begin(rc, a, jb, row, list);
  if (a.raw_m != nullptr && owner)
    a.raw_m[row] = row_margin(a.metaA[jb.a_prow0 + row], jb.gmaxB, a.acc_coef);
  if constexpr (FP8) {
    // E4M3 scores come out of the tensor core as acc = s~ 2^(e_i + e_B): the
    // filter works on acc (thresholds scaled exactly by the power of two)
    // and stored values are scaled back
    if (owner) {
      const int e = a.metaA[jb.a_prow0 + row].sexp + jb.eB;
      rc.to_s = __int_as_float((127 - e) << 23);
      const float sc = __int_as_float((127 + e) << 23);
      rc.theta *= sc;
      rc.tau_lo *= sc;
      rc.two_m *= sc;
    }
  }
  const int64_t ct0 = (int64_t)un.split * jb.tiles_per_split;
  const int64_t ct1 = min64(jb.n_col_tiles, ct0 + jb.tiles_per_split);
  for (int64_t ct = ct0; ct < ct1; ++ct, ++tile) {
    const int acc = (int)(tile & 1);
    const uint32_t aph = (uint32_t)((tile >> 1) & 1);
    // warp-uniform outcome: the TMEM loads below are .sync.aligned
    const bool w = mbar_wait(&sm.tmem_full[acc], aph, limit_ns, abort);
    if (!__all_sync(0xffffffffu, w)) {
      flag_timeout(sm, a.ctr);
      ok = false;
      break;
    }
    fence_after();
    const int bn = jb.bn;
    const int64_t col0 = ct * bn;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN);
    // block-sparse: a tile without a common nonzero k-block is all zeros and
    // its accumulator was not written
    bool zero_tile = false;
    if constexpr (SPARSE)
      zero_tile = tile_kblocks<true>(a, 0 /* only the bitmaps are read */,
                                     jb.a_prow0 + (int64_t)un.rb * BM, jb.b_prow0 + col0, bn,
                                     [](int64_t) { return false; }) == 0;
    if (owner && kj > 0) theta_adopt(sm, half, rt, tag, rc);
    // kEpiChunks 32-column chunks per TMEM round trip
#pragma unroll 1
    for (int c0 = half * (bn / 2); c0 < (half + 1) * (bn / 2); c0 += 32 * kEpiChunks) {
      float v0[32], v1[32];
      if (SPARSE && zero_tile) {
#pragma unroll
        for (int t = 0; t < 32; ++t) v0[t] = v1[t] = 0.f;
      } else {
        tmem_ld32_nowait(taddr + c0, v0);
        if constexpr (kEpiChunks == 2) {
          tmem_ld32_nowait(taddr + c0 + 32, v1);
          tmem_wait_ld(v0, v1);
        } else {
          tmem_wait_ld1(v0);
        }
      }
      if (a.raw != nullptr && owner) {
        float *dst = a.raw + row * nB;
#pragma unroll
        for (int t = 0; t < 32; ++t) {  // static indices: v0/v1 stay in registers
          if (col0 + c0 + t < nB) dst[col0 + c0 + t] = v0[t] * rc.to_s;
          if (kEpiChunks == 2 && col0 + c0 + 32 + t < nB) dst[col0 + c0 + 32 + t] = v1[t] * rc.to_s;
        }
      }
      if (kj > 0) warp_compact<KM == 0>(rc, owner, kj, limit);
      if (owner) epilogue_chunk<KM>(rc, h, a, v0, col0 + c0, nB, qv, qj, qn);
      if constexpr (kEpiChunks == 2) {
        if (kj > 0) warp_compact<KM == 0>(rc, owner, kj, limit);
        if (owner) epilogue_chunk<KM>(rc, h, a, v1, col0 + c0 + 32, nB, qv, qj, qn);
      }
    }
    if (owner && kj > 0) theta_publish(sm, half, rt, tag, rc);
    fence_before();
    mbar_arrive(&sm.tmem_empty[acc]);
    // the accumulator is released: drain once a lane holds kQueueFlush visits
    if (__any_sync(0xffffffffu, qn >= kQueueFlush)) {
      if (kj > 0) warp_compact<KM == 0>(rc, owner, kj, limit_drain);
      if (owner) drain_queue<KM>(rc, h, a, qv, qj, qn);
      if (owner && kj > 0) theta_publish(sm, half, rt, tag, rc);
    }
  }
  if (kj > 0) warp_compact<KM == 0>(rc, owner, kj, limit_drain);
  if (owner) {
    drain_queue<KM>(rc, h, a, qv, qj, qn);
    row_end(rc, a);
    if constexpr (KM > 0) {
      if (jb.topv0 >= 0) {
        // the list's k best (any order)
        float *tv = a.topv + jb.topv0 + (row * jb.lists + list) * (int64_t)kj;
#pragma unroll
        for (int t = 0; t < KM; ++t)
          if (t >= KM - kj) tv[t - (KM - kj)] = h[t] * rc.to_s;
      }
    }
  }
}

template <bool FP8, bool SPARSE>
__global__ void __launch_bounds__(kThreads, 1)
    score_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmB128, ScoreArgs a, uint32_t flags) {
  extern __shared__ unsigned char smem_raw[];
  TcSmem &sm = *reinterpret_cast<TcSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool debug_timeout = (flags & SJ_FLAG_DEBUG_TIMEOUT) != 0;
  const uint64_t limit_ns = 4000000000ull;  // 4 s per wait
  volatile int *abort = &sm.abort;
  // inputs that failed validation: nothing to score (uniform over the grid)
  if (*(volatile unsigned *)&a.ctr->err_flags & (kErrNonFinite | kErrNotUnit)) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&sm.tmem_full[q], 1);
      mbar_init(&sm.tmem_empty[q], kEpiWarps * 32);
    }
    mbar_init(&sm.drain, 1);
    mbar_init(&sm.never, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int t = threadIdx.x; t < 2 * BM; t += kThreads) (&sm.kpub[0][0])[t] = 0ull;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&sm.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;

  constexpr int BKE = FP8 ? 2 * BK : BK;  // elements per 128-byte k-block
  const int64_t nkb = a.dp / BKE;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint64_t it = 0;
      bool ok = true;
      for (int64_t unit = blockIdx.x; unit < a.n_units && ok; unit += gridDim.x) {
        const UnitDev un = a.units[unit];
        const JobDev &jb = a.jobs[un.job];
        const int64_t ct0 = (int64_t)un.split * jb.tiles_per_split;
        const int64_t ct1 = min64(jb.n_col_tiles, ct0 + jb.tiles_per_split);
        const int arow = (int)(jb.a_prow0 + (int64_t)un.rb * BM);
        for (int64_t ct = ct0; ct < ct1 && ok; ++ct) {
          const bool narrow = jb.bn == kTcBNNarrow;
          const int brow = (int)(jb.b_prow0 + ct * jb.bn);
          const int n = tile_kblocks<SPARSE>(a, nkb, arow, brow, jb.bn, [&](int64_t kb) {
            const int s = (int)(it % STAGES);
            const uint32_t ph = (uint32_t)((it / STAGES) & 1);
            if (!mbar_wait(&sm.empty[s], ph ^ 1, limit_ns, abort)) {
              flag_timeout(sm, a.ctr);
              return false;
            }
            ++it;
            mbar_arrive_expect_tx(&sm.full[s],
                                  kTileABytes + (narrow ? kTileBBytes / 2 : kTileBBytes));
            tma_load_2d(sm.a[s], &tmA, (int)(kb * BKE), arow, &sm.full[s]);
            tma_load_2d(sm.b[s], narrow ? &tmB128 : &tmB, (int)(kb * BKE), brow, &sm.full[s]);
            return true;
          });
          if (n < 0) ok = false;
        }
      }
      // Drain: the last load issued into each stage must have landed before the
      // CTA may exit (normal exit: they were consumed long ago).
      for (uint64_t q = (it > STAGES ? it - STAGES : 0); q < it; ++q) {
        const int s = (int)(q % STAGES);
        const uint32_t ph = (uint32_t)((q / STAGES) & 1);
        uint64_t t0 = now_ns();
        while (!mbar_try(&sm.full[s], ph) && now_ns() - t0 < limit_ns) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint64_t it = 0, tile = 0;
      bool ok = true;
      for (int64_t unit = blockIdx.x; unit < a.n_units && ok; unit += gridDim.x) {
        const UnitDev un = a.units[unit];
        const JobDev &jb = a.jobs[un.job];
        const int64_t ct0 = (int64_t)un.split * jb.tiles_per_split;
        const int64_t ct1 = min64(jb.n_col_tiles, ct0 + jb.tiles_per_split);
        const uint32_t idesc = FP8 ? (jb.bn == kTcBNNarrow ? kIdesc8Narrow : kIdesc8)
                                   : (jb.bn == kTcBNNarrow ? kIdescNarrow : kIdesc);
        for (int64_t ct = ct0; ct < ct1 && ok; ++ct, ++tile) {
          const int acc = (int)(tile & 1);
          const uint32_t aph = (uint32_t)((tile >> 1) & 1);
          if (!mbar_wait(&sm.tmem_empty[acc], aph ^ 1, limit_ns, abort)) {
            flag_timeout(sm, a.ctr);
            ok = false;
            break;
          }
          fence_after();
          const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
          const int arow = (int)(jb.a_prow0 + (int64_t)un.rb * BM);
          const int brow = (int)(jb.b_prow0 + ct * jb.bn);
          bool first = true;  // the tile's first MMA overwrites the accumulator
          const int n = tile_kblocks<SPARSE>(a, nkb, arow, brow, jb.bn, [&](int64_t) {
            const int s = (int)(it % STAGES);
            const uint32_t ph = (uint32_t)((it / STAGES) & 1);
            if (!mbar_wait(&sm.full[s], ph, limit_ns, abort)) {
              flag_timeout(sm, a.ctr);
              return false;
            }
            ++it;
            fence_after();
            const uint32_t a0 = su32(sm.a[s]), b0 = su32(sm.b[s]);
#pragma unroll
            for (int kk = 0; kk < kMmaPerStage; ++kk) {
              if constexpr (FP8)
                mma_e4m3(d_tmem, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc,
                         (!first || kk > 0) ? 1u : 0u);
              else
                mma_bf16(d_tmem, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc,
                         (!first || kk > 0) ? 1u : 0u);
            }
            first = false;
            mma_commit(&sm.empty[s]);  // frees the smem stage once these MMAs finish
            return true;
          });
          if (n < 0) ok = false;
          if (!ok) break;
          mma_commit(&sm.tmem_full[acc]);  // accumulator ready for the epilogue
        }
      }
      // Drain: every MMA issued so far completes before tensor memory is freed.
      mma_commit(&sm.drain);
      uint64_t t0 = now_ns();
      while (!mbar_try(&sm.drain, 0) && now_ns() - t0 < limit_ns) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int quarter = warp & 3;        // TMEM lanes this warp may access
    const int half = (warp - 2) >> 2;    // column half of each tile
    const int r_in_tile = quarter * 32 + lane;
    uint64_t tile = 0;
    bool ok = true;
    if (debug_timeout) {
      // test hook: a wait on a barrier nothing arrives at must give up cleanly
      const bool w = mbar_wait(&sm.never, 0, 1000000ull, abort);
      if (!__all_sync(0xffffffffu, w)) {
        flag_timeout(sm, a.ctr);
        ok = false;
      }
    }
    for (int64_t unit = blockIdx.x; unit < a.n_units && ok; unit += gridDim.x) {
      const UnitDev un = a.units[unit];
      const JobDev &jb = a.jobs[un.job];
      const int64_t row = (int64_t)un.rb * BM + r_in_tile;  // local row of the job
      const bool owner = row < jb.nA;
      const int kj = jb.k;
      const int list = un.split * a.bands_per_split + half;
      const uint32_t tag = (uint32_t)unit + 1u;  // never 0, the cleared value
      if (kj > 0 && kj <= kRegsSmallK)
        epilogue_unit<kRegsSmallK, FP8, SPARSE>(sm, a, un, jb, row, owner, list, tmem, quarter, half,
                                        limit_ns, tile, ok, tag);
      else if (kj > 0 && kj <= kTcExactMaxK)
        epilogue_unit<kTcExactMaxK, FP8, SPARSE>(sm, a, un, jb, row, owner, list, tmem, quarter, half,
                                         limit_ns, tile, ok, tag);
      else
        epilogue_unit<0, FP8, SPARSE>(sm, a, un, jb, row, owner, list, tmem, quarter, half, limit_ns,
                                      tile, ok, tag);
    }
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side

struct TcContext {
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};

sj_status tc_create(TcContext **out) {
  TcContext *c = new TcContext();
  cudaDriverEntryPointQueryResult q;
  void *fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                    cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    delete c;
    return SJ_ERR_UNSUPPORTED;
  }
  c->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  *out = c;
  return SJ_OK;
}

void tc_destroy(TcContext *ctx) { delete ctx; }

sj_status tc_encode_2d(TcContext *ctx, const void *base, int64_t inner, int64_t rows,
                       int box_inner, int box_rows, unsigned char out[128], int elem) {
  if (!ctx || !ctx->encode) return SJ_ERR_UNSUPPORTED;
  CUtensorMap m;
  std::memset(&m, 0, sizeof m);
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(inner * elem)};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode(&m, elem == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                         : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           2, const_cast<void *>(base),
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return SJ_ERR_CUDA;
  static_assert(sizeof(CUtensorMap) == 128, "CUtensorMap size");
  std::memcpy(out, &m, sizeof m);
  return SJ_OK;
}

sj_status tc_make_maps(TcContext *ctx, const void *Ap, int64_t nA_pad, const void *Bp,
                       int64_t nB_pad, int64_t dp, TcMaps *out, int elem) {
  if (!ctx || !ctx->encode) return SJ_ERR_UNSUPPORTED;
  // B tiles never cross a segment end (segments are padded to BN rows)
  const int box = kRowBytes / elem;  // elements per 128-byte swizzle row
  if (dp % box != 0 || nA_pad % BM != 0 || nB_pad < BN) return SJ_ERR_INTERNAL;
  sj_status s = tc_encode_2d(ctx, Ap, dp, nA_pad, box, BM, out->a, elem);
  if (s == SJ_OK) s = tc_encode_2d(ctx, Bp, dp, nB_pad, box, BN, out->b, elem);
  if (s == SJ_OK) s = tc_encode_2d(ctx, Bp, dp, nB_pad, box, kTcBNNarrow, out->b128, elem);
  return s;
}

cudaError_t launch_score_tc(const ScoreArgs &a, int grid, const TcMaps *maps, uint32_t flags,
                            bool fp8, cudaStream_t st) {
  if (a.n_units == 0) return cudaSuccess;
  if (a.bands_per_split != 2) return cudaErrorInvalidValue;  // one list per column half
  const size_t smem = sizeof(TcSmem) + 1024;
  // the dense instantiations carry none of the block-sparse code
  auto kern = a.occ != nullptr ? (fp8 ? score_tc_kernel<true, true> : score_tc_kernel<false, true>)
                               : (fp8 ? score_tc_kernel<true, false> : score_tc_kernel<false, false>);
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  CUtensorMap ma, mb, mb128;
  std::memcpy(&ma, maps->a, sizeof ma);
  std::memcpy(&mb, maps->b, sizeof mb);
  std::memcpy(&mb128, maps->b128, sizeof mb128);
  kern<<<grid, kThreads, smem, st>>>(ma, mb, mb128, a, flags);
  return cudaGetLastError();
}

}  // namespace sj
