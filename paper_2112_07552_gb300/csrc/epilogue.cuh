// epilogue.cuh -- the fused filter every scoring kernel applies to its tile.
//
// The thread that owns left row i sees the low-precision scores s~_ij of one
// tile, in increasing j, and keeps
//   * (s~, j) in the row's band list when s~ >= theta_i,
//   * (i, j, s~) in the threshold candidate list when s~ >= tau - m_i,
// so the |A| x |B| score matrix never reaches HBM (the analogue of fusing
// nonzero() of Sec. 3.2 into the product).
//
// Top-k filter.  |s~_ij - s_ij| <= m_i for every j.  With s~_(k) the k-th
// largest s~ of the row, every exact top-k member has s~ >= s~_(k) - 2 m_i
// (k rows have s >= s~_(k) - m_i).  theta_i is at most s~_(k) - 2 m_i over
// the columns seen so far, which never exceeds the final value, so the band
// list is a superset of the final candidates.  The tensor-core epilogue
// tracks the running k best exactly for k <= 32 (a sorted register array);
// otherwise theta_i is refreshed from the list when it has doubled since the
// last refresh or is full: the warp finds the k-th largest banded score
// (bisection on order-preserving integer keys) and compacts the list.  The
// row's k best scores always pass and are never compacted away, so the final
// list holds them and the finaliser recomputes s~_(k) from it.
#pragma once

#include <cooperative_groups.h>

#include "sj_device.cuh"
#include "sj_internal.h"

namespace sj {

struct RowCtx {
  int64_t slot;   // band-list slot (band_cnt index)
  int k;          // the job's k (0: no top-k part)
  float theta;    // top-k filter (+inf: no top-k part)
  float tau_lo;   // threshold filter: keep if s~ >= tau - m_i (+inf: off)
  float two_m;    // 2 m_i, rounded up
  int cnt;        // band list fill
  int last;       // fill right after the last refresh of theta
  int overflow;   // band list could not be compacted below the limit
  Cand *band;     // cap entries
  bool exact;     // theta tracks the running k-th best exactly (kept by the caller)
  uint32_t kth_key;  // lazy theta: key of the list's k-th entry at the last refresh
  float to_s;     // stored score = visited value * to_s (a power of two; E4M3 scoring
                  // visits accumulator units, with theta, tau_lo, two_m in those units)
  int32_t i;      // global left row
};

// Running k best of a row in registers, for k <= KM (KM = 16 or 32): a
// descending array whose first KM - k slots hold +inf sentinels, so the k-th
// best is always the last slot (static index, no local memory).
constexpr int kTopKRegs = 32;

template <int KM>
__device__ __forceinline__ void topk_regs_init(float (&h)[KM], int k) {
#pragma unroll
  for (int t = 0; t < KM; ++t) h[t] = t < KM - k ? INFINITY : -INFINITY;
}

// Insert v (> h[last]) and drop the smallest: branch-free shift-insert.
template <int KM>
__device__ __forceinline__ void topk_regs_insert(float (&h)[KM], float v) {
#pragma unroll
  for (int t = KM - 1; t >= 1; --t) h[t] = fmaxf(h[t], fminf(v, h[t - 1]));
  h[0] = fmaxf(h[0], v);
}

// Append a threshold candidate (warp-aggregated atomic on the global count).
__device__ __forceinline__ void push_thr(const ScoreArgs &a, int32_t i, int32_t j, float v) {
  namespace cg = cooperative_groups;
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&a.ctr->thr_count, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  unsigned long long slot = base + g.thread_rank();
  if (slot < a.thr_cap) a.thr[slot] = ThrCand{i, j, v, 0};
}

// Margin m_i: |s~_ij - s_ij| <= m_i for every j.
//   <a,b> - <a~,b~> = <a - a~, b> + <a~, b - b~>  (Cauchy-Schwarz on each)
//   plus the accumulation error of the scoring pass, acc_coef ||a~|| ||b~||.
// With the hi/lo split the products summed are hi.hi + hi.lo + lo.hi =
// <a~, b~> - <a_lo, b_lo> (a~ = a_hi + a_lo), so the dropped term adds
// ||a_lo|| ||b_lo||, and the accumulation acts on a sum of |products| at most
// (||a_hi|| + ||a_lo||)(||b_hi|| + ||b_lo||), the qnrm of the split.
// All factors are upper bounds, combined with upward rounding.
__device__ __forceinline__ float row_margin(const RowMeta &m, const float *gmaxB, float acc_coef) {
  float t1 = __fmul_ru(m.qerr, gmaxB[0]);
  float t2 = __fmul_ru(m.qnrm, gmaxB[2]);
  float t3 = __fmul_ru(__fmul_ru(acc_coef, m.qnrm), gmaxB[1]);
  float t4 = __fmul_ru(m.lonrm, gmaxB[3]);
  return __fadd_ru(__fadd_ru(__fadd_ru(t1, t2), t3), t4);
}

// `local` is the row within its job; `list` numbers the row's band lists:
// split * bands_per_split + column group.
__device__ __forceinline__ void row_begin(RowCtx &r, const ScoreArgs &a, const JobDev &jb,
                                          int64_t local, int list) {
  r.i = (int32_t)(jb.row0 + local);
  r.k = jb.k;
  const float m = row_margin(a.metaA[jb.a_prow0 + local], jb.gmaxB, a.acc_coef);
  r.two_m = __fmul_ru(2.f, m);
  r.tau_lo = __fsub_rd(jb.tau_f, m);
  r.cnt = 0;
  r.last = 0;
  r.overflow = 0;
  r.slot = jb.slot0 + local * jb.lists + list;
  r.band = a.band + jb.band0 + (local * jb.lists + list) * (int64_t)jb.cap;
  r.theta = jb.k > 0 ? -INFINITY : INFINITY;
  r.kth_key = 0;
  r.to_s = 1.f;
}

// Band count of the (row, split); an overflowed list stores -(cnt + 1), its
// entries up to the overflow staying valid.
__device__ __forceinline__ void row_end(const RowCtx &r, const ScoreArgs &a) {
  if (r.k > 0) a.band_cnt[r.slot] = r.overflow ? -r.cnt - 1 : r.cnt;
}

// Visit one score that passed min(theta, tau_lo).  The band list always has
// room for a chunk of 32 visits (the owner compacts before each chunk).
__device__ __forceinline__ void row_push(RowCtx &r, const ScoreArgs &a, float v, int32_t j) {
  if (v >= r.theta && !r.overflow) {
    r.band[r.cnt] = Cand{v * r.to_s, j};
    r.cnt += 1;
  }
  if (v >= r.tau_lo) push_thr(a, r.i, j, v * r.to_s);
}

// The same with the running k best in registers: theta is exact at all times.
template <int KM>
__device__ __forceinline__ void row_push_regs(RowCtx &r, float (&h)[KM], const ScoreArgs &a,
                                              float v, int32_t j) {
  // branch-free apart from the stores: lanes of a warp visit different
  // scores at once, and an insert of -inf (a score below theta) leaves the
  // array, and so theta, unchanged
  const bool in = v >= r.theta;
  if (in && !r.overflow) {
    r.band[r.cnt] = Cand{v * r.to_s, j};
    r.cnt += 1;
  }
  topk_regs_insert<KM>(h, in ? v : -INFINITY);
  // never below a bound adopted from the row's other list
  r.theta = fmaxf(r.theta, __fsub_rd(h[KM - 1], r.two_m));
  if (v >= r.tau_lo) push_thr(a, r.i, j, v * r.to_s);
}

// Order-preserving map of non-NaN floats to unsigned integers.
__device__ __forceinline__ uint32_t fkey(float v) {
  uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Warp-cooperative refresh of theta and compaction of every row of this warp
// whose band list holds more than `limit` entries, or at least k entries and
// twice as many as right after its last refresh (at least kRefresh more).  A
// refresh is a 32-step bisection over the whole list, so refreshes are spaced
// geometrically: a list whose band is dense (hundreds of near-ties) is
// refreshed a few times, not once per 32 entries; a stale theta only lets
// more scores into the list, which the next refresh drops.  Must be called
// by all 32 lanes (each lane owning at most one row; non-owners pass
// has_row = false).
// LAZY: theta is refreshed from the list (r.exact false); otherwise the
// caller tracks the running k-th exactly (r.exact true) and the list is only
// compacted when full.  A template parameter, so that the exact kernels carry
// no bisection code (registers).
constexpr int kRefresh = 32;
template <bool LAZY>
__device__ __forceinline__ void warp_compact(RowCtx &r, bool has_row, int k, int limit) {
  const int lane = threadIdx.x & 31;
  // with an exact theta: compact only when the list is full
  const bool due = !LAZY ? r.cnt > limit
                         : (r.cnt > limit ||
                            (r.cnt >= k && r.cnt >= r.last + max(kRefresh, r.last)));
  unsigned need = __ballot_sync(0xffffffffu, has_row && !r.overflow && due);
  while (need) {
    const int src = __ffs(need) - 1;
    need &= need - 1;
    const int n = __shfl_sync(0xffffffffu, r.cnt, src);
    const unsigned long long bp =
        __shfl_sync(0xffffffffu, (unsigned long long)reinterpret_cast<uintptr_t>(r.band), src);
    Cand *band = reinterpret_cast<Cand *>((uintptr_t)bp);
    // band values are scores; the row's thresholds are in its visiting units
    // (score / to_s): convert exactly (to_s is a power of two)
    const float to_s = __shfl_sync(0xffffffffu, r.to_s, src);
    const float two_m = __shfl_sync(0xffffffffu, r.two_m, src) * to_s;
    const float theta_old = __shfl_sync(0xffffffffu, r.theta, src) * to_s;
    float theta = theta_old;
    uint32_t T = 0;
    if constexpr (LAZY) {
      // k-th largest banded score: the largest key T with #{key >= T} >= k,
      // by bisection between the k-th of the last refresh (the list's k-th
      // only rises: entries are only added, and compaction drops entries
      // below theta, which stays below it) and the list's largest key.  A
      // result without k entries at or above it can only be that earlier
      // k-th, itself a lower bound of the row's k-th score, so theta stays
      // valid either way.
      uint32_t lo = __shfl_sync(0xffffffffu, r.kth_key, src), hi = 0;
      for (int q = lane; q < n; q += 32) hi = max(hi, fkey(band[q].v));
      hi = __reduce_max_sync(0xffffffffu, hi);
      if (hi < lo) hi = lo;
      while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1) + 1;  // in (lo, hi]
        unsigned c = 0;
        for (int q = lane; q < n; q += 32) c += fkey(band[q].v) >= mid;
        c = __reduce_add_sync(0xffffffffu, c);
        if (c >= (unsigned)k) lo = mid;
        else hi = mid - 1;
      }
      T = lo;
      theta = fmaxf(theta_old, __fsub_rd(fkey_inv(T), two_m));
    }
    // stable in-place compaction: a chunk is read fully before it is written
    int w = 0;
    for (int base = 0; base < n; base += 32) {
      const int q = base + lane;
      Cand cd = q < n ? band[q] : Cand{-INFINITY, 0};
      const bool keep = q < n && cd.v >= theta;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) band[w + __popc(bal & ((1u << lane) - 1u))] = cd;
      w += __popc(bal);
    }
    __syncwarp();
    if (lane == src) {
      if (LAZY) r.kth_key = T;
      r.theta = theta / to_s;
      r.cnt = w;
      r.last = w;
      if (w > limit) {
        // the band near the k-th score is too dense: the row goes to the
        // fallback, which needs only the entries kept so far (their k-th
        // largest bounds the row's k-th score from below), so the rest of
        // its columns make no more top-k visits (threshold visits go on)
        r.overflow = 1;
        r.theta = INFINITY;
      }
    }
  }
}

}  // namespace sj
