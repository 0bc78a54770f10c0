// finalize.cu -- from low-precision candidates to exact results.
//
// Top-k, per left row (one warp for the common case, one CTA otherwise):
//   1. theta = (k-th best s~ over all splits) - 2 m_i; keep band entries with
//      s~ >= theta.  They contain the exact top-k (see RowFilter).
//   2. Dot2 (compensated FP32) for each candidate -> a 64-bit key interval
//      [L, U] (units of 2^-60) that contains the exact score.
//   3. Sort by U desc; sweep into groups of chained overlapping intervals.
//      Groups are totally ordered (every member of a later group is strictly
//      below every member of an earlier one), so only the order INSIDE a
//      multi-member group is undecided.
//   4. Members of multi-member groups within the first k positions get their
//      exact value (fixed-point accumulator); sort those groups by
//      (exact desc, j asc).  Scores: float32 rounding of the interval when
//      both ends round alike, else of the exact value.
// The warp finaliser takes rows with at most 512 banded entries, at most 64
// candidates and no multi-member group in the needed prefix (no exact value
// needed); every other row goes to the CTA finaliser, in two tiers of
// shared-memory capacity.  A row whose band list overflowed, or with more
// candidates than the last tier holds, is re-ranked from scratch against all
// of B (fallback).
//
// Threshold: per candidate, Dot2 decides s >= tau unless tau lies inside the
// interval, where the exact value decides; accepted pairs are counted per row,
// placed by an exclusive scan of the counts and sorted by j inside each row.
#include <cfloat>
#include <climits>

#include "epilogue.cuh"

#include "rank.cuh"
#include "sj_device.cuh"
#include "sj_internal.h"

namespace sj {

namespace {

constexpr int kFinThreads = 128;
constexpr int kCMax = 1024;   // candidates per row, second tier
constexpr int kCSmall = 384;  // candidates per row, first tier (higher occupancy)
constexpr int64_t kRowInSmemMax = 16384;  // left row cached in shared memory up to this width

template <int CMAX>
struct FinSmemLayout {
  long long U[CMAX];
  long long L[CMAX];
  Exact ex[CMAX];
  int32_t j[CMAX];
  float v[CMAX];
  int32_t perm[CMAX];
  int32_t perm2[CMAX];
  int32_t grp[CMAX];
  float sc[CMAX];
  uint8_t flag[CMAX];
};

// One row (global row g) by the whole CTA.  A row whose band list overflowed
// goes to the rescan list with its key bound; a row with more than CMAX
// candidates goes to `defer` (with its key bound in defer_key when given: the
// last tier defers to the rescan list).
template <int CMAX>
__device__ void fin_row(const TopkFinalArgs &a, int64_t g, FinSmemLayout<CMAX> &sm, float *a_row,
                        int *defer, long long *defer_key, unsigned *n_defer) {
  __shared__ int s_n, s_overflow;
  __shared__ unsigned int s_maxerr;
  __shared__ unsigned s_cnt[kFinThreads / 32];
  if (g >= a.rows) return;
  const JobDev &jb = a.jobs[find_job_row0(a.jobs, a.n_jobs, g)];
  const int k = jb.k;
  if (k == 0) return;
  const int64_t i = g - jb.row0;  // row within the job
  const int S = jb.lists;
  const int *cnts = a.band_cnt + jb.slot0 + i * S;
  const Cand *bands = a.band + jb.band0 + i * S * (int64_t)jb.cap;
  const int64_t d = a.d;
  if (threadIdx.x == 0) {
    s_n = 0;
    s_overflow = 0;
    s_maxerr = 0;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x)
    if (cnts[s] < 0) s_overflow = 1;
  // k-th largest banded score over all lists (an overflowed list holds the
  // entries up to its overflow, which still bound the final value from below):
  // bisection on order-preserving keys, reading the lists in place
  uint32_t T = 0;
  int n_all = 0;
  for (int s = 0; s < S; ++s) {
    const int c = cnts[s];
    n_all += c < 0 ? -c - 1 : c;
  }
  for (int b = 31; b >= 0; --b) {
    const uint32_t t = T | (1u << b);
    unsigned c = 0;
    for (int s = 0; s < S; ++s) {
      const int cs = cnts[s];
      const int cnt = cs < 0 ? -cs - 1 : cs;
      const Cand *bl = bands + s * (int64_t)jb.cap;
      for (int q = threadIdx.x; q < cnt; q += blockDim.x) c += fkey(bl[q].v) >= t;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    unsigned tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_cnt[w];
    __syncthreads();
    if (tot >= (unsigned)k) T = t;
  }
  const float kth = n_all >= k ? fkey_inv(T) : -INFINITY;
  const float m = row_margin(a.metaA[jb.a_prow0 + i], jb.gmaxB, a.acc_coef);
  if (threadIdx.x == 0) atomicMax(&a.ctr->max_margin_bits, __float_as_uint(m));
  if (s_overflow) {
    if (threadIdx.x == 0) {
      // At least k rows have s~ >= kth, hence s >= kth - m: every exact top-k
      // member has s >= kth - m.  Key of that bound, rounded down.
      unsigned slot = atomicAdd(&a.ctr->overflow_rows, 1u);
      a.overflow_rows[slot] = (int)g;
      if (a.overflow_band) a.overflow_band[slot] = 0;  // needs the rescan of all of B
      a.overflow_key[slot] = kth == -INFINITY
                                 ? LLONG_MIN
                                 : __float2ll_rd(__fmul_rd(__fsub_rd(kth, m), 0x1p60f));
    }
    return;
  }
  const float theta = __fsub_rd(kth, __fmul_ru(2.f, m));
  for (int s = 0; s < S; ++s) {
    const int cnt = cnts[s];
    const Cand *bl = bands + s * (int64_t)jb.cap;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const Cand cd = bl[t];
      if (cd.v >= theta) {
        const int p = atomicAdd(&s_n, 1);
        if (p < CMAX) {
          sm.j[p] = cd.j;
          sm.v[p] = cd.v;
        }
      }
    }
  }
  __syncthreads();
  if (s_n > CMAX) {
    if (threadIdx.x == 0) {
      unsigned slot = atomicAdd(n_defer, 1u);
      defer[slot] = (int)g;
      if (defer_key) {  // the last tier: to the fallback, which scans the band lists
        defer_key[slot] = kth == -INFINITY
                              ? LLONG_MIN
                              : __float2ll_rd(__fmul_rd(__fsub_rd(kth, m), 0x1p60f));
        if (a.overflow_band) a.overflow_band[slot] = 1;
      }
    }
    return;
  }
  const int n = s_n;
  const float *a_src = jb.A + i * d;
  const float *B = jb.B;
  if (d <= kRowInSmemMax) {
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) a_row[t] = a_src[t];
    a_src = a_row;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const float nrm_a = a.metaA[jb.a_prow0 + i].nrm;
  const RowMeta *metaB = a.metaB + jb.b_prow0;
  for (int p = warp; p < n; p += nwarps) {
    float hi, lo;
    const int32_t j = sm.j[p];
    dot2_warp(a_src, B + (int64_t)j * d, d, hi, lo);
    if (lane == 0) {
      long long K = dot2_key(hi, lo);
      long long D = dot2_halfwidth(a.dot2_coef_key, nrm_a, metaB[j].nrm);
      sm.U[p] = K + D;
      sm.L[p] = K - D;
      float err = fabsf(__fsub_rn(__fsub_rn(sm.v[p], hi), lo));
      atomicMax(&s_maxerr, __float_as_uint(err));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&a.ctr->n_candidates, (unsigned long long)n);
    atomicAdd(&a.ctr->n_rescored, (unsigned long long)n);
    atomicMax(&a.ctr->max_err_bits, s_maxerr);
  }
  CandArrays c{sm.U, sm.L, sm.j, sm.v, sm.perm, sm.perm2, sm.grp, sm.flag, sm.sc, sm.ex};
  rank_and_emit(c, n, k, a_src, B, d, jb.out_idx + i * k, jb.out_score + i * k, a.ctr);
}

// CTA finaliser over a list of rows whose length a previous launch wrote.
template <int CMAX>
__global__ void __launch_bounds__(kFinThreads)
    topk_finalize_kernel(TopkFinalArgs a, const int *rows, const unsigned *n_rows, int *defer,
                         long long *defer_key, unsigned *n_defer) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FinSmemLayout<CMAX> &sm = *reinterpret_cast<FinSmemLayout<CMAX> *>(smem_raw);
  float *a_row = reinterpret_cast<float *>(smem_raw + sizeof(FinSmemLayout<CMAX>));
  const unsigned nr = *n_rows;
  if (a.ctr->err_flags) return;
  for (unsigned r = blockIdx.x; r < nr; r += gridDim.x) {
    fin_row<CMAX>(a, rows[r], sm, a_row, defer, defer_key, n_defer);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Warp finaliser.  Steps 1-4 of the CTA finaliser for one row per warp.  The
// k-th banded score comes from the lists' exact top-k values when the scoring
// pass kept them (the union's k best lie in the per-list k best), else from a
// bisection over the band entries; candidates are compacted into a per-warp
// shared-memory area holding their Dot2 key intervals, sorted by index with a
// bitonic network on (U desc, j asc); the group sweep is a running minimum of
// L.  Rows it cannot finish without an exact value, or with too many
// candidates, are appended to `defer` untouched (nothing of the row is
// written).
constexpr int kWarpMaxCand = 128;
constexpr int kFinWarps = 8;

struct WarpFinSmem {
  long long U[kWarpMaxCand], L[kWarpMaxCand];
  int32_t j[kWarpMaxCand];
  float v[kWarpMaxCand];
  int16_t perm[kWarpMaxCand];
  uint8_t open[kWarpMaxCand];  // position opens a group
};

__device__ __forceinline__ bool cand_before(const WarpFinSmem &w, int x, int y) {
  return w.U[x] > w.U[y] || (w.U[x] == w.U[y] && w.j[x] < w.j[y]);
}

// Largest key T with #{values with key >= T} >= k over n values at
// vals[0 .. n) (warp-cooperative bisection).
template <typename Get>
__device__ __forceinline__ uint32_t warp_kth_key(int n, int k, Get get) {
  uint32_t T = 0;
  for (int b = 31; b >= 0; --b) {
    const uint32_t tt = T | (1u << b);
    unsigned cnt = 0;
    for (int e = threadIdx.x & 31; e < n; e += 32) cnt += fkey(get(e)) >= tt;
    if (__reduce_add_sync(0xffffffffu, cnt) >= (unsigned)k) T = tt;
  }
  return T;
}

// Four blocks (32 warps) per SM: the kernel is bound by the latency of its
// gathers, so occupancy matters more than registers.
__global__ void __launch_bounds__(kFinWarps * 32, 4)
    topk_finalize_warp_kernel(TopkFinalArgs a, int *defer, unsigned *n_defer) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpFinSmem &w = reinterpret_cast<WarpFinSmem *>(smem_raw)[wib];
  const int64_t d = a.d;
  unsigned long long my_cand = 0;
  float my_err = 0.f, my_margin = 0.f;
  if (a.ctr->err_flags) return;
  const int64_t nwarps = (int64_t)gridDim.x * kFinWarps;
  const int64_t g0 = (int64_t)blockIdx.x * kFinWarps + wib;
  int q = g0 < a.rows ? find_job_row0(a.jobs, a.n_jobs, g0) : 0;
  for (int64_t g = g0; g < a.rows; g += nwarps) {
    q = advance_job_row0(a.jobs, a.n_jobs, q, g);
    const JobDev &jb = a.jobs[q];
    const int k = jb.k;
    if (k == 0) continue;
    const int64_t i = g - jb.row0;
    const int S = jb.lists;
    int c = 0;
    if (S <= 32 && lane < S) c = a.band_cnt[jb.slot0 + i * S + lane];
    int pre = c;  // inclusive prefix of the list counts
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(FULL, pre, off);
      if (lane >= off) pre += y;
    }
    const int n_all = __shfl_sync(FULL, pre, 31);
    if (S > 32 || __any_sync(FULL, c < 0)) {
      if (lane == 0) defer[atomicAdd(n_defer, 1u)] = (int)g;
      continue;
    }
    const Cand *bands = a.band + jb.band0 + i * S * (int64_t)jb.cap;
    // k-th largest banded score
    float kth = -INFINITY;
    if (jb.topv0 >= 0) {
      const float *tv = a.topv + jb.topv0 + i * S * (int64_t)k;
      if (S * k <= 32) {
        // one value per lane, loaded once (-inf padding adds to no count
        // above the smallest real value)
        const float mine = lane < S * k ? tv[lane] : -INFINITY;
        kth = fkey_inv(warp_kth_key(32, k, [&](int) { return mine; }));
      } else {
        kth = fkey_inv(warp_kth_key(S * k, k, [&](int e) { return tv[e]; }));
      }
    } else if (n_all >= k) {
      // bisection over the band entries, list by list (uniform list loop)
      uint32_t T = 0;
      for (int b = 31; b >= 0; --b) {
        const uint32_t tt = T | (1u << b);
        unsigned cnt = 0;
        for (int s = 0; s < S; ++s) {
          const int cs = __shfl_sync(FULL, c, s);
          const Cand *bl = bands + s * (int64_t)jb.cap;
          for (int qq = lane; qq < cs; qq += 32) cnt += fkey(bl[qq].v) >= tt;
        }
        if (__reduce_add_sync(FULL, cnt) >= (unsigned)k) T = tt;
      }
      kth = fkey_inv(T);
    }
    const float m = row_margin(a.metaA[jb.a_prow0 + i], jb.gmaxB, a.acc_coef);
    my_margin = fmaxf(my_margin, m);
    const float theta = __fsub_rd(kth, __fmul_ru(2.f, m));
    // candidates: band entries >= theta, compacted in list order
    int n = 0;
    for (int s = 0; s < S; ++s) {
      const int cs = __shfl_sync(FULL, c, s);
      const Cand *bl = bands + s * (int64_t)jb.cap;
      for (int q0 = 0; q0 < cs; q0 += 32) {
        const int qq = q0 + lane;
        const Cand cd = qq < cs ? bl[qq] : Cand{-INFINITY, 0};
        const bool pass = qq < cs && cd.v >= theta;
        const unsigned bal = __ballot_sync(FULL, pass);
        const int p = n + __popc(bal & ((1u << lane) - 1u));
        if (pass && p < kWarpMaxCand) {
          w.j[p] = cd.j;
          w.v[p] = cd.v;
        }
        n += __popc(bal);
      }
    }
    if (n > kWarpMaxCand) {
      if (lane == 0) defer[atomicAdd(n_defer, 1u)] = (int)g;
      __syncwarp();
      continue;
    }
    __syncwarp();
    // Dot2 key intervals of the candidates
    const float *a_src = jb.A + i * d;
    const float *B = jb.B;
    const RowMeta *metaB = a.metaB + jb.b_prow0;
    const float nrm_a = a.metaA[jb.a_prow0 + i].nrm;
    float err = 0.f;
    constexpr int NC = 4;
    for (int p0 = 0; p0 < n; p0 += NC) {
      const float *bp[NC];
      int32_t jq[NC];
#pragma unroll
      for (int t = 0; t < NC; ++t) {
        jq[t] = w.j[p0 + t < n ? p0 + t : p0];
        bp[t] = B + (int64_t)jq[t] * d;
      }
      float hi[NC], lo[NC];
      dot2_warp_sa<NC>(a_src, bp, d, hi, lo);
      // lane t < NC finishes candidate p0 + t, all NC lanes at once (each
      // picks its candidate's values by a select chain: static indices)
      float hm = hi[0], lm = lo[0];
      int32_t jm = jq[0];
#pragma unroll
      for (int t = 1; t < NC; ++t) {
        hm = lane == t ? hi[t] : hm;
        lm = lane == t ? lo[t] : lm;
        jm = lane == t ? jq[t] : jm;
      }
      if (lane < NC && p0 + lane < n) {
        const long long K = dot2_key(hm, lm);
        const long long D = dot2_halfwidth(a.dot2_coef_key, nrm_a, metaB[jm].nrm);
        w.U[p0 + lane] = K + D;
        w.L[p0 + lane] = K - D;
        err = fmaxf(err, fabsf(__fsub_rn(__fsub_rn(w.v[p0 + lane], hm), lm)));
      }
    }
    // sort candidate indices by (U desc, j asc); padding indices sort last
    int n_pad = 1;
    while (n_pad < n) n_pad <<= 1;
    for (int t = lane; t < n_pad; t += 32) w.perm[t] = (int16_t)(t < n ? t : -1);
    __syncwarp();
    for (int size = 2; size <= n_pad; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = lane; t < (n_pad >> 1); t += 32) {
          const int x = 2 * t - (t & (stride - 1));
          const int y = x + stride;
          const bool asc = (x & size) == 0;
          const int px = w.perm[x], py = w.perm[y];
          // "before": a real candidate earlier in (U desc, j asc); padding last
          const bool y_first = py >= 0 && (px < 0 || cand_before(w, py, px));
          if (asc == y_first) {
            w.perm[x] = (int16_t)py;
            w.perm[y] = (int16_t)px;
          }
        }
        __syncwarp();
      }
    }
    // group openings: U_p below every L before position p
    long long carry = LLONG_MAX;
    int n_need = n;
    for (int p0 = 0; p0 < n; p0 += 32) {
      const int p = p0 + lane;
      const int x = p < n ? w.perm[p] : 0;
      const long long Lp = p < n ? w.L[x] : LLONG_MAX;
      long long incl = Lp;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl = y < incl ? y : incl;
      }
      long long excl = __shfl_up_sync(FULL, incl, 1);
      if (lane == 0) excl = LLONG_MAX;
      excl = excl < carry ? excl : carry;
      const bool op = p < n && (p == 0 || w.U[x] < excl);
      if (p < n) w.open[p] = op ? 1 : 0;
      const unsigned bal = __ballot_sync(FULL, op && p >= k);
      if (bal && n_need == n) n_need = p0 + __ffs(bal) - 1;
      const long long tot = __shfl_sync(FULL, incl, 31);
      carry = tot < carry ? tot : carry;
    }
    __syncwarp();
    // needed positions must be single-member groups whose interval rounds to
    // one float32; otherwise the CTA finaliser resolves the row exactly
    const int kk = k < n ? k : n;
    bool bad = false;
    for (int p = lane; p < n_need; p += 32) {
      if (p >= 1 && !w.open[p]) bad = true;
      if (p < kk) {
        float sc;
        const int x = w.perm[p];
        if (!key_interval_round(w.L[x], w.U[x], sc)) bad = true;
      }
    }
    if (__any_sync(FULL, bad)) {
      if (lane == 0) defer[atomicAdd(n_defer, 1u)] = (int)g;
      __syncwarp();
      continue;
    }
    int64_t *oi = jb.out_idx + i * k;
    float *os = jb.out_score + i * k;
    for (int r = lane; r < k; r += 32) {
      int64_t jo = -1;
      float so = -INFINITY;
      if (r < kk) {
        const int x = w.perm[r];
        jo = w.j[x];
        key_interval_round(w.L[x], w.U[x], so);
      }
      oi[r] = jo;
      os[r] = so;
    }
    __syncwarp();
    my_cand += (unsigned long long)n;
    my_err = fmaxf(my_err, err);
  }
  my_err = fmaxf(my_err, __shfl_xor_sync(FULL, my_err, 1));
  my_err = fmaxf(my_err, __shfl_xor_sync(FULL, my_err, 2));
  if (lane == 0 && my_margin > 0.f) atomicMax(&a.ctr->max_margin_bits, __float_as_uint(my_margin));
  if (lane == 0 && my_cand) {
    atomicAdd(&a.ctr->n_candidates, my_cand);
    atomicAdd(&a.ctr->n_rescored, my_cand);
    atomicMax(&a.ctr->max_err_bits, __float_as_uint(my_err));
  }
}

// Fallback for rows whose candidates did not fit: rescan all of B with Dot2
// and keep every j whose upper bound reaches the row's key bound T (a proven
// superset of the exact top-k, see topk_finalize_kernel).  A block takes a
// range of columns and up to kRescanRows rows, so each B row is read once per
// block for all of them.
constexpr int kRescanRows = 8;
constexpr int kRescanCols = 256;

__global__ void __launch_bounds__(256) topk_rescan_kernel(RescanArgs a) {
  extern __shared__ __align__(16) float arows[];  // kRescanRows x d
  const int r0 = blockIdx.y * kRescanRows;
  const int nr = min(kRescanRows, a.n_rows - r0);
  for (int r = 0; r < nr; ++r)
    for (int64_t t = threadIdx.x; t < a.d; t += blockDim.x)
      arows[r * a.d + t] = a.A[(int64_t)a.rows[r0 + r] * a.d + t];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kRescanCols;
  const int64_t c1 = min64(a.nB, c0 + kRescanCols);
  for (int64_t j = c0 + warp; j < c1; j += nwarps) {
    const float *br = a.B + j * a.d;
    float s[kRescanRows], c[kRescanRows];
#pragma unroll
    for (int r = 0; r < kRescanRows; ++r) s[r] = c[r] = 0.f;
    for (int64_t k = lane; k < a.d; k += 32) {
      const float y = __ldg(br + k);
#pragma unroll
      for (int r = 0; r < kRescanRows; ++r)
        if (r < nr) dot2_step(arows[r * a.d + k], y, s[r], c[r]);
    }
    const float nb = a.metaB[j].nrm;
#pragma unroll
    for (int r = 0; r < kRescanRows; ++r) {
      if (r >= nr) break;
      float hi = s[r], lo = c[r];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        float s2 = __shfl_xor_sync(0xffffffffu, hi, off);
        float c2 = __shfl_xor_sync(0xffffffffu, lo, off);
        float t, q;
        two_sum(hi, s2, t, q);
        hi = t;
        lo = __fadd_rn(__fadd_rn(lo, c2), q);
      }
      if (lane == 0) {
        const int row = r0 + r;
        long long K = dot2_key(hi, lo);
        long long D = dot2_halfwidth(a.dot2_coef_key, a.metaA[a.rows[row]].nrm, nb);
        if (K + D >= a.keys[row]) {
          int slot = atomicAdd(a.count + row, 1);
          if (slot < a.cap) {
            KeyCand kc{K + D, K - D, (int32_t)j, 0};
            a.lists[(int64_t)row * a.cap + slot] = kc;
          }
        }
      }
    }
  }
  if (threadIdx.x == 0)
    atomicAdd(&a.ctr->n_rescored, (unsigned long long)((c1 - c0) * (int64_t)nr));
}

// Fallback for rows whose band lists are complete but hold more candidates
// than the block tiers take: Dot2 of every band entry of the row (a superset
// of the candidates >= the row's key bound, since the lists are) instead of
// all of B, kept when its upper bound reaches the key bound, into the same
// (U, L, j) lists as the rescan.  One block per row.
__global__ void __launch_bounds__(256) topk_bandscan_kernel(RescanArgs a) {
  extern __shared__ __align__(16) float arow[];  // the row, d floats
  const int r = blockIdx.x;
  const int i = a.rows[r];
  for (int64_t t = threadIdx.x; t < a.d; t += blockDim.x) arow[t] = a.A[(int64_t)i * a.d + t];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const float na = a.metaA[i].nrm;
  const long long key = a.keys[r];
  const int *cnts = a.band_cnt + (int64_t)i * a.band_lists;
  const Cand *bands = a.band + (int64_t)i * a.band_lists * a.band_cap;
  unsigned long long done = 0;
  for (int s = 0; s < a.band_lists; ++s) {
    const int cs = cnts[s];
    const int cnt = min(cs < 0 ? -cs - 1 : cs, a.band_cap);
    const Cand *bl = bands + (int64_t)s * a.band_cap;
    for (int q = warp; q < cnt; q += nwarps) {
      const int32_t j = bl[q].j;
      float hi, lo;
      dot2_warp(arow, a.B + (int64_t)j * a.d, a.d, hi, lo);
      if (lane == 0) {
        const long long K = dot2_key(hi, lo);
        const long long D = dot2_halfwidth(a.dot2_coef_key, na, a.metaB[j].nrm);
        if (K + D >= key) {
          const int slot = atomicAdd(a.count + r, 1);
          if (slot < a.cap) a.lists[(int64_t)r * a.cap + slot] = KeyCand{K + D, K - D, j, 0};
        }
        ++done;
      }
    }
  }
  if (lane == 0 && done) atomicAdd(&a.ctr->n_rescored, done);
}

// Rank each rescanned row from its (U, L, j) list.  Lists of up to kCMax
// entries are ranked in shared memory; longer ones are listed in `big` for
// the global-memory ranker; lists cut off at the capacity are listed in
// `redo` (the count is the capacity they need).
__global__ void __launch_bounds__(kFinThreads) topk_rank_lists_kernel(RankListArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FinSmemLayout<kCMax> &sm = *reinterpret_cast<FinSmemLayout<kCMax> *>(smem_raw);
  float *a_row = reinterpret_cast<float *>(smem_raw + sizeof(FinSmemLayout<kCMax>));
  __shared__ unsigned s_cnt[kFinThreads / 32];
  const int r = blockIdx.x;
  if (r >= a.n_rows) return;
  const int64_t i = a.rows[r];
  const int n = a.count[r];
  if (n > a.cap) {
    // Cut off: the k-th largest lower bound L among the stored entries bounds
    // the row's k-th exact score from below (k real scores are at least it),
    // so the redo only needs the columns whose upper bound reaches it.
    const KeyCand *lst = a.lists + (int64_t)r * a.cap;
    long long Lk = LLONG_MIN;
    if (a.cap >= a.k) {
      unsigned long long T = 0;  // order-preserving image of L: L ^ sign bit
      for (int b = 63; b >= 0; --b) {
        const unsigned long long t = T | (1ull << b);
        unsigned c = 0;
        for (int q = threadIdx.x; q < a.cap; q += blockDim.x)
          c += ((unsigned long long)lst[q].L ^ 0x8000000000000000ull) >= t;
        c = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = c;
        __syncthreads();
        unsigned tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_cnt[w];
        __syncthreads();
        if (tot >= (unsigned)a.k) T = t;
      }
      Lk = (long long)(T ^ 0x8000000000000000ull);
    }
    if (threadIdx.x == 0) {
      unsigned q = atomicAdd(&a.ctr->redo_rows, 1u);
      a.redo[q] = r;
      a.redo_key[q] = Lk > a.keys[r] ? Lk : a.keys[r];
      atomicMax(&a.ctr->redo_cap, (unsigned)n);
    }
    return;
  }
  if (n > kCMax) {
    if (threadIdx.x == 0) a.big[atomicAdd(&a.ctr->big_rows, 1u)] = r;
    return;
  }
  const KeyCand *lst = a.lists + (int64_t)r * a.cap;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    KeyCand kc = lst[t];
    sm.U[t] = kc.U;
    sm.L[t] = kc.L;
    sm.j[t] = kc.j;
    sm.v[t] = NAN;
  }
  const float *a_src = a.A + i * a.d;
  if (a.d <= kRowInSmemMax) {
    for (int64_t t = threadIdx.x; t < a.d; t += blockDim.x) a_row[t] = a_src[t];
    a_src = a_row;
  }
  __syncthreads();
  CandArrays c{sm.U, sm.L, sm.j, sm.v, sm.perm, sm.perm2, sm.grp, sm.flag, sm.sc, sm.ex};
  rank_and_emit(c, n, a.k, a_src, a.B, a.d, a.out_idx + i * a.k, a.out_score + i * a.k, a.ctr);
}

// Global-memory ranker for long lists (rare: massive exact ties).
__global__ void __launch_bounds__(1024) topk_rank_global_kernel(RankListArgs a, const int *big,
                                                               void *scratch, size_t per_row) {
  const int b = blockIdx.x;
  const int r = big[b];
  const int64_t i = a.rows[r];
  const int n = a.count[r];
  const int n_pad = next_pow2(n > 0 ? n : 1);
  unsigned char *base = static_cast<unsigned char *>(scratch) + (size_t)b * per_row;
  CandArrays c;
  c.U = reinterpret_cast<long long *>(base);
  c.L = c.U + n_pad;
  c.ex = reinterpret_cast<Exact *>(c.L + n_pad);
  c.j = reinterpret_cast<int32_t *>(c.ex + n_pad);
  c.v = reinterpret_cast<float *>(c.j + n_pad);
  c.perm = reinterpret_cast<int32_t *>(c.v + n_pad);
  c.perm2 = c.perm + n_pad;
  c.grp = c.perm2 + n_pad;
  c.sc = reinterpret_cast<float *>(c.grp + n_pad);
  c.flag = reinterpret_cast<uint8_t *>(c.sc + n_pad);
  const KeyCand *lst = a.lists + (int64_t)r * a.cap;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    KeyCand kc = lst[t];
    c.U[t] = kc.U;
    c.L[t] = kc.L;
    c.j[t] = kc.j;
    c.v[t] = NAN;
  }
  __syncthreads();
  rank_and_emit(c, n, a.k, a.A + i * a.d, a.B, a.d, a.out_idx + i * a.k, a.out_score + i * a.k,
                a.ctr);
}

// ---------------------------------------------------------------------------
// Threshold

// Threshold candidates bucketed by left row before rescoring.  The scoring
// CTAs push candidates of many jobs at once, so in push order the Dot2
// gathers touch the B rows of many jobs together (far more than L2 holds).
// In row order the rows of one job are contiguous: the warps in flight read
// one or two jobs' B rows, which stay in L2, and share each A row.
// Counting pass, then (after an exclusive scan of the counts) placement.
__global__ void thr_count_kernel(const ThrCand *cand, const unsigned long long *n_cand,
                                 int64_t cap, const Counters *ctr, int64_t *cnt) {
  const int64_t n = ctr->err_flags ? 0 : min64((int64_t)*n_cand, cap);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long *>(cnt + cand[c].i), 1ull);
}

// cursor[i] starts at row i's exclusive offset; the order inside a row is
// arbitrary (the accepted pairs are sorted by j afterwards).
__global__ void thr_bucket_kernel(const ThrCand *cand, const unsigned long long *n_cand,
                                  int64_t cap, const Counters *ctr, int64_t *cursor,
                                  ThrCand *out) {
  const int64_t n = ctr->err_flags ? 0 : min64((int64_t)*n_cand, cap);
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const ThrCand cd = cand[c];
    const unsigned long long slot =
        atomicAdd(reinterpret_cast<unsigned long long *>(cursor + cd.i), 1ull);
    out[slot] = cd;
  }
}

// One warp evaluates four candidates at a time (Dot2 gathers interleaved).
__global__ void thr_rescore_kernel(ThrFinalArgs a) {
  constexpr int NC = 4;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_cand = a.ctr->err_flags ? 0 : min64((int64_t)*a.n_cand, a.cand_cap);
  const int64_t d = a.d;
  unsigned long long n_exact = 0;
  int hint = 0;  // candidates arrive grouped by job (pushed per scoring unit)
  for (int64_t c0 = w0 * NC; c0 < n_cand; c0 += nw * NC) {
    ThrCand t[NC];
    const JobDev *jq[NC];
    int64_t li[NC];
    const float *ap[NC], *bp[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      t[q] = a.cand[c0 + q < n_cand ? c0 + q : c0];
      hint = find_job_row0_hint(a.jobs, a.n_jobs, hint, t[q].i);
      jq[q] = &a.jobs[hint];
      li[q] = t[q].i - jq[q]->row0;
      ap[q] = jq[q]->A + li[q] * d;
      bp[q] = jq[q]->B + (int64_t)t[q].j * d;
    }
    float hi[NC], lo[NC];
    bool same_a = true;
#pragma unroll
    for (int q = 1; q < NC; ++q) same_a = same_a && ap[q] == ap[0];
    if (same_a)  // the common case: candidates are grouped by row
      dot2_warp_sa<NC>(ap[0], bp, d, hi, lo);
    else
      dot2_warp_n<NC>(ap, bp, d, hi, lo);
    // decisions are warp-uniform (every lane holds the reduced hi, lo)
    unsigned acc = 0;
    float sq[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      sq[q] = 0.f;
      if (c0 + q >= n_cand) break;
      const JobDev &jb = *jq[q];
      const long long K = dot2_key(hi[q], lo[q]);
      const long long D = dot2_halfwidth(a.dot2_coef_key, a.metaA[jb.a_prow0 + li[q]].nrm,
                                         a.metaB[jb.b_prow0 + t[q].j].nrm);
      int in;
      bool have_ex = false;
      Exact ex;
      if (K - D >= jb.tau_key) {
        in = 1;
      } else if (K + D < jb.tau_key) {
        in = 0;
      } else {
        ex = exact_dot_warp(ap[q], bp[q], d);
        have_ex = true;
        ++n_exact;
        in = exact_cmp(ex, jb.tau_exact) >= 0;
      }
      if (!in) continue;
      float s;
      if (!key_interval_round(K - D, K + D, s)) {
        if (!have_ex) {
          ex = exact_dot_warp(ap[q], bp[q], d);
          ++n_exact;
        }
        s = exact_to_float(ex);
      }
      sq[q] = s;
      acc |= 1u << q;
    }
    // one slot reservation per warp and group of candidates; lane q stores
    // candidate q
    if (acc) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&a.ctr->n_pairs, (unsigned long long)__popc(acc));
      base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        if (lane == q && ((acc >> q) & 1u)) {
          atomicAdd(reinterpret_cast<unsigned long long *>(a.row_count + t[q].i), 1ull);
          a.accepted[base + __popc(acc & ((1u << q) - 1u))] = ThrCand{t[q].i, t[q].j, sq[q], 0};
        }
      }
    }
  }
  if (lane == 0 && n_exact) atomicAdd(&a.ctr->n_exact, n_exact);
}

// Exclusive scan helpers (3 phases).
constexpr int kScanThreads = 1024, kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ long long block_exclusive_scan(long long v, long long *sh, long long &total) {
  // sh: blockDim.x / 32 entries
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < nw) sh[lane] = w;
  }
  __syncthreads();
  long long before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
  total = sh[nw - 1];
  __syncthreads();
  return before;
}

__global__ void scan_reduce_kernel(const int64_t *in, int64_t n, long long *block_sums) {
  __shared__ long long sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  long long s = 0;
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
    if (idx < n) s += in[idx];
  }
  long long total;
  block_exclusive_scan(s, sh, total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void scan_top_kernel(long long *block_sums, int64_t nb, int64_t *total_out) {
  __shared__ long long sh[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    int64_t idx = b0 + threadIdx.x;
    long long v = idx < nb ? block_sums[idx] : 0;
    long long total;
    long long ex = block_exclusive_scan(v, sh, total);
    if (idx < nb) block_sums[idx] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void scan_apply_kernel(const int64_t *in, int64_t *out, int64_t n,
                                  const long long *block_sums) {
  __shared__ long long sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  long long vals[kScanItems];
  long long s = 0;
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
    vals[q] = idx < n ? in[idx] : 0;
    s += vals[q];
  }
  long long total;
  long long ex = block_exclusive_scan(s, sh, total) + block_sums[blockIdx.x];
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
    if (idx < n) out[idx] = ex;
    ex += vals[q];
  }
}

// Destination of global row i's pairs (see launch_thr_scatter).
__device__ __forceinline__ PairOut *pair_seg(const JobDev &jb, PairOut *staging,
                                             const int64_t *row_off, int64_t i) {
  return jb.out_pairs ? jb.out_pairs + (row_off[i] - row_off[jb.row0]) : staging + row_off[i];
}

__global__ void job_pairs_kernel(JobDev *jobs, int n_jobs, int64_t rows, const int64_t *row_off,
                                 const int64_t *total, int64_t *job_info) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_jobs) return;
  JobDev &jb = jobs[q];
  int64_t np = 0, off = 0;
  if (jb.nA > 0) {
    off = row_off[jb.row0];
    const int64_t end = jb.row0 + jb.nA < rows ? row_off[jb.row0 + jb.nA] : *total;
    np = end - off;
  }
  jb.n_pairs = np;
  job_info[2 * q] = np;
  job_info[2 * q + 1] = off;
}

__global__ void thr_scatter_kernel(const JobDev *jobs, int n_jobs, const ThrCand *acc,
                                   const unsigned long long *n_acc_dev, int64_t cap,
                                   const int64_t *row_off, int64_t *row_fill, PairOut *staging) {
  const int64_t n = min64((int64_t)*n_acc_dev, cap);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const ThrCand c = acc[t];
    const JobDev &jb = jobs[find_job_row0(jobs, n_jobs, c.i)];
    if (jb.n_pairs > jb.capacity) continue;
    unsigned long long r =
        atomicAdd(reinterpret_cast<unsigned long long *>(row_fill + c.i), 1ull);
    pair_seg(jb, staging, row_off, c.i)[r] = PairOut{c.i - jb.row0, c.j, c.v, 0};
  }
}

// Sort each row's pairs by j: rows of <= 32 pairs inside one warp, larger
// rows are listed for the block kernel.
__global__ void thr_sort_small_kernel(const JobDev *jobs, int n_jobs, int64_t rows,
                                      const int64_t *row_off, const int64_t *row_count,
                                      PairOut *staging, int *big_rows, int *n_big) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= rows) return;
  const int64_t cnt = row_count[row];
  if (cnt <= 1) return;
  const JobDev &jb = jobs[find_job_row0(jobs, n_jobs, row)];
  if (jb.n_pairs > jb.capacity) return;
  if (cnt > 32) {
    if (lane == 0) big_rows[atomicAdd(n_big, 1)] = (int)row;
    return;
  }
  PairOut *seg = pair_seg(jb, staging, row_off, row);
  PairOut p = lane < cnt ? seg[lane] : PairOut{0, INT64_MAX, 0.f, 0};
  // bitonic over 32 lanes by j
  for (int size = 2; size <= 32; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      long long oj = __shfl_xor_sync(0xffffffffu, (long long)p.j, stride);
      float os = __shfl_xor_sync(0xffffffffu, p.score, stride);
      const bool lower = (lane & stride) == 0;
      const bool asc = (lane & size) == 0;
      const bool keep_min = (lower == asc);
      const bool take_other = keep_min ? (oj < p.j) : (oj > p.j);
      if (take_other) {
        p.j = oj;
        p.score = os;
      }
    }
  }
  if (lane < cnt) seg[lane] = p;
}

// Rank-based merge sort of one large row in global memory (distinct j keys),
// ping-ponging with the row's range of `tmp` (concatenated order).
__global__ void thr_sort_big_kernel(const JobDev *jobs, int n_jobs, PairOut *staging,
                                    PairOut *tmp, const int64_t *row_off,
                                    const int64_t *row_count, const int *big_rows,
                                    const int *n_big) {
  const int nb = *n_big;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t row = big_rows[b];
    const int64_t n = row_count[row];
    const JobDev &jb = jobs[find_job_row0(jobs, n_jobs, row)];
    PairOut *const home = pair_seg(jb, staging, row_off, row);
    PairOut *src = home;
    PairOut *dst = tmp + row_off[row];
    for (int64_t width = 1; width < n; width <<= 1) {
      for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        int64_t run = t / width;
        int64_t run_start = run * width;
        int64_t pair_start = (run & ~1ll) * width;
        bool left = (run & 1) == 0;
        int64_t other_start = left ? run_start + width : run_start - width;
        int64_t other_len = left ? max64(0, min64(width, n - other_start)) : width;
        long long key = src[t].j;
        // number of elements in the other run with a smaller key
        int64_t lo = 0, hi = other_len;
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (src[other_start + mid].j < key) lo = mid + 1;
          else hi = mid;
        }
        dst[pair_start + (t - run_start) + lo] = src[t];
      }
      __syncthreads();
      PairOut *sw = src;
      src = dst;
      dst = sw;
    }
    if (src != home) {
      for (int64_t t = threadIdx.x; t < n; t += blockDim.x) home[t] = src[t];
    }
    __syncthreads();
  }
}

}  // namespace

template <int CMAX>
static cudaError_t launch_fin(const TopkFinalArgs &a, const int *rows, const unsigned *n_rows,
                              int grid, int *defer, long long *defer_key, unsigned *n_defer,
                              cudaStream_t st) {
  const size_t smem =
      sizeof(FinSmemLayout<CMAX>) + (a.d <= kRowInSmemMax ? (size_t)a.d * sizeof(float) : 0);
  cudaError_t e = cudaFuncSetAttribute(topk_finalize_kernel<CMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  topk_finalize_kernel<CMAX><<<(unsigned)grid, kFinThreads, smem, st>>>(a, rows, n_rows, defer,
                                                                       defer_key, n_defer);
  return cudaGetLastError();
}

cudaError_t launch_topk_finalize(const TopkFinalArgs &a, int sm_count, cudaStream_t st) {
  if (a.rows == 0) return cudaSuccess;
  // warp finaliser over every row; the rows it defers go to the first CTA
  // tier, whose rows beyond kCSmall candidates go to the second, whose rows
  // beyond kCMax go to the rescan list.  Counts stay on the device.
  const int64_t want = (a.rows + kFinWarps - 1) / kFinWarps;
  const int gw = (int)min64(want, (int64_t)sm_count * 4);
  const size_t wsm = sizeof(WarpFinSmem) * kFinWarps;
  cudaError_t e = cudaFuncSetAttribute(topk_finalize_warp_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
  if (e != cudaSuccess) return e;
  topk_finalize_warp_kernel<<<(unsigned)gw, kFinWarps * 32, wsm, st>>>(a, a.defer_rows,
                                                                       &a.ctr->defer_rows);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_fin<kCSmall>(a, a.defer_rows, &a.ctr->defer_rows, sm_count * 4, a.tier2_rows,
                          nullptr, &a.ctr->tier2_rows, st);
  if (e != cudaSuccess) return e;
  return launch_fin<kCMax>(a, a.tier2_rows, &a.ctr->tier2_rows, sm_count * 2, a.overflow_rows,
                           a.overflow_key, &a.ctr->overflow_rows, st);
}

size_t topk_rank_global_row_bytes(int64_t n) {
  int64_t n_pad = 1;
  while (n_pad < n) n_pad <<= 1;
  // U, L, ex, j, v, perm, perm2, grp, sc, flag
  return (size_t)n_pad * (8 + 8 + sizeof(Exact) + 4 + 4 + 4 + 4 + 4 + 4 + 1) + 256;
}

cudaError_t launch_topk_rescan(const RescanArgs &a, cudaStream_t st) {
  if (a.n_rows == 0 || a.nB == 0) return cudaSuccess;
  if (a.band) {
    const size_t smem = (size_t)a.d * sizeof(float);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(topk_bandscan_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    topk_bandscan_kernel<<<(unsigned)a.n_rows, 256, smem, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)kRescanRows * a.d * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(topk_rescan_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((a.nB + kRescanCols - 1) / kRescanCols),
            (unsigned)((a.n_rows + kRescanRows - 1) / kRescanRows));
  topk_rescan_kernel<<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_topk_rank_lists(const RankListArgs &a, cudaStream_t st) {
  if (a.n_rows == 0) return cudaSuccess;
  const size_t smem =
      sizeof(FinSmemLayout<kCMax>) + (a.d <= kRowInSmemMax ? (size_t)a.d * sizeof(float) : 0);
  cudaError_t e = cudaFuncSetAttribute(topk_rank_lists_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  topk_rank_lists_kernel<<<a.n_rows, kFinThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_topk_rank_global(const RankListArgs &a, const int *big, int n_big,
                                    void *scratch, size_t per_row, cudaStream_t st) {
  if (n_big == 0) return cudaSuccess;
  topk_rank_global_kernel<<<n_big, 1024, 0, st>>>(a, big, scratch, per_row);
  return cudaGetLastError();
}

cudaError_t launch_thr_bucket(const ThrCand *cand, const unsigned long long *n_cand,
                              int64_t cap, const Counters *ctr, int64_t rows, int64_t *cnt,
                              int64_t *off, int64_t *total, void *scan_scratch, ThrCand *out,
                              int grid, cudaStream_t st) {
  if (grid <= 0 || rows == 0) return cudaSuccess;
  thr_count_kernel<<<(unsigned)grid, 256, 0, st>>>(cand, n_cand, cap, ctr, cnt);
  cudaError_t e = launch_exclusive_scan(cnt, off, rows, total, scan_scratch, st);
  if (e != cudaSuccess) return e;
  thr_bucket_kernel<<<(unsigned)grid, 256, 0, st>>>(cand, n_cand, cap, ctr, off, out);
  return cudaGetLastError();
}

cudaError_t launch_thr_rescore(const ThrFinalArgs &a, int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  thr_rescore_kernel<<<(unsigned)grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

size_t scan_scratch_bytes(int64_t n) {
  int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  return (size_t)(nb + 1) * sizeof(long long);
}

cudaError_t launch_exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                                  void *scratch, cudaStream_t st) {
  int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  long long *bs = static_cast<long long *>(scratch);
  if (nb == 0) {
    return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
  }
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, bs);
  scan_top_kernel<<<1, kScanThreads, 0, st>>>(bs, nb, total);
  scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, bs);
  return cudaGetLastError();
}

cudaError_t launch_job_pairs(JobDev *jobs, int n_jobs, int64_t rows, const int64_t *row_off,
                             const int64_t *total, int64_t *job_info, cudaStream_t st) {
  if (n_jobs == 0) return cudaSuccess;
  job_pairs_kernel<<<(n_jobs + 255) / 256, 256, 0, st>>>(jobs, n_jobs, rows, row_off, total,
                                                         job_info);
  return cudaGetLastError();
}

cudaError_t launch_thr_scatter(const JobDev *jobs, int n_jobs, const ThrCand *accepted,
                               const unsigned long long *n_acc, int64_t acc_cap,
                               const int64_t *row_off, int64_t *row_fill, PairOut *staging,
                               int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  thr_scatter_kernel<<<(unsigned)grid, 256, 0, st>>>(jobs, n_jobs, accepted, n_acc, acc_cap,
                                                     row_off, row_fill, staging);
  return cudaGetLastError();
}

cudaError_t launch_thr_sort_rows(const JobDev *jobs, int n_jobs, int64_t rows,
                                 const int64_t *row_off, const int64_t *row_count,
                                 PairOut *staging, int *big_rows, int *n_big, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const int64_t blocks = (rows * 32 + 255) / 256;
  thr_sort_small_kernel<<<(unsigned)blocks, 256, 0, st>>>(jobs, n_jobs, rows, row_off, row_count,
                                                          staging, big_rows, n_big);
  return cudaGetLastError();
}

cudaError_t launch_thr_sort_big(const JobDev *jobs, int n_jobs, PairOut *staging, PairOut *tmp,
                                const int64_t *row_off, const int64_t *row_count,
                                const int *big_rows, const int *n_big, int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  thr_sort_big_kernel<<<(unsigned)grid, 512, 0, st>>>(jobs, n_jobs, staging, tmp, row_off,
                                                      row_count, big_rows, n_big);
  return cudaGetLastError();
}

}  // namespace sj
