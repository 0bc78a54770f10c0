// epilogue.cuh -- the fused filter every scoring kernel applies to its tile.
//
// The thread that owns left row i sees the low-precision scores s~_ij of one
// tile, column by column in increasing j, and keeps
//   * j in the row's band list when s~_ij >= theta_i (running top-k bound),
//   * (i, j) in the threshold candidate list when s~_ij >= tau - m_i,
// so the |A| x |B| score matrix never reaches HBM (the analogue of fusing
// nonzero() of Sec. 3.2 into the product).
#pragma once

#include <cooperative_groups.h>

#include "sj_device.cuh"
#include "sj_internal.h"

namespace sj {

struct RowCtx {
  RowFilter f;
  float *heap;  // k floats (min-heap of the k best s~ of this row and split)
  Cand *band;   // cap entries
  int32_t i;    // global left row
};

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
// All factors are upper bounds, combined with upward rounding.
__device__ __forceinline__ float row_margin(const RowMeta &m, const float *gmaxB, float acc_coef) {
  float t1 = __fmul_ru(m.qerr, gmaxB[0]);
  float t2 = __fmul_ru(m.qnrm, gmaxB[2]);
  float t3 = __fmul_ru(__fmul_ru(acc_coef, m.qnrm), gmaxB[1]);
  return __fadd_ru(__fadd_ru(t1, t2), t3);
}

__device__ __forceinline__ void row_begin(RowCtx &r, const ScoreArgs &a, int64_t row,
                                          int split) {
  r.i = (int32_t)row;
  float m = row_margin(a.metaA[row], a.gmaxB, a.acc_coef);
  r.f.two_m = __fmul_ru(2.f, m);
  r.f.tau_lo = __fsub_rd(a.tau_f, m);
  r.f.cnt = 0;
  r.f.overflow = 0;
  size_t slot = (size_t)row * a.n_splits + split;
  r.heap = a.heaps + slot * a.k;
  r.band = a.band + slot * a.cap;
  if (a.k > 0) {
    for (int t = 0; t < a.k; ++t) r.heap[t] = -INFINITY;
    r.f.theta = -INFINITY;
  } else {
    r.f.theta = INFINITY;
  }
}

__device__ __forceinline__ void row_end(const RowCtx &r, const ScoreArgs &a, int split) {
  if (a.k > 0) a.band_cnt[(size_t)r.i * a.n_splits + split] = r.f.overflow ? -1 : r.f.cnt;
}

__device__ __forceinline__ void row_visit_topk(RowCtx &r, const ScoreArgs &a, float v, int32_t j) {
  if (r.f.overflow == 0) {
    if (r.f.cnt == a.cap) {
      int w = 0;
      for (int t = 0; t < a.cap; ++t) {
        Cand c = r.band[t];
        if (c.v >= r.f.theta) r.band[w++] = c;
      }
      r.f.cnt = w;
      if (w > a.cap - 32) r.f.overflow = 1;
    }
    if (r.f.overflow == 0) r.band[r.f.cnt++] = Cand{v, j};
  }
  if (v > r.heap[0]) {
    heap_replace_min(r.heap, a.k, v);
    r.f.theta = __fsub_rd(r.heap[0], r.f.two_m);
  }
}

__device__ __forceinline__ void row_visit(RowCtx &r, const ScoreArgs &a, float v, int32_t j) {
  if (v >= r.f.theta) row_visit_topk(r, a, v, j);
  if (v >= r.f.tau_lo) push_thr(a, r.i, j, v);
}

}  // namespace sj
