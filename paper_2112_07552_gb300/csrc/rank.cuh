// rank.cuh -- block-level exact ranking of one left row's candidates.
//
// Given candidates with Dot2 key intervals [L, U] (units of 2^-60) that
// contain the exact scores: sort by U desc, sweep into groups of chained
// overlapping intervals (groups are totally ordered), evaluate members of
// multi-member groups within the first k positions exactly, order those by
// (exact desc, j asc), and emit k (index, float32 score) pairs.
#pragma once

#include "sj_device.cuh"

namespace sj {
namespace {

// Candidate arrays (shared memory in the normal path, global in the fallback).
struct CandArrays {
  long long *U, *L;
  int32_t *j;
  float *v;        // low-precision score (NaN when unknown)
  int32_t *perm;   // sorted order (candidate ids), length n_pad
  int32_t *perm2;  // final order (sorted positions), length n_pad
  int32_t *grp;    // group id per sorted position
  uint8_t *flag;   // per sorted position: 1 = exact computed
  float *sc;       // score per sorted position
  Exact *ex;       // exact value per sorted position
};

__device__ __forceinline__ int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// Block-wide bitonic sort of idx[0, n_pad) (entries >= 0 are items, -1 pads
// that sort last) with before(x, y) = "x goes first".
template <typename Before>
__device__ void block_bitonic(int32_t *idx, int n_pad, Before before) {
  for (int size = 2; size <= n_pad; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (n_pad >> 1); t += blockDim.x) {
        int lo = 2 * stride * (t / stride) + (t % stride);
        int hi = lo + stride;
        bool asc = (lo & size) == 0;
        int32_t x = idx[lo], y = idx[hi];
        bool y_first = (x < 0) ? (y >= 0) : (y >= 0 && before(y, x));
        bool x_first = (y < 0) ? (x >= 0) : (x >= 0 && before(x, y));
        bool sw = asc ? y_first : x_first;
        if (sw) {
          idx[lo] = y;
          idx[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

// Steps 3-4 above on n candidates whose U, L, j (and v) are filled in.
// Writes k outputs.  a_row: the left row (shared or global memory).
__device__ void rank_and_emit(CandArrays c, int n, int k, const float *a_row, const float *B,
                              int64_t d, int64_t *out_idx, float *out_score, Counters *ctr) {
  __shared__ int s_n_need;
  __shared__ unsigned long long s_n_exact;
  const int n_pad = next_pow2(n > 0 ? n : 1);
  for (int t = threadIdx.x; t < n_pad; t += blockDim.x) c.perm[t] = t < n ? t : -1;
  if (threadIdx.x == 0) s_n_exact = 0;
  __syncthreads();
  block_bitonic(c.perm, n_pad, [&](int32_t x, int32_t y) {
    return c.U[x] > c.U[y] || (c.U[x] == c.U[y] && c.j[x] < c.j[y]);
  });
  // group sweep (sequential; n <= a few thousand in practice)
  if (threadIdx.x == 0) {
    int g = -1;
    long long Lmin = 0;
    int n_need = n;
    for (int p = 0; p < n; ++p) {
      int32_t x = c.perm[p];
      if (g < 0 || c.U[x] < Lmin) {
        if (p >= k) { n_need = p; break; }
        ++g;
        Lmin = c.L[x];
      } else if (c.L[x] < Lmin) {
        Lmin = c.L[x];
      }
      c.grp[p] = g;
    }
    s_n_need = n_need;
  }
  __syncthreads();
  const int n_need = s_n_need;
  // which positions need the exact value
  for (int p = threadIdx.x; p < n_need; p += blockDim.x) {
    bool multi = (p > 0 && c.grp[p - 1] == c.grp[p]) || (p + 1 < n_need && c.grp[p + 1] == c.grp[p]);
    int32_t x = c.perm[p];
    float s = 0.f;
    bool need = multi;
    if (!multi && p < k) need = !key_interval_round(c.L[x], c.U[x], s);
    c.flag[p] = need ? 1 : 0;
    c.sc[p] = s;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < n_need; p += nwarps) {
    if (!c.flag[p]) continue;
    int32_t x = c.perm[p];
    Exact e = exact_dot_warp(a_row, B + (int64_t)c.j[x] * d, d);
    if (lane == 0) {
      c.ex[p] = e;
      c.sc[p] = exact_to_float(e);
      atomicAdd(&s_n_exact, 1ull);
    }
  }
  __syncthreads();
  const int n2_pad = next_pow2(n_need > 0 ? n_need : 1);
  for (int t = threadIdx.x; t < n2_pad; t += blockDim.x) c.perm2[t] = t < n_need ? t : -1;
  __syncthreads();
  block_bitonic(c.perm2, n2_pad, [&](int32_t p, int32_t q) {
    if (c.grp[p] != c.grp[q]) return c.grp[p] < c.grp[q];
    int r = exact_cmp(c.ex[p], c.ex[q]);  // same multi-member group: both exact
    if (r != 0) return r > 0;
    return c.j[c.perm[p]] < c.j[c.perm[q]];
  });
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    if (r < n_need && r < n) {
      int32_t p = c.perm2[r];
      out_idx[r] = c.j[c.perm[p]];
      out_score[r] = c.sc[p];
    } else {
      out_idx[r] = -1;
      out_score[r] = -INFINITY;
    }
  }
  if (threadIdx.x == 0 && s_n_exact) atomicAdd(&ctr->n_exact, s_n_exact);
  __syncthreads();
}

}  // namespace
}  // namespace sj
