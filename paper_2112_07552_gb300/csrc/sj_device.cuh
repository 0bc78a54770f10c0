// sj_device.cuh -- device-side building blocks shared by the join kernels.
//
//  * Dot2: compensated FP32 dot product (Ogita, Rump & Oishi, "Accurate sum
//    and dot product", SIAM J. Sci. Comput. 26(6), 2005, Algorithm 5.3),
//    split over the 32 lanes of a warp and combined with error-free
//    transformations (TwoProduct via fmaf, Knuth's TwoSum).
//  * An exact fixed-point accumulator for dot products of float32 rows whose
//    entries are below 2 in magnitude (Kulisch's long accumulator, restricted
//    to the exponent range such rows can produce), its comparison, and its
//    correctly rounded conversion to float32.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sj {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Fixed-point scale of the 64-bit keys used to order Dot2 results: a key K
// stands for K * 2^-60.  |s| < 2 keeps |K| < 2^61.
constexpr int kKeyShift = 60;

// Exact accumulator: 10 digits of 32 bits, digit t has weight 2^(32 t - 298).
// For float32 x with |x| < 2, x = m 2^e with m < 2^24 and -149 <= e <= -23,
// so a product lies on the grid 2^-298 and below 2^2, and any dot product of
// unit-norm rows (sum |p| <= 1 + 1e-5) lies far inside the 2^21 top range.
constexpr int kExDigits = 10;
constexpr int kExLsb = -298;

struct Exact {
  int32_t top;      // digit 9, signed (carries the sign of the value)
  uint32_t d[9];    // digits 0..8, each in [0, 2^32)
};

// Candidate in a band list: low-precision score and right index.
struct Cand {
  float v;
  int32_t j;
};

// Threshold candidate (left row, right row, low-precision score).
struct ThrCand {
  int32_t i;
  int32_t j;
  float v;
  int32_t pad;
};

// Device-side counters and error flags of one call.
struct Counters {
  unsigned long long thr_count;     // threshold candidates produced
  unsigned long long n_candidates;  // top-k band entries kept at finalize
  unsigned long long n_rescored;    // Dot2 evaluations
  unsigned long long n_exact;       // exact evaluations
  unsigned long long n_pairs;       // threshold pairs accepted
  unsigned int err_flags;           // kErr* bits
  unsigned int overflow_rows;       // rows needing the fallback pass
  unsigned int max_err_bits;        // max |s~ - s| as float bits (>= 0)
  unsigned int tier2_rows;          // rows for the second finalisation tier
  unsigned int redo_rows;           // rescan lists cut off at their capacity
  unsigned int redo_cap;            // capacity they need
  unsigned int big_rows;            // rescan lists for the global-memory ranker
  unsigned int defer_rows;          // rows the warp finaliser hands to the block tiers
  unsigned int max_margin_bits;     // max proven margin m_i over finalised top-k rows
                                    // (float bits, >= 0)
};

constexpr unsigned kErrNonFinite = 1u;
constexpr unsigned kErrNotUnit = 2u;
constexpr unsigned kErrTimeout = 4u;
constexpr unsigned kErrInternal = 8u;

// Per-row metadata written by the prepare kernels.
struct RowMeta {
  float nrm;    // upper bound on ||x|| (float32 row)
  float qnrm;   // upper bound on ||x~|| (the row the scoring pass sees, dequantised;
                // hi/lo split: on ||hi|| + ||lo||)
  float qerr;   // upper bound on ||x~ - x|| (hi/lo split: x~ = hi + lo)
  int32_t sexp; // power-of-two scale exponent (FP8), else 0
  float lonrm;  // hi/lo split: upper bound on ||lo||, else 0
};

// ---------------------------------------------------------------------------
// Error-free transformations (no contraction: explicit _rn intrinsics).

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Warp-cooperative Dot2 over d entries (lane l takes k = l, l+32, ...).
// Returns the unevaluated sum hi + lo, identical on every lane.  a may point
// to shared or global memory.
__device__ __forceinline__ void dot2_step(float x, float y, float &s, float &c) {
  float p = __fmul_rn(x, y);
  float e = __fmaf_rn(x, y, -p);
  float t, q;
  two_sum(s, p, t, q);
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, e));
}

__device__ __forceinline__ void dot2_warp(const float *a, const float *b, int64_t d,
                                          float &hi, float &lo) {
  const int lane = threadIdx.x & 31;
  float s = 0.f, c = 0.f;
  int64_t k = lane;
  // four independent gathers in flight per lane; the arithmetic stays in
  // index order k, k+32, k+64, ... of this lane's chain
  for (; k + 96 < d; k += 128) {
    float x0 = a[k], x1 = a[k + 32], x2 = a[k + 64], x3 = a[k + 96];
    float y0 = __ldg(b + k), y1 = __ldg(b + k + 32), y2 = __ldg(b + k + 64), y3 = __ldg(b + k + 96);
    dot2_step(x0, y0, s, c);
    dot2_step(x1, y1, s, c);
    dot2_step(x2, y2, s, c);
    dot2_step(x3, y3, s, c);
  }
  for (; k < d; k += 32) dot2_step(a[k], __ldg(b + k), s, c);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, off);
    float c2 = __shfl_xor_sync(0xffffffffu, c, off);
    float t, q;
    two_sum(s, s2, t, q);
    s = t;
    c = __fadd_rn(__fadd_rn(c, c2), q);
  }
  hi = s;
  lo = c;
}

// NC Dot2 evaluations of one row a against NC rows b[q], by one warp.  With
// d a multiple of 128 and every row 16-byte aligned, lane l takes the
// entries 4l .. 4l+3 of each 128-entry block through one 16-byte load per
// row, a shared by the NC evaluations; otherwise the lane chains of
// dot2_warp_n.  Either way each lane chain holds at most ceil(d/32) products
// summed in index order and the combination tree is that of dot2_warp, so
// the error bound of dot2_warp holds (the values may differ from it in the
// last bits, within that bound).
template <int NC>
__device__ __forceinline__ void dot2_warp_sa(const float *a, const float *const (&b)[NC],
                                             int64_t d, float (&hi)[NC], float (&lo)[NC]) {
  const int lane = threadIdx.x & 31;
  float s[NC], c[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) s[q] = c[q] = 0.f;
  uintptr_t al = reinterpret_cast<uintptr_t>(a);
#pragma unroll
  for (int q = 0; q < NC; ++q) al |= reinterpret_cast<uintptr_t>(b[q]);
  if ((d & 127) == 0 && (al & 15) == 0) {
#pragma unroll 1
    for (int64_t k = 4 * lane; k < d; k += 128) {
      const float4 x = *reinterpret_cast<const float4 *>(a + k);
      float4 y[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) y[q] = __ldg(reinterpret_cast<const float4 *>(b[q] + k));
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        dot2_step(x.x, y[q].x, s[q], c[q]);
        dot2_step(x.y, y[q].y, s[q], c[q]);
        dot2_step(x.z, y[q].z, s[q], c[q]);
        dot2_step(x.w, y[q].w, s[q], c[q]);
      }
    }
  } else {
    int64_t k = lane;
    for (; k + 96 < d; k += 128) {
      float x[4], y[NC][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = a[k + 32 * u];
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) y[q][u] = __ldg(b[q] + k + 32 * u);
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) dot2_step(x[u], y[q][u], s[q], c[q]);
    }
    for (; k < d; k += 32) {
      const float x = a[k];
#pragma unroll
      for (int q = 0; q < NC; ++q) dot2_step(x, __ldg(b[q] + k), s[q], c[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      float s2 = __shfl_xor_sync(0xffffffffu, s[q], off);
      float c2 = __shfl_xor_sync(0xffffffffu, c[q], off);
      float t, e;
      two_sum(s[q], s2, t, e);
      s[q] = t;
      c[q] = __fadd_rn(__fadd_rn(c[q], c2), e);
    }
    hi[q] = s[q];
    lo[q] = c[q];
  }
}

// NC independent Dot2 evaluations by one warp, interleaved so that 4 * NC
// gathers per lane are in flight.  Each evaluation has exactly the lane chains
// and combination tree of dot2_warp (same values, same error bound).
template <int NC>
__device__ __forceinline__ void dot2_warp_n(const float *const (&a)[NC],
                                            const float *const (&b)[NC], int64_t d,
                                            float (&hi)[NC], float (&lo)[NC]) {
  const int lane = threadIdx.x & 31;
  float s[NC], c[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) s[q] = c[q] = 0.f;
  int64_t k = lane;
  for (; k + 96 < d; k += 128) {
    float x[NC][4], y[NC][4];
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[q][u] = a[q][k + 32 * u];
        y[q][u] = __ldg(b[q] + k + 32 * u);
      }
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) dot2_step(x[q][u], y[q][u], s[q], c[q]);
  }
  for (; k < d; k += 32) {
#pragma unroll
    for (int q = 0; q < NC; ++q) dot2_step(a[q][k], __ldg(b[q] + k), s[q], c[q]);
  }
#pragma unroll
  for (int q = 0; q < NC; ++q) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      float s2 = __shfl_xor_sync(0xffffffffu, s[q], off);
      float c2 = __shfl_xor_sync(0xffffffffu, c[q], off);
      float t, e;
      two_sum(s[q], s2, t, e);
      s[q] = t;
      c[q] = __fadd_rn(__fadd_rn(c[q], c2), e);
    }
    hi[q] = s[q];
    lo[q] = c[q];
  }
}

// Key of an unevaluated sum hi + lo: round(hi 2^60) + round(lo 2^60), within
// 1 unit of (hi + lo) 2^60.
__device__ __forceinline__ long long dot2_key(float hi, float lo) {
  return __float2ll_rn(__fmul_rn(hi, 0x1p60f)) + __float2ll_rn(__fmul_rn(lo, 0x1p60f));
}

// Key half-width of a Dot2 result: coef bounds |hi + lo - s| / (||a|| ||b||)
// in key units (host-computed, rounded up); +3 covers the two key roundings
// and the underflow allowance.
__device__ __forceinline__ long long dot2_halfwidth(float coef_key, float nrm_a, float nrm_b) {
  float w = __fmul_ru(__fmul_ru(coef_key, nrm_a), nrm_b);
  return (long long)ceilf(w) + 3;
}

// RN_fp32 of a value known to lie in [lo, hi] key units; returns false when
// the two ends round differently (the caller then evaluates exactly).
__device__ __forceinline__ bool key_interval_round(long long lo, long long hi, float &out) {
  float a = __fmul_rn(__ll2float_rn(lo), 0x1p-60f);
  float b = __fmul_rn(__ll2float_rn(hi), 0x1p-60f);
  // Results in the subnormal range would make the scaling inexact.
  if (a != b || fabsf(a) < 0x1p-120f) return false;
  out = a;
  return true;
}

// ---------------------------------------------------------------------------
// Exact accumulation.

// Warp-cooperative exact <a, b>; the result is returned on every lane.
// Requires |a_k|, |b_k| < 2 (guaranteed for rows that passed validation).
__device__ __forceinline__ Exact exact_dot_warp(const float *a, const float *b, int64_t d) {
  const int lane = threadIdx.x & 31;
  long long acc[kExDigits];
#pragma unroll
  for (int t = 0; t < kExDigits; ++t) acc[t] = 0;
  for (int64_t k = lane; k < d; k += 32) {
    uint32_t xa = __float_as_uint(a[k]);
    uint32_t xb = __float_as_uint(__ldg(b + k));
    uint32_t ea = (xa >> 23) & 0xffu, eb = (xb >> 23) & 0xffu;
    uint32_t ma = xa & 0x7fffffu, mb = xb & 0x7fffffu;
    if ((ea == 0 && ma == 0) || (eb == 0 && mb == 0)) continue;
    // value = m * 2^(e - 150) for normals (implicit bit), m * 2^-149 for subnormals
    if (ea) { ma |= 0x800000u; } else { ea = 1; }
    if (eb) { mb |= 0x800000u; } else { eb = 1; }
    unsigned long long P = (unsigned long long)ma * (unsigned long long)mb;  // < 2^48
    int pos = (int)ea + (int)eb - 300 - kExLsb;  // product exponent - LSB, >= 0 for |x| < 2
    int t0 = pos >> 5, r = pos & 31;
    unsigned long long lo64 = P << r;                       // bits 0..63 of P*2^r
    unsigned long long hi64 = r ? (P >> (64 - r)) : 0ull;   // bits 64..
    long long p0 = (long long)(lo64 & 0xffffffffull);
    long long p1 = (long long)(lo64 >> 32);
    long long p2 = (long long)hi64;
    bool neg = ((xa ^ xb) >> 31) != 0;
    if (neg) { p0 = -p0; p1 = -p1; p2 = -p2; }
#pragma unroll
    for (int t = 0; t < kExDigits; ++t) {
      long long add = (t == t0) ? p0 : (t == t0 + 1) ? p1 : (t == t0 + 2) ? p2 : 0ll;
      acc[t] += add;
    }
  }
#pragma unroll
  for (int t = 0; t < kExDigits; ++t) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], off);
  }
  // carry propagation: digits 0..8 into [0, 2^32), signed top digit
#pragma unroll
  for (int t = 0; t < kExDigits - 1; ++t) {
    long long c = acc[t] >> 32;  // arithmetic shift = floor division
    acc[t] -= c * 4294967296ll;
    acc[t + 1] += c;
  }
  Exact x;
  x.top = (int32_t)acc[kExDigits - 1];
#pragma unroll
  for (int t = 0; t < 9; ++t) x.d[t] = (uint32_t)acc[t];
  return x;
}

// sign(a - b) of two canonical exact values.
__host__ __device__ __forceinline__ int exact_cmp(const Exact &a, const Exact &b) {
  if (a.top != b.top) return a.top < b.top ? -1 : 1;
  for (int t = 8; t >= 0; --t)
    if (a.d[t] != b.d[t]) return a.d[t] < b.d[t] ? -1 : 1;
  return 0;
}

// Round an exact value to the nearest float32 (ties to even).
__device__ __forceinline__ float exact_to_float(const Exact &x) {
  uint32_t m[10];
  bool neg = x.top < 0;
#pragma unroll
  for (int t = 0; t < 9; ++t) m[t] = x.d[t];
  m[9] = (uint32_t)x.top;
  if (neg) {  // two's complement negation over 320 bits
    unsigned long long carry = 1;
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      unsigned long long v = (unsigned long long)(~m[t]) + carry;
      m[t] = (uint32_t)v;
      carry = v >> 32;
    }
  }
  int T = -1;  // top set bit
  for (int t = 9; t >= 0; --t)
    if (m[t]) { T = 32 * t + 31 - __clz(m[t]); break; }
  if (T < 0) return 0.f;
  // quantum bit: 24 significant bits, or 2^-149 (bit 149) in the subnormal range
  int qb = T - 23;
  if (qb < 149) qb = 149;
  auto bit = [&](int i) -> uint32_t { return (i < 0 || i >= 320) ? 0u : (m[i >> 5] >> (i & 31)) & 1u; };
  uint32_t M = 0;
  for (int i = T; i >= qb; --i) M = (M << 1) | bit(i);
  uint32_t rb = bit(qb - 1);
  uint32_t sticky = 0;
  int below = qb - 1;  // bits [0, below) feed the sticky bit
  for (int t = 0; t < 10 && 32 * t < below; ++t) {
    int hi = below - 32 * t;  // number of bits of digit t below the round bit
    uint32_t mask = hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u);
    sticky |= m[t] & mask;
  }
  if (rb && (sticky || (M & 1u))) M += 1;
  uint32_t bits;
  if (qb == 149 && M <= 0x800000u) {
    bits = M;  // subnormal (or the smallest normal after rounding up)
  } else {
    int e = qb - 298 + 23;  // exponent of the leading bit of M when M in [2^23, 2^24)
    if (M == 0x1000000u) { M = 0x800000u; e += 1; }
    bits = ((uint32_t)(e + 127) << 23) | (M & 0x7fffffu);
  }
  if (neg) bits |= 0x80000000u;
  return __uint_as_float(bits);
}

}  // namespace sj
