// prepare.cu -- validation and operand packing for the scoring pass.
//
// One warp per row.  Every input row is checked (finite entries,
// | ||x||^2 - 1 | <= 1e-5 with a compensated norm) and rewritten in the
// layout the scoring kernel consumes: a zero-padded copy in FP32 or BF16
// (rounded to nearest-even), plus per-row bounds used by the error margins:
// ||x||, ||x~|| and ||x~ - x||, all rounded up.  Zero padding of rows and
// columns is exact for the products.  This is the analogue of the on-device
// table -> matrix transformation of Sec. 4.2.2 ("data transformation" cost).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "sj_device.cuh"
#include "sj_internal.h"

namespace sj {

namespace {

// Compensated sum of squares across the warp: returns hi + lo (same on all lanes).
__device__ __forceinline__ float warp_sumsq2(float s, float c) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, off);
    float c2 = __shfl_xor_sync(0xffffffffu, c, off);
    float t, q;
    two_sum(s, s2, t, q);
    s = t;
    c = __fadd_rn(__fadd_rn(c, c2), q);
  }
  return __fadd_rn(s, c);
}

__device__ __forceinline__ void acc_sq(float x, float &s, float &c) {
  float p = __fmul_rn(x, x);
  float e = __fmaf_rn(x, x, -p);
  float t, q;
  two_sum(s, p, t, q);
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, e));
}

__device__ __forceinline__ void atomic_max_pos(float *addr, float v) {
  // non-negative floats order like their bit patterns
  atomicMax(reinterpret_cast<unsigned int *>(addr), __float_as_uint(v));
}

// Upper bound on sqrt(x) for a compensated sum of squares x (relative error of
// x far below 2^-40): inflate by 2^-20 and take the square root rounded up.
__device__ __forceinline__ float sqrt_up(float x) {
  return __fsqrt_ru(__fmul_ru(fmaxf(x, 0.f), 1.0f + 0x1p-20f));
}

// Last segment starting at or before packed row p (prow0 ascending).
__device__ __forceinline__ int find_seg(const PackSeg *segs, int n_segs, int64_t p) {
  int lo = 0, hi = n_segs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].prow0 <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int kPrepWarps = 8;

// Four packed elements at dst (aligned to four elements) in one store.
__device__ __forceinline__ void store4(float *dst, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(dst) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(__nv_bfloat16 *dst, __nv_bfloat16 a, __nv_bfloat16 b,
                                       __nv_bfloat16 c, __nv_bfloat16 d) {
  uint2 w;
  w.x = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
  w.y = (uint32_t)__bfloat16_as_ushort(c) | ((uint32_t)__bfloat16_as_ushort(d) << 16);
  *reinterpret_cast<uint2 *>(dst) = w;
}
__device__ __forceinline__ void store4(__nv_fp8_e4m3 *dst, __nv_fp8_e4m3 a, __nv_fp8_e4m3 b,
                                       __nv_fp8_e4m3 c, __nv_fp8_e4m3 d) {
  *reinterpret_cast<uint32_t *>(dst) = (uint32_t)a.__x | ((uint32_t)b.__x << 8) |
                                       ((uint32_t)c.__x << 16) | ((uint32_t)d.__x << 24);
}

// E4M3 scale exponent: the largest e with mx 2^e <= 448 (the largest finite
// E4M3 value, 0.875 2^9), clamped to [-60, 60]; 0 for mx == 0.
__device__ __forceinline__ int e4m3_exponent(float mx) {
  if (!(mx > 0.f) || !isfinite(mx)) return 0;
  int E;
  const float f = frexpf(mx, &E);  // mx = f 2^E, f in [0.5, 1)
  const int e = f <= 0.875f ? 9 - E : 8 - E;
  return e < -60 ? -60 : (e > 60 ? 60 : e);
}

__device__ __forceinline__ float warp_absmax(const float *src, int64_t d) {
  float m = 0.f;
  for (int64_t k = threadIdx.x & 31; k < d; k += 32) {
    const float x = fabsf(src[k]);
    if (x > m) m = x;  // NaN never wins; non-finite rows are flagged by the packing pass
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  return m;
}

// E4M3 packing, first pass: max |x| over each job's B rows (jobs[q].bmax).
__global__ void __launch_bounds__(kPrepWarps * 32)
    bmax_kernel(const PackSeg *segs, int n_segs, JobDev *jobs, int64_t prows, int64_t d) {
  __shared__ int s_seg0;
  __shared__ int s_seg[kPrepWarps];
  __shared__ float s_m[kPrepWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * kPrepWarps;
  if (threadIdx.x == 0) s_seg0 = find_seg(segs, n_segs, row0);
  __syncthreads();
  const int64_t prow = row0 + wib;
  int si = s_seg0;
  while (si + 1 < n_segs && segs[si + 1].prow0 <= prow) ++si;
  float mx = 0.f;
  if (prow < prows) {
    const PackSeg sg = segs[si];
    const int64_t local = prow - sg.prow0;
    if (sg.side != 0 && local < sg.n) mx = warp_absmax(sg.src + local * d, d);
  }
  if (lane == 0) {
    s_seg[wib] = prow < prows ? si : -1;
    s_m[wib] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int cur = -1;
    float v = 0.f;
    for (int w = 0; w <= kPrepWarps; ++w) {
      const int sw = w < kPrepWarps ? s_seg[w] : -1;
      if (sw != cur) {
        if (cur >= 0 && segs[cur].side != 0 && v > 0.f) atomic_max_pos(&jobs[segs[cur].job].bmax, v);
        cur = sw;
        v = 0.f;
      }
      if (w < kPrepWarps) v = fmaxf(v, s_m[w]);
    }
  }
}

// One warp per packed row, kPrepWarps rows per block.  Segments hold at least
// 128 rows, so a block's rows fall in at most two segments: one binary search
// per block, and the B-side maxima are reduced per block before the atomics.
// X3: the hi/lo split, a row of 3d bfloat16 ([hi | hi | lo] for A rows,
// [hi | lo | hi] for B rows; zeros after 3d).
template <typename OutT, bool X3 = false>
__global__ void __launch_bounds__(kPrepWarps * 32)
    prepare_kernel(const PackSeg *segs, int n_segs, JobDev *jobs, int64_t prows, int64_t d,
                   OutT *__restrict__ Xp, int64_t dp, RowMeta *__restrict__ meta,
                   Counters *ctr) {
  __shared__ int s_seg0;
  __shared__ int s_seg[kPrepWarps];
  __shared__ float s_m[kPrepWarps][4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * kPrepWarps;
  if (threadIdx.x == 0) s_seg0 = find_seg(segs, n_segs, row0);
  __syncthreads();
  const int64_t prow = row0 + wib;
  int si = s_seg0;
  while (si + 1 < n_segs && segs[si + 1].prow0 <= prow) ++si;
  float mx[4] = {0.f, 0.f, 0.f, 0.f};
  if (prow < prows) {
    const PackSeg sg = segs[si];
    const int64_t local = prow - sg.prow0;
    OutT *dst = Xp + prow * dp;
    if (local >= sg.n) {
      for (int64_t k = lane; k < dp; k += 32) dst[k] = OutT(0.f);
      if (lane == 0) meta[prow] = RowMeta{0.f, 0.f, 0.f, 0, 0.f};
    } else if constexpr (X3) {
      const float *src = sg.src + local * d;
      float ns = 0.f, nc = 0.f;   // ||x||^2
      float hs = 0.f, hc = 0.f;   // ||hi||^2
      float ls = 0.f, lc = 0.f;   // ||lo||^2
      float es = 0.f, ec = 0.f;   // ||x - hi - lo||^2
      bool bad = false;
      const bool a_side = sg.side == 0;
      for (int64_t k = lane; k < d; k += 32) {
        float x = src[k];
        if (!isfinite(x)) { bad = true; x = 0.f; }
        const OutT hi = OutT(x);
        const float r = __fsub_rn(x, float(hi));  // exact: x minus its rounding
        const OutT lo = OutT(r);
        const float e = __fsub_rn(r, float(lo));  // exact as well
        dst[k] = hi;
        dst[d + k] = a_side ? hi : lo;
        dst[2 * d + k] = a_side ? lo : hi;
        acc_sq(x, ns, nc);
        acc_sq(float(hi), hs, hc);
        acc_sq(float(lo), ls, lc);
        acc_sq(e, es, ec);
      }
      for (int64_t k = 3 * d + lane; k < dp; k += 32) dst[k] = OutT(0.f);
      const bool any_bad = __any_sync(0xffffffffu, bad);
      const float n2 = warp_sumsq2(ns, nc);
      const float h2 = warp_sumsq2(hs, hc);
      const float l2 = warp_sumsq2(ls, lc);
      const float e2 = warp_sumsq2(es, ec);
      if (lane == 0) {
        unsigned flags = 0;
        if (any_bad) flags |= kErrNonFinite;
        else if (!(fabsf(n2 - 1.0f) <= 1e-5f)) flags |= kErrNotUnit;
        if (flags) atomicOr(&ctr->err_flags, flags);
        RowMeta m;
        m.nrm = sqrt_up(n2);
        m.lonrm = l2 > 0.f ? sqrt_up(l2) : 0.f;
        m.qnrm = __fadd_ru(sqrt_up(h2), m.lonrm);
        m.qerr = e2 > 0.f ? sqrt_up(e2) : 0.f;
        m.sexp = 0;
        meta[prow] = m;
        if (sg.side != 0) {
          mx[0] = m.nrm;
          mx[1] = m.qnrm;
          mx[2] = m.qerr;
          mx[3] = m.lonrm;
        }
      }
    } else {
      const float *src = sg.src + local * d;
      constexpr bool kE4M3 = std::is_same<OutT, __nv_fp8_e4m3>::value;
      int e = 0;  // stored value = x 2^e (E4M3), dequantised = stored 2^-e
      if constexpr (kE4M3) {
        if (sg.side == 0) {
          e = e4m3_exponent(warp_absmax(src, d));
        } else {
          e = e4m3_exponent(jobs[sg.job].bmax);
          if (lane == 0) jobs[sg.job].eB = e;  // same value from every B row
        }
      }
      const float up = __int_as_float((127 + e) << 23), down = __int_as_float((127 - e) << 23);
      float ns = 0.f, nc = 0.f;   // ||x||^2
      float qs = 0.f, qc = 0.f;   // ||x~||^2
      float es = 0.f, ec = 0.f;   // ||x~ - x||^2
      bool bad = false;
      // one element of the row: validity, rounding, the three sums of squares
      auto pack1 = [&](float x) -> OutT {
        if (!isfinite(x)) { bad = true; x = 0.f; }
        OutT qv;
        float qf;
        if constexpr (kE4M3) {
          qv = OutT(x * up);  // round to nearest even, saturating
          qf = float(qv) * down;
        } else {
          qv = OutT(x);
          qf = float(qv);
        }
        acc_sq(x, ns, nc);
        acc_sq(qf, qs, qc);
        acc_sq(__fsub_rn(qf, x), es, ec);  // exact difference of x and its rounding
        return qv;
      };
      if ((d & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        // 16-byte loads: lane l takes entries 4l .. 4l+3 of each 128-entry
        // block (a group of four lies wholly inside or outside the row)
        for (int64_t k0 = 0; k0 < dp; k0 += 512) {
          float4 xv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + 128 * u + 4 * lane;
            xv[u] = k < d ? *reinterpret_cast<const float4 *>(src + k)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + 128 * u + 4 * lane;
            if (k >= dp) break;
            const OutT q0 = pack1(xv[u].x), q1 = pack1(xv[u].y);
            const OutT q2 = pack1(xv[u].z), q3 = pack1(xv[u].w);
            store4(dst + k, q0, q1, q2, q3);
          }
        }
      } else {
      for (int64_t k0 = 0; k0 < dp; k0 += 128) {
        float xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t k = k0 + 32 * u + lane;
          xv[u] = k < d ? src[k] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t k = k0 + 32 * u + lane;
          if (k >= dp) break;
          dst[k] = pack1(xv[u]);
        }
      }
      }
      bool any_bad = __any_sync(0xffffffffu, bad);
      float n2 = warp_sumsq2(ns, nc);
      float q2 = warp_sumsq2(qs, qc);
      float e2 = warp_sumsq2(es, ec);
      if (lane == 0) {
        unsigned flags = 0;
        if (any_bad) flags |= kErrNonFinite;
        else if (!(fabsf(n2 - 1.0f) <= 1e-5f)) flags |= kErrNotUnit;
        if (flags) atomicOr(&ctr->err_flags, flags);
        RowMeta m;
        m.nrm = sqrt_up(n2);
        m.qnrm = sqrt_up(q2);
        m.qerr = e2 > 0.f ? sqrt_up(e2) : 0.f;
        m.sexp = e;
        m.lonrm = 0.f;
        meta[prow] = m;
        if (sg.side != 0) {
          mx[0] = m.nrm;
          mx[1] = m.qnrm;
          mx[2] = m.qerr;
        }
      }
    }
  }
  if (lane == 0) {
    s_seg[wib] = prow < prows ? si : -1;
    s_m[wib][0] = mx[0];
    s_m[wib][1] = mx[1];
    s_m[wib][2] = mx[2];
    s_m[wib][3] = mx[3];
  }
  __syncthreads();
  // B-side maxima: one set of atomics per segment present in the block
  if (threadIdx.x < 4) {
    const int c = threadIdx.x;
    int cur = -1;
    float v = 0.f;
    for (int w = 0; w <= kPrepWarps; ++w) {
      const int sw = w < kPrepWarps ? s_seg[w] : -1;
      if (sw != cur) {
        if (cur >= 0 && segs[cur].side != 0 && v > 0.f)
          atomic_max_pos(jobs[segs[cur].job].gmaxB + c, v);
        cur = sw;
        v = 0.f;
      }
      if (w < kPrepWarps) v = fmaxf(v, s_m[w][c]);
    }
  }
}

// One block per 128-row group: which 128-byte k-blocks hold a nonzero byte in
// any of the group's rows (each warp scans 16 rows, 512 bytes per step; the
// four k-blocks of a step are decided by ballots of 8 lanes each).
__global__ void __launch_bounds__(256)
    occupancy_kernel(const unsigned char *Xp, int64_t row_bytes, uint32_t *occ, int words) {
  __shared__ uint32_t s_occ[kOccMaxWords];
  for (int w = threadIdx.x; w < words; w += blockDim.x) s_occ[w] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t g = blockIdx.x;
  for (int r = wib; r < 128; r += 8) {
    const unsigned char *row = Xp + (g * 128 + r) * row_bytes;
    for (int64_t off = 0; off < row_bytes; off += 512) {
      const int64_t o = off + lane * 16;
      bool nz = false;
      if (o < row_bytes) {
        const uint4 v = *reinterpret_cast<const uint4 *>(row + o);
        nz = (v.x | v.y | v.z | v.w) != 0u;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, nz);
      if (lane < 4 && ((bal >> (lane * 8)) & 0xffu)) {
        const int64_t kb = off / 128 + lane;
        atomicOr(&s_occ[kb >> 5], 1u << (kb & 31));
      }
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < words; w += blockDim.x) occ[g * words + w] = s_occ[w];
}

}  // namespace

cudaError_t launch_occupancy(const void *Xp, int64_t prows, int64_t row_bytes, uint32_t *occ,
                             int words, cudaStream_t st) {
  if (prows == 0) return cudaSuccess;
  if (words > kOccMaxWords || prows % 128 != 0 || row_bytes % 128 != 0)
    return cudaErrorInvalidValue;
  occupancy_kernel<<<(unsigned)(prows / 128), 256, 0, st>>>(
      static_cast<const unsigned char *>(Xp), row_bytes, occ, words);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const PackSeg *segs, int n_segs, JobDev *jobs, int64_t prows,
                           int64_t d, PackFormat fmt, void *Xp, int64_t dp, RowMeta *meta,
                           Counters *ctr, cudaStream_t st) {
  if (prows == 0 || n_segs == 0) return cudaSuccess;
  dim3 grid((unsigned)((prows + kPrepWarps - 1) / kPrepWarps)), block(32 * kPrepWarps);
  switch (fmt) {
    case PackFormat::kF32:
      prepare_kernel<float><<<grid, block, 0, st>>>(segs, n_segs, jobs, prows, d,
                                                    static_cast<float *>(Xp), dp, meta, ctr);
      break;
    case PackFormat::kBF16:
      prepare_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(
          segs, n_segs, jobs, prows, d, static_cast<__nv_bfloat16 *>(Xp), dp, meta, ctr);
      break;
    case PackFormat::kBF16X3:
      prepare_kernel<__nv_bfloat16, true><<<grid, block, 0, st>>>(
          segs, n_segs, jobs, prows, d, static_cast<__nv_bfloat16 *>(Xp), dp, meta, ctr);
      break;
    case PackFormat::kFP8:
      bmax_kernel<<<grid, block, 0, st>>>(segs, n_segs, jobs, prows, d);
      prepare_kernel<__nv_fp8_e4m3><<<grid, block, 0, st>>>(
          segs, n_segs, jobs, prows, d, static_cast<__nv_fp8_e4m3 *>(Xp), dp, meta, ctr);
      break;
  }
  return cudaGetLastError();
}

}  // namespace sj
