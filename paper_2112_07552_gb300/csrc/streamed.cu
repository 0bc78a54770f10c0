// streamed.cu -- joins whose right table stays in host memory, streamed
// through the device in row chunks (the paper's MSplitGEMM-style pipelined
// blocking for inputs larger than device memory, Sec. 4.3).
//
// B (host memory) is registered as mapped, page-locked memory and cut into
// chunks of rows.  Chunk c + 1 is copied to a device staging buffer on a
// second stream while chunk c is joined with the library's pipeline on the
// handle's stream, so transfers overlap the joins.  Each chunk's results are
// exact, and so are their unions:
//   * threshold: the pairs of the chunks, column indices offset by the chunk
//     start, merged by row in chunk order (each chunk's pairs are sorted by
//     (i, j) and the chunks' columns increase);
//   * top-k: row i's global top-k lies in the union of the chunks' top-k
//     lists.  A warp per row merges them by (float32 score desc, column asc),
//     which is exact wherever no two chunks meet with equal float32 scores
//     (each chunk's list is in exact order and rounding is monotone); a row
//     where they do is ranked by the same exact ranker as the fallback path
//     (Dot2 key intervals, then the fixed-point accumulator), reading those B
//     rows through the mapped host pointer (NVLink-C2C on GB300).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sj.h"
#include "rank.cuh"
#include "sj_device.cuh"
#include "sj_internal.h"

namespace sj {
namespace {

sj_status st_fail(cudaError_t e, const char *what, int line) {
  record_cuda_error(e, what, "streamed.cu", line);
  return e == cudaErrorMemoryAllocation ? SJ_ERR_OOM : SJ_ERR_CUDA;
}
#define ST_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return st_fail(e__, #call, __LINE__); \
  } while (0)

struct DMem {
  void *p = nullptr;
  ~DMem() {
    if (p) cudaFree(p);
  }
};

// B registered as mapped page-locked memory for the call (unless the caller
// pinned it already), and the device address of the mapping.
struct MappedB {
  const float *host = nullptr;
  const float *dev = nullptr;
  bool registered = false;
  ~MappedB() {
    if (registered) cudaHostUnregister(const_cast<float *>(host));
  }
  cudaError_t map(const float *B, size_t bytes) {
    host = B;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, B);
    if (e != cudaSuccess || at.type == cudaMemoryTypeUnregistered) {
      cudaGetLastError();
      e = cudaHostRegister(const_cast<float *>(B), bytes, cudaHostRegisterMapped);
      if (e != cudaSuccess) return e;
      registered = true;
    }
    void *d = nullptr;
    e = cudaHostGetDevicePointer(&d, const_cast<float *>(B), 0);
    dev = static_cast<const float *>(d);
    return e;
  }
};

__device__ __forceinline__ float warp_norm_up(const float *x, int64_t d) {
  float s = 0.f, c = 0.f;
  for (int64_t k = threadIdx.x & 31; k < d; k += 32) dot2_step(x[k], x[k], s, c);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, off);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, off);
    float t, q;
    two_sum(s, s2, t, q);
    s = t;
    c = __fadd_rn(__fadd_rn(c, c2), q);
  }
  return __fsqrt_ru(__fmul_ru(fmaxf(__fadd_rn(s, c), 0.f), 1.0f + 0x1p-20f));
}

constexpr int kMergeThreads = 256;

// Per-block candidate storage of the merge (global scratch): n_pad slots.
__host__ __device__ constexpr size_t merge_slot_bytes(int n_pad) {
  return ((size_t)n_pad * (8 + 8 + sizeof(Exact) + 6 * 4 + 1) + 511) / 256 * 256;
}

// Fast merge, a warp per row (at most 32 chunks, one per lane): each chunk's
// list is already in exact order with exact float32 scores, and float32
// rounding is monotone, so a k-way merge by (float32 score desc, column asc)
// is exact -- except where equal float32 scores of different chunks meet,
// whose exact order is unknown.  A row with such a meeting among its first
// k + 1 merged entries goes to `slow` (the exact ranker); the others are
// written out here, without reading B.
__global__ void __launch_bounds__(256)
    merge_fast_kernel(int64_t nA, int k, int n_chunks, const int64_t *chunk0,
                      const int64_t *cidx, const float *csc, int64_t *out_idx,
                      float *out_score, int *slow, unsigned *n_slow) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < nA; i += nw) {
    const int64_t *li = cidx + ((int64_t)lane * nA + i) * k;
    const float *ls = csc + ((int64_t)lane * nA + i) * k;
    int pos = 0;
    // the lane's head as an order key: larger score first, then lower column
    auto head = [&](float &sc, int64_t &j) {
      sc = -INFINITY;
      j = INT64_MAX;
      if (lane < n_chunks && pos < k) {
        const int64_t jj = li[pos];
        if (jj >= 0) {
          sc = ls[pos];
          j = jj + chunk0[lane];
        }
      }
    };
    float prev_s = 0.f;
    int prev_c = -1;
    bool need_exact = false;
    for (int r = 0; r <= k && !need_exact; ++r) {
      float sc;
      int64_t j;
      head(sc, j);
      // warp arg-best: (sc desc, j asc)
      float bs = sc;
      int64_t bj = j;
      int bl = lane;
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, bs, off);
        const int64_t oj = __shfl_xor_sync(0xffffffffu, bj, off);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
        if (os > bs || (os == bs && oj < bj)) {
          bs = os;
          bj = oj;
          bl = ol;
        }
      }
      const bool valid = bs != -INFINITY;
      if (valid && r > 0 && prev_c >= 0 && bs == prev_s && bl != prev_c) need_exact = true;
      if (r < k && lane == 0) {
        out_idx[i * k + r] = valid ? bj : -1;
        out_score[i * k + r] = valid ? bs : -INFINITY;
      }
      if (lane == bl && valid) ++pos;
      prev_s = bs;
      prev_c = valid ? bl : -1;
    }
    if (need_exact && lane == 0) slow[atomicAdd(n_slow, 1u)] = (int)i;
  }
}

// Exact merge of the listed rows: the chunks' top-k lists (columns offset by
// the chunk starts) ranked into the global top-k.
__global__ void __launch_bounds__(kMergeThreads)
    merge_topk_kernel(const int *rows, const unsigned *n_rows, const float *A, const float *Bm,
                      int64_t nA, int64_t d, int k, int n_chunks, const int64_t *chunk0,
                      const int64_t *cidx, const float *csc, float coef_key, int64_t *out_idx,
                      float *out_score, unsigned char *scratch, size_t slot_bytes,
                      Counters *ctr) {
  const int n_max = k * n_chunks;
  const int n_pad = next_pow2(n_max > 0 ? n_max : 1);
  unsigned char *base = scratch + (size_t)blockIdx.x * slot_bytes;
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
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
  __shared__ int s_n;
  __shared__ float s_nrm_a;
  const unsigned nr = *n_rows;
  for (unsigned r = blockIdx.x; r < nr; r += gridDim.x) {
    const int64_t i = rows[r];
    const float *a = A + i * d;
    if (threadIdx.x == 0) {
      // compact the chunks' (valid) entries in chunk order
      int n = 0;
      for (int ch = 0; ch < n_chunks; ++ch)
        for (int t = 0; t < k; ++t) {
          const int64_t jj = cidx[((int64_t)ch * nA + i) * k + t];
          if (jj < 0) continue;
          c.j[n] = (int32_t)(jj + chunk0[ch]);
          c.v[n] = csc[((int64_t)ch * nA + i) * k + t];
          ++n;
        }
      s_n = n;
    }
    if (warp == 0) {
      const float na = warp_norm_up(a, d);
      if (lane == 0) s_nrm_a = na;
    }
    __syncthreads();
    const int n = s_n;
    const float nrm_a = s_nrm_a;
    for (int p = warp; p < n; p += nwarps) {
      const float *b = Bm + (int64_t)c.j[p] * d;
      float hi, lo;
      dot2_warp(a, b, d, hi, lo);
      const float nrm_b = warp_norm_up(b, d);
      if (lane == 0) {
        const long long K = dot2_key(hi, lo);
        const long long D = dot2_halfwidth(coef_key, nrm_a, nrm_b);
        c.U[p] = K + D;
        c.L[p] = K - D;
      }
    }
    __syncthreads();
    rank_and_emit(c, n, k, a, Bm, d, out_idx + i * k, out_score + i * k, ctr);
    __syncthreads();
  }
}

float dot2_coef_key_of(int64_t d) {
  const double u = 0x1p-24;
  const double n = (double)((d + 31) / 32) + 1.0;
  const double g = n * u / (1.0 - n * u);
  const double coef = 2.0 * (g * g + 10.0 * u * (g + 5.0 * u)) * (1.0 + 1e-6) * 0x1p60;
  float f = (float)coef;
  if ((double)f < coef) f = nextafterf(f, INFINITY);
  return f;
}

int where_dev(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeManaged) return 1;
  if (at.type == cudaMemoryTypeDevice) return at.device == dev ? 1 : -1;
  return 0;
}

// Shared set-up: A on the device (staged once when given in host memory), B
// mapped, the chunk plan, the staging buffers and the copy stream.
struct Stream2 {
  cudaStream_t s = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~Stream2() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (s) cudaStreamDestroy(s);
  }
};

struct StreamPlan {
  const float *Adev = nullptr;
  DMem a_stage, stage[2];
  MappedB mb;
  Stream2 cs;
  int64_t rows = 0;  // rows per chunk
  int n_chunks = 0;
};

sj_status stream_setup(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                       int64_t chunk_rows, StreamPlan &sp) {
  const int dev = handle_device(h);
  const int64_t d = handle_config(h)->d;
  cudaStream_t stm = static_cast<cudaStream_t>(handle_stream(h));
  ST_CUDA(cudaSetDevice(dev));
  const int wa = where_dev(A, dev), wb = where_dev(B, dev);
  if (wa < 0 || wb != 0) return SJ_ERR_INVALID_ARG;  // B must be host memory
  if (wa == 1) {
    sp.Adev = A;
  } else {
    ST_CUDA(cudaMalloc(&sp.a_stage.p, (size_t)nA * d * 4));
    ST_CUDA(cudaMemcpyAsync(sp.a_stage.p, A, (size_t)nA * d * 4, cudaMemcpyHostToDevice, stm));
    sp.Adev = static_cast<const float *>(sp.a_stage.p);
  }
  ST_CUDA(sp.mb.map(B, (size_t)nB * d * 4));
  sp.rows = std::min<int64_t>(nB, chunk_rows > 0 ? chunk_rows : (int64_t)1 << 20);
  sp.n_chunks = (int)((nB + sp.rows - 1) / sp.rows);
  for (int t = 0; t < 2 && t < sp.n_chunks; ++t)
    ST_CUDA(cudaMalloc(&sp.stage[t].p, (size_t)sp.rows * d * 4));
  ST_CUDA(cudaStreamCreateWithFlags(&sp.cs.s, cudaStreamNonBlocking));
  for (cudaEvent_t &e : sp.cs.ev) ST_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return SJ_OK;
}

// Copy chunk c of B into staging buffer c % 2 on the copy stream.
sj_status stage_chunk(const StreamPlan &sp, int64_t nB, int64_t d, int c) {
  const int64_t c0 = (int64_t)c * sp.rows, nc = std::min(sp.rows, nB - c0);
  ST_CUDA(cudaMemcpyAsync(sp.stage[c & 1].p, sp.mb.host + c0 * d, (size_t)nc * d * 4,
                          cudaMemcpyHostToDevice, sp.cs.s));
  ST_CUDA(cudaEventRecord(sp.cs.ev[c & 1], sp.cs.s));
  return SJ_OK;
}

void add_chunk_stats(sj_stats *acc, const sj_stats &one) {
  acc->ms_prepare += one.ms_prepare;
  acc->ms_score += one.ms_score;
  acc->ms_select += one.ms_select;
  acc->n_candidates += one.n_candidates;
  acc->n_rescored += one.n_rescored;
  acc->n_exact += one.n_exact;
  acc->n_overflow_rows += one.n_overflow_rows;
  acc->n_pairs += one.n_pairs;
  acc->n_launches += one.n_launches;
  acc->padded_pair_scores += one.padded_pair_scores;
  acc->margin_max = std::max(acc->margin_max, one.margin_max);
  acc->max_abs_err_lowprec = std::max(acc->max_abs_err_lowprec, one.max_abs_err_lowprec);
}

}  // namespace
}  // namespace sj

using namespace sj;

extern "C" sj_status sj_topk_streamed(sj_handle *h, const float *A, int64_t nA, const float *B,
                                      int64_t nB, int32_t k, int64_t chunk_rows,
                                      int64_t *out_idx, float *out_score, sj_stats *st) {
  if (!h || !A || !B || nA < 1 || nB < 1 || k < 1 || k > 1024 || !out_idx || !out_score ||
      chunk_rows < 0)
    return SJ_ERR_INVALID_ARG;
  const int dev = handle_device(h);
  const int64_t d = handle_config(h)->d;
  if (where_dev(out_idx, dev) != 1 || where_dev(out_score, dev) != 1) return SJ_ERR_INVALID_ARG;
  cudaStream_t stm = static_cast<cudaStream_t>(handle_stream(h));
  sj_stats acc{};
  StreamPlan sp;
  sj_status s = stream_setup(h, A, nA, B, nB, chunk_rows, sp);
  if (s != SJ_OK) return s;
  const int nch = sp.n_chunks;
  DMem cidx, csc, c0d, scratch, ctr;
  ST_CUDA(cudaMalloc(&cidx.p, (size_t)nch * nA * k * 8));
  ST_CUDA(cudaMalloc(&csc.p, (size_t)nch * nA * k * 4));
  std::vector<int64_t> c0h(nch);
  for (int c = 0; c < nch; ++c) c0h[c] = (int64_t)c * sp.rows;
  ST_CUDA(cudaMalloc(&c0d.p, (size_t)nch * 8));
  ST_CUDA(cudaMemcpyAsync(c0d.p, c0h.data(), (size_t)nch * 8, cudaMemcpyHostToDevice, stm));
  s = stage_chunk(sp, nB, d, 0);
  if (s != SJ_OK) return s;
  for (int c = 0; c < nch; ++c) {
    const int64_t nc = std::min(sp.rows, nB - c0h[c]);
    ST_CUDA(cudaStreamWaitEvent(stm, sp.cs.ev[c & 1], 0));
    // the next chunk goes into the other buffer, which the previous join
    // (synchronous: finished on return) no longer reads
    if (c + 1 < nch) {
      s = stage_chunk(sp, nB, d, c + 1);
      if (s != SJ_OK) return s;
    }
    sj_stats one;
    s = sj_topk(h, sp.Adev, nA, static_cast<const float *>(sp.stage[c & 1].p), nc, k,
                static_cast<int64_t *>(cidx.p) + (size_t)c * nA * k,
                static_cast<float *>(csc.p) + (size_t)c * nA * k, &one);
    if (s != SJ_OK) return s;
    add_chunk_stats(&acc, one);
  }
  // merge of the chunks' lists: the fast k-way merge (up to 32 chunks), the
  // exact ranker for the rows it leaves (all rows with more chunks)
  int n_pad = 1;
  while (n_pad < k * nch) n_pad <<= 1;
  const size_t slot = merge_slot_bytes(n_pad);
  const int grid = (int)std::min<int64_t>(nA, (int64_t)handle_sm_count(h) * 4);
  DMem slow;
  ST_CUDA(cudaMalloc(&scratch.p, slot * grid));
  ST_CUDA(cudaMalloc(&ctr.p, sizeof(Counters) + 16));
  ST_CUDA(cudaMalloc(&slow.p, (size_t)nA * 4));
  ST_CUDA(cudaMemsetAsync(ctr.p, 0, sizeof(Counters) + 16, stm));
  unsigned *n_slow = reinterpret_cast<unsigned *>(static_cast<unsigned char *>(ctr.p) +
                                                  sizeof(Counters));
  if (nch <= 32) {
    merge_fast_kernel<<<(unsigned)std::min<int64_t>((nA + 7) / 8, 65535), 256, 0, stm>>>(
        nA, k, nch, static_cast<int64_t *>(c0d.p), static_cast<int64_t *>(cidx.p),
        static_cast<float *>(csc.p), out_idx, out_score, static_cast<int *>(slow.p), n_slow);
    ST_CUDA(cudaGetLastError());
  } else {
    std::vector<int> all((size_t)nA);
    for (int64_t i = 0; i < nA; ++i) all[i] = (int)i;
    const unsigned na = (unsigned)nA;
    ST_CUDA(cudaMemcpyAsync(slow.p, all.data(), (size_t)nA * 4, cudaMemcpyHostToDevice, stm));
    ST_CUDA(cudaMemcpyAsync(n_slow, &na, 4, cudaMemcpyHostToDevice, stm));
    ST_CUDA(cudaStreamSynchronize(stm));
  }
  merge_topk_kernel<<<grid, kMergeThreads, 0, stm>>>(
      static_cast<int *>(slow.p), n_slow, sp.Adev, sp.mb.dev, nA, d, k, nch,
      static_cast<int64_t *>(c0d.p), static_cast<int64_t *>(cidx.p),
      static_cast<float *>(csc.p), dot2_coef_key_of(d), out_idx, out_score,
      static_cast<unsigned char *>(scratch.p), slot, static_cast<Counters *>(ctr.p));
  ST_CUDA(cudaGetLastError());
  acc.n_launches += 1;
  Counters hc;
  ST_CUDA(cudaMemcpyAsync(&hc, ctr.p, sizeof hc, cudaMemcpyDeviceToHost, stm));
  ST_CUDA(cudaStreamSynchronize(stm));
  acc.n_launches += 1;
  acc.n_exact += (int64_t)hc.n_exact;
  if (st) *st = acc;
  return SJ_OK;
}

extern "C" sj_status sj_threshold_streamed(sj_handle *h, const float *A, int64_t nA,
                                           const float *B, int64_t nB, double tau,
                                           int64_t chunk_rows, sj_pair *out, int64_t capacity,
                                           int64_t *n_out, sj_stats *st) {
  if (!h || !A || !B || nA < 1 || nB < 1 || std::isnan(tau) || !n_out || capacity < 0 ||
      (capacity > 0 && !out) || chunk_rows < 0)
    return SJ_ERR_INVALID_ARG;
  const int dev = handle_device(h);
  const int64_t d = handle_config(h)->d;
  cudaStream_t stm = static_cast<cudaStream_t>(handle_stream(h));
  sj_stats acc{};
  StreamPlan sp;
  sj_status s = stream_setup(h, A, nA, B, nB, chunk_rows, sp);
  if (s != SJ_OK) return s;
  const int nch = sp.n_chunks;
  // every chunk's pairs (sorted by (i, j)), columns offset to B's rows
  std::vector<std::vector<sj_pair>> parts(nch);
  DMem buf;
  int64_t buf_cap = 0;
  s = stage_chunk(sp, nB, d, 0);
  if (s != SJ_OK) return s;
  for (int c = 0; c < nch; ++c) {
    const int64_t c0 = (int64_t)c * sp.rows, nc = std::min(sp.rows, nB - c0);
    ST_CUDA(cudaStreamWaitEvent(stm, sp.cs.ev[c & 1], 0));
    if (c + 1 < nch) {
      s = stage_chunk(sp, nB, d, c + 1);
      if (s != SJ_OK) return s;
    }
    int64_t m = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (buf_cap == 0 || (attempt == 1 && m > buf_cap)) {
        if (buf.p) cudaFree(buf.p);
        buf.p = nullptr;
        buf_cap = std::max<int64_t>({m, buf_cap, (int64_t)1 << 20});
        ST_CUDA(cudaMalloc(&buf.p, (size_t)buf_cap * sizeof(sj_pair)));
      }
      sj_stats one;
      s = sj_threshold(h, sp.Adev, nA, static_cast<const float *>(sp.stage[c & 1].p), nc, tau,
                       static_cast<sj_pair *>(buf.p), buf_cap, &m, &one);
      if (s == SJ_ERR_CAPACITY) continue;
      if (s != SJ_OK) return s;
      add_chunk_stats(&acc, one);
      break;
    }
    if (s != SJ_OK) return s;
    parts[c].resize((size_t)m);
    if (m > 0)
      ST_CUDA(cudaMemcpyAsync(parts[c].data(), buf.p, (size_t)m * sizeof(sj_pair),
                              cudaMemcpyDeviceToHost, stm));
    ST_CUDA(cudaStreamSynchronize(stm));
    for (sj_pair &p : parts[c]) p.j += c0;
  }
  // merge by row in chunk order: within a row the chunks' columns increase
  int64_t total = 0;
  for (const auto &p : parts) total += (int64_t)p.size();
  if (st) {
    acc.n_pairs = total;
    *st = acc;
  }
  const int wn = where_dev(n_out, dev);
  if (wn < 0) return SJ_ERR_INVALID_ARG;
  if (wn == 1) ST_CUDA(cudaMemcpy(n_out, &total, 8, cudaMemcpyHostToDevice));
  else *n_out = total;
  if (total > capacity) return SJ_ERR_CAPACITY;
  std::vector<sj_pair> merged;
  merged.reserve((size_t)total);
  std::vector<size_t> pos(nch, 0);
  for (int64_t i = 0; i < nA; ++i)
    for (int c = 0; c < nch; ++c)
      while (pos[c] < parts[c].size() && parts[c][pos[c]].i == i) merged.push_back(parts[c][pos[c]++]);
  const int wo = total > 0 ? where_dev(out, dev) : 0;
  if (wo < 0) return SJ_ERR_INVALID_ARG;
  if (total > 0) {
    if (wo == 1)
      ST_CUDA(cudaMemcpy(out, merged.data(), (size_t)total * sizeof(sj_pair),
                         cudaMemcpyHostToDevice));
    else
      std::memcpy(out, merged.data(), (size_t)total * sizeof(sj_pair));
  }
  return SJ_OK;
}
