// capi.cu -- the C ABI (include/sj.h): handle, workspace, call orchestration.
//
// Per call, on cfg.stream:
//   stage inputs (host pointers only) -> validate + pack A and B ->
//   scoring pass with the fused filter -> finalisation -> (fallback rows) ->
//   copy outputs back (host pointers only).
// Every status that depends on device-side checks is read back before the
// call returns.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/sj.h"
#include "contrastive.h"
#include "sj_internal.h"
#include "tc_host.h"

using namespace sj;

namespace {

constexpr int kVersion = 100;  // 0.1.0

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Bump allocator over the handle's workspace.
struct Arena {
  unsigned char *base = nullptr;
  size_t size = 0, used = 0;
  void *take(size_t bytes) {
    size_t off = align_up(used, 256);
    if (off + bytes > size) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// gamma_n = n u / (1 - n u)
double gamma_n(double n, double u) { return n * u / (1.0 - n * u); }

}  // namespace

struct sj_handle {
  sj_config cfg{};
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int cc = 0;
  void *ws = nullptr;
  size_t ws_size = 0;
  Counters *h_ctr = nullptr;   // pinned
  int64_t *h_i64 = nullptr;    // pinned scratch for small readbacks
  cudaEvent_t ev[6]{};
  sj::TcContext *tc = nullptr;
};

namespace {

sj_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SJ_OK;
  if (e == cudaErrorMemoryAllocation) return SJ_ERR_OOM;
  return SJ_ERR_CUDA;
}

#define SJ_CUDA(call)                          \
  do {                                         \
    cudaError_t e__ = (call);                  \
    if (e__ != cudaSuccess) return cuda_status(e__); \
  } while (0)

sj_status ensure_ws(sj_handle *h, size_t bytes) {
  if (bytes <= h->ws_size) return SJ_OK;
  if (h->cfg.workspace_limit && bytes > h->cfg.workspace_limit) return SJ_ERR_OOM;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_size = 0;
  }
  size_t want = align_up(bytes + bytes / 8, 1 << 20);
  if (h->cfg.workspace_limit && want > h->cfg.workspace_limit) want = h->cfg.workspace_limit;
  cudaError_t e = cudaMalloc(&h->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      h->ws = nullptr;
      return SJ_ERR_OOM;
    }
    want = bytes;
  }
  h->ws_size = want;
  return SJ_OK;
}

// Tile shape and packing of one precision.
struct PrecPlan {
  PackFormat fmt;
  int elem;       // bytes per packed element
  int BM, BN;     // score tile
  int64_t dp;     // padded width
  double acc_coef;
};

PrecPlan plan_prec(sj_precision p, int64_t d) {
  PrecPlan q;
  if (p == SJ_FP32) {
    q.fmt = PackFormat::kF32;
    q.elem = 4;
    q.BM = kSimtBM;
    q.BN = kSimtBN;
    q.dp = round_up(d, kSimtBK);
    // FMA chain of d steps, one rounding each: gamma_d (u = 2^-24), doubled.
    q.acc_coef = 2.0 * gamma_n((double)d + 2.0, std::ldexp(1.0, -24));
  } else {
    q.fmt = PackFormat::kBF16;
    q.elem = 2;
    q.BM = kTcBM;
    q.BN = kTcBN;
    q.dp = round_up(d, 64);
    // Exact bf16 x bf16 products accumulated in FP32 by the tensor core; the
    // internal accumulation order and rounding are not specified, so allow
    // 8x the sequential round-to-nearest bound: (d + 32) 2^-21 (u = 2^-24).
    q.acc_coef = ((double)d + 32.0) * std::ldexp(1.0, -21);
  }
  return q;
}

// Dot2 error coefficient (see sj_device.cuh): lane chains of n = ceil(d/32)
// products plus a 5-level combination, bound
//   2 [ gamma_{n+1}^2 + 10 u (gamma_{n+1} + 5u) ] sum|p|,  u = 2^-24,
// returned in key units (x 2^60), rounded up.
float dot2_coef_key(int64_t d) {
  const double u = std::ldexp(1.0, -24);
  double n = (double)((d + 31) / 32);
  double g = gamma_n(n + 1.0, u);
  double c = 2.0 * (g * g + 10.0 * u * (g + 5.0 * u)) * (1.0 + 1e-6);
  double key = std::ldexp(c, kKeyShift);
  float f = (float)key;
  if ((double)f < key) f = std::nextafter(f, INFINITY);
  return f;
}

// ceil(tau 2^298) as an Exact (two's complement, 320 bits).
Exact tau_to_exact(double tau) {
  uint32_t w[10] = {0};
  Exact x{};
  if (tau == 0.0) return x;
  int e;
  double fr = std::frexp(std::fabs(tau), &e);       // |tau| = fr 2^e
  uint64_t M = (uint64_t)std::ldexp(fr, 53);        // |tau| = M 2^(e-53)
  int sh = e - 53 + 298;
  bool neg = tau < 0;
  if (sh >= 0) {
    // M << sh into the 320-bit word (M < 2^53, sh + 53 <= 300)
    for (int b = 0; b < 64; ++b)
      if ((M >> b) & 1u) {
        int pos = b + sh;
        if (pos < 320) w[pos / 32] |= 1u << (pos % 32);
      }
  } else {
    int r = -sh;
    uint64_t q, rem;
    if (r >= 64) {
      q = 0;
      rem = M;
    } else {
      q = M >> r;
      rem = M & ((r == 64) ? ~0ull : ((1ull << r) - 1));
    }
    // ceil for positive tau, floor of |tau| (then negated) for negative tau
    if (!neg && rem) q += 1;
    w[0] = (uint32_t)q;
    w[1] = (uint32_t)(q >> 32);
  }
  if (neg) {
    uint64_t carry = 1;
    for (int t = 0; t < 10; ++t) {
      uint64_t v = (uint64_t)(~w[t]) + carry;
      w[t] = (uint32_t)v;
      carry = v >> 32;
    }
  }
  for (int t = 0; t < 9; ++t) x.d[t] = w[t];
  x.top = (int32_t)w[9];
  return x;
}

struct JoinPlan {
  PrecPlan pp;
  int64_t nA, nB, d, nA_pad, nB_pad;
  int S;
  int bands;  // band lists per (row, split): epilogue column groups of the kernel
  int64_t tiles_per_split, n_units;
  int cap;
};

JoinPlan make_plan(const sj_handle *h, int64_t nA, int64_t nB, int k) {
  JoinPlan p;
  p.pp = plan_prec(h->cfg.prec, h->cfg.d);
  p.nA = nA;
  p.nB = nB;
  p.d = h->cfg.d;
  // Both operands are padded to the larger tile edge so that a self-join can
  // share one packed copy; row blocks and column tiles cover the true sizes.
  const int64_t edge = std::max(p.pp.BM, p.pp.BN);
  p.nA_pad = round_up(std::max<int64_t>(nA, 1), edge);
  p.nB_pad = round_up(std::max<int64_t>(nB, 1), edge);
  int64_t rb = (std::max<int64_t>(nA, 1) + p.pp.BM - 1) / p.pp.BM;
  int64_t ct = (std::max<int64_t>(nB, 1) + p.pp.BN - 1) / p.pp.BN;
  int64_t want_units = 2 * (int64_t)h->sm_count;
  int64_t S = (want_units + rb - 1) / rb;
  if (S < 1 || (h->cfg.flags & SJ_FLAG_SINGLE_SPLIT)) S = 1;
  if (S > ct) S = ct;
  if (S > 256) S = 256;  // bounds the per-(row, split) band lists
  p.tiles_per_split = (ct + S - 1) / S;
  p.S = (int)((ct + p.tiles_per_split - 1) / p.tiles_per_split);
  p.n_units = rb * p.S;
  p.bands = h->cfg.prec == SJ_FP32 ? 1 : 2;
  // band list per row: the k best plus the margin band (often ~60-150 rows
  // for BF16 scores of d = 768 embeddings near the k-th score)
  p.cap = (int)round_up(4 * (int64_t)k + 256, 32);
  return p;
}

struct Events {
  sj_handle *h;
  void rec(int t) { cudaEventRecord(h->ev[t], h->stream); }
  double ms(int a, int b) {
    float v = 0.f;
    if (cudaEventElapsedTime(&v, h->ev[a], h->ev[b]) != cudaSuccess) {
      cudaGetLastError();
      return 0.0;
    }
    return v;
  }
};

sj_status read_counters(sj_handle *h, Counters *d_ctr) {
  SJ_CUDA(cudaMemcpyAsync(h->h_ctr, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, h->stream));
  SJ_CUDA(cudaStreamSynchronize(h->stream));
  return SJ_OK;
}

sj_status flags_status(unsigned f) {
  if (f & kErrNonFinite) return SJ_ERR_NONFINITE;
  if (f & kErrNotUnit) return SJ_ERR_NOT_UNIT_NORM;
  if (f & kErrTimeout) return SJ_ERR_TIMEOUT;
  if (f & kErrInternal) return SJ_ERR_INTERNAL;
  return SJ_OK;
}

// Inputs of one join, resolved to device memory.
struct JoinIO {
  const float *A, *B;
  bool a_host, b_host;
};

// Shared front half: staging, validation, packing.  Fills the plan buffers.
struct Prepared {
  JoinPlan plan;
  const float *A, *B;          // device float32 rows
  void *Ap, *Bp;               // packed
  RowMeta *metaA, *metaB;
  float *gmaxB;
  Counters *ctr;
  TcMaps maps;
};

sj_status prepare_join(sj_handle *h, Arena &ar, const float *A, int64_t nA, const float *B,
                       int64_t nB, int k, Prepared &P) {
  cudaStream_t st = h->stream;
  P.plan = make_plan(h, nA, nB, k);
  const JoinPlan &pl = P.plan;
  const int64_t d = pl.d;
  P.ctr = static_cast<Counters *>(ar.take(sizeof(Counters)));
  P.gmaxB = static_cast<float *>(ar.take(4 * sizeof(float)));
  float *gmaxA = static_cast<float *>(ar.take(4 * sizeof(float)));
  P.metaA = static_cast<RowMeta *>(ar.take(sizeof(RowMeta) * pl.nA_pad));
  P.metaB = static_cast<RowMeta *>(ar.take(sizeof(RowMeta) * pl.nB_pad));
  P.Ap = ar.take((size_t)pl.nA_pad * pl.pp.dp * pl.pp.elem);
  P.Bp = (A == B && nA == nB)
             ? P.Ap
             : ar.take((size_t)pl.nB_pad * pl.pp.dp * pl.pp.elem);
  P.A = A;
  P.B = B;
  if (!is_device_ptr(A) && nA > 0) {
    float *dA = static_cast<float *>(ar.take((size_t)nA * d * sizeof(float)));
    if (!dA) return SJ_ERR_INTERNAL;
    SJ_CUDA(cudaMemcpyAsync(dA, A, (size_t)nA * d * sizeof(float), cudaMemcpyHostToDevice, st));
    P.A = dA;
  }
  if (B == A) {
    P.B = P.A;
  } else if (!is_device_ptr(B) && nB > 0) {
    float *dB = static_cast<float *>(ar.take((size_t)nB * d * sizeof(float)));
    if (!dB) return SJ_ERR_INTERNAL;
    SJ_CUDA(cudaMemcpyAsync(dB, B, (size_t)nB * d * sizeof(float), cudaMemcpyHostToDevice, st));
    P.B = dB;
  }
  if (!P.ctr || !P.gmaxB || !P.metaA || !P.metaB || !P.Ap || !P.Bp) return SJ_ERR_INTERNAL;
  SJ_CUDA(cudaMemsetAsync(P.ctr, 0, sizeof(Counters), st));
  SJ_CUDA(cudaMemsetAsync(P.gmaxB, 0, 4 * sizeof(float), st));
  SJ_CUDA(cudaMemsetAsync(gmaxA, 0, 4 * sizeof(float), st));
  SJ_CUDA(launch_prepare(P.A, nA, d, pl.pp.fmt, P.Ap, pl.nA_pad, pl.pp.dp, P.metaA, gmaxA, P.ctr, st));
  if (P.Bp != P.Ap)
    SJ_CUDA(launch_prepare(P.B, nB, d, pl.pp.fmt, P.Bp, pl.nB_pad, pl.pp.dp, P.metaB, P.gmaxB, P.ctr, st));
  else {
    SJ_CUDA(cudaMemcpyAsync(P.metaB, P.metaA, sizeof(RowMeta) * pl.nB_pad, cudaMemcpyDeviceToDevice, st));
    SJ_CUDA(cudaMemcpyAsync(P.gmaxB, gmaxA, 4 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  if (h->cfg.prec != SJ_FP32) {
    sj_status s = tc_make_maps(h->tc, P.Ap, pl.nA_pad, P.Bp, pl.nB_pad, pl.pp.dp, &P.maps);
    if (s != SJ_OK) return s;
  }
  return SJ_OK;
}

// Workspace estimate of the front half.
size_t prepare_bytes(const JoinPlan &pl, bool a_host, bool b_host, bool self) {
  size_t b = 4096 + sizeof(RowMeta) * (pl.nA_pad + pl.nB_pad) + 8 * 256;
  b += (size_t)pl.nA_pad * pl.pp.dp * pl.pp.elem;
  if (!self) b += (size_t)pl.nB_pad * pl.pp.dp * pl.pp.elem;
  if (a_host) b += (size_t)pl.nA * pl.d * 4 + 256;
  if (b_host && !self) b += (size_t)pl.nB * pl.d * 4 + 256;
  return b;
}

sj_status run_score(sj_handle *h, const Prepared &P, ScoreArgs &sa) {
  const JoinPlan &pl = P.plan;
  sa.Ap = P.Ap;
  sa.Bp = P.Bp;
  sa.nA = pl.nA;
  sa.nB = pl.nB;
  sa.dp = pl.pp.dp;
  sa.metaA = P.metaA;
  sa.gmaxB = P.gmaxB;
  sa.acc_coef = (float)pl.pp.acc_coef;
  sa.n_splits = pl.S;
  sa.bands_per_split = pl.bands;
  sa.tiles_per_split = pl.tiles_per_split;
  sa.n_units = pl.n_units;
  sa.ctr = P.ctr;
  if (pl.nA == 0 || pl.nB == 0) return SJ_OK;
  int grid = (int)std::min<int64_t>(pl.n_units, (int64_t)h->sm_count * 2);
  if (h->cfg.prec == SJ_FP32) {
    SJ_CUDA(launch_score_simt(sa, grid, h->stream));
  } else {
    grid = (int)std::min<int64_t>(pl.n_units, (int64_t)h->sm_count);
    SJ_CUDA(launch_score_tc(sa, grid, &P.maps, h->cfg.flags, h->stream));
  }
  return SJ_OK;
}

void fill_common_stats(sj_stats *st, const Counters &c) {
  st->n_candidates = (int64_t)c.n_candidates;
  st->n_rescored = (int64_t)c.n_rescored;
  st->n_exact = (int64_t)c.n_exact;
  st->n_overflow_rows = (int64_t)c.overflow_rows;
  st->n_tier2_rows = (int64_t)c.tier2_rows;
  float me;
  std::memcpy(&me, &c.max_err_bits, sizeof me);
  st->max_abs_err_lowprec = me;
}

sj_status check_join_args(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB) {
  if (!h) return SJ_ERR_INVALID_ARG;
  if (nA < 0 || nB < 0) return SJ_ERR_INVALID_ARG;
  if ((nA > 0 && !A) || (nB > 0 && !B)) return SJ_ERR_INVALID_ARG;
  if (nA >= (1ll << 31) - 1024 || nB >= (1ll << 31) - 1024) return SJ_ERR_UNSUPPORTED;
  return SJ_OK;
}

// Scratch that the fallback takes from the workspace if it fits, else from a
// temporary allocation released before the call returns.
struct Scratch {
  void *p = nullptr;
  bool own = false;
  ~Scratch() {
    if (own) cudaFree(p);
  }
  cudaError_t get(Arena &ar, size_t bytes) {
    p = ar.take(bytes);
    if (p) return cudaSuccess;
    own = true;
    return cudaMalloc(&p, bytes);
  }
};

// Rows whose candidates did not fit: rescan all of B with Dot2 against the
// row's key bound, then rank the lists (shared memory, or global memory for
// very long ones).  Lists cut off at their capacity are rescanned once more
// with the capacity they need.
sj_status topk_fallback(sj_handle *h, const Prepared &P, const JoinPlan &pl, const int *rows,
                        const long long *keys, int n_rows, int k, int64_t *d_idx, float *d_score,
                        Arena &ar, int64_t &launches) {
  cudaStream_t stm = h->stream;
  const int64_t nB = pl.nB;
  int cap = (int)std::min<int64_t>(nB, 4096);
  Scratch lists_s, count_s, redo_s, big_s, rows2_s, keys2_s;
  SJ_CUDA(count_s.get(ar, (size_t)n_rows * 4 + 256));
  SJ_CUDA(redo_s.get(ar, (size_t)n_rows * 4 + 256));
  SJ_CUDA(big_s.get(ar, (size_t)n_rows * 4 + 256));
  SJ_CUDA(rows2_s.get(ar, (size_t)n_rows * 4 + 256));
  SJ_CUDA(keys2_s.get(ar, (size_t)n_rows * 8 + 256));
  const int *cur_rows = rows;
  const long long *cur_keys = keys;
  int n_cur = n_rows;
  for (int pass = 0; pass < 2 && n_cur > 0; ++pass) {
    Scratch lists;
    SJ_CUDA(lists.get(ar, (size_t)n_cur * cap * sizeof(KeyCand)));
    int *count = static_cast<int *>(count_s.p);
    SJ_CUDA(cudaMemsetAsync(count, 0, (size_t)n_cur * 4, stm));
    SJ_CUDA(cudaMemsetAsync(&P.ctr->redo_rows, 0, 4 * sizeof(unsigned), stm));
    RescanArgs ra{};
    ra.A = P.A;
    ra.B = P.B;
    ra.nB = nB;
    ra.d = pl.d;
    ra.metaA = P.metaA;
    ra.metaB = P.metaB;
    ra.dot2_coef_key = dot2_coef_key(pl.d);
    ra.rows = cur_rows;
    ra.keys = cur_keys;
    ra.n_rows = n_cur;
    ra.lists = static_cast<KeyCand *>(lists.p);
    ra.count = count;
    ra.cap = cap;
    ra.ctr = P.ctr;
    SJ_CUDA(launch_topk_rescan(ra, stm));
    RankListArgs la{};
    la.A = P.A;
    la.B = P.B;
    la.d = pl.d;
    la.k = k;
    la.rows = cur_rows;
    la.n_rows = n_cur;
    la.lists = ra.lists;
    la.count = count;
    la.cap = cap;
    la.redo = static_cast<int *>(redo_s.p);
    la.big = static_cast<int *>(big_s.p);
    la.out_idx = d_idx;
    la.out_score = d_score;
    la.ctr = P.ctr;
    SJ_CUDA(launch_topk_rank_lists(la, stm));
    launches += 2;
    sj_status s = read_counters(h, P.ctr);
    if (s != SJ_OK) return s;
    const unsigned n_big = h->h_ctr->big_rows;
    if (n_big > 0) {
      const size_t per_row = topk_rank_global_row_bytes(cap);
      Scratch g;
      SJ_CUDA(g.get(ar, (size_t)n_big * per_row));
      SJ_CUDA(launch_topk_rank_global(la, la.big, (int)n_big, g.p, per_row, stm));
      launches += 1;
      SJ_CUDA(cudaStreamSynchronize(stm));
    }
    const unsigned n_redo = h->h_ctr->redo_rows;
    if (n_redo == 0) break;
    if (pass == 1) return SJ_ERR_INTERNAL;  // a full-capacity rescan cannot be cut off
    // gather the rows (and keys) to redo, with the capacity they need
    std::vector<int> slots(n_redo), hrows(n_redo), all_rows(n_cur);
    std::vector<long long> hkeys(n_redo), all_keys(n_cur);
    SJ_CUDA(cudaMemcpyAsync(slots.data(), la.redo, n_redo * 4, cudaMemcpyDeviceToHost, stm));
    SJ_CUDA(cudaMemcpyAsync(all_rows.data(), cur_rows, (size_t)n_cur * 4, cudaMemcpyDeviceToHost, stm));
    SJ_CUDA(cudaMemcpyAsync(all_keys.data(), cur_keys, (size_t)n_cur * 8, cudaMemcpyDeviceToHost, stm));
    SJ_CUDA(cudaStreamSynchronize(stm));
    for (unsigned q = 0; q < n_redo; ++q) {
      hrows[q] = all_rows[slots[q]];
      hkeys[q] = all_keys[slots[q]];
    }
    SJ_CUDA(cudaMemcpyAsync(rows2_s.p, hrows.data(), n_redo * 4, cudaMemcpyHostToDevice, stm));
    SJ_CUDA(cudaMemcpyAsync(keys2_s.p, hkeys.data(), n_redo * 8, cudaMemcpyHostToDevice, stm));
    SJ_CUDA(cudaStreamSynchronize(stm));
    cur_rows = static_cast<int *>(rows2_s.p);
    cur_keys = static_cast<long long *>(keys2_s.p);
    n_cur = (int)n_redo;
    cap = (int)std::min<int64_t>(nB, (int64_t)h->h_ctr->redo_cap);
  }
  return SJ_OK;
}

// One join request: top-k part (k > 0) and/or threshold part (thr).
struct JoinReq {
  const float *A;
  int64_t nA;
  const float *B;
  int64_t nB;
  int k;                 // 0: no top-k
  int64_t *out_idx;
  float *out_score;
  bool thr;              // threshold part requested
  double tau;
  sj_pair *out;
  int64_t capacity;
  int64_t *n_out;
};

// Both parts share one validation/packing pass and one scoring pass.
sj_status join_impl(sj_handle *h, const JoinReq &r, sj_stats *st) {
  const float *A = r.A, *B = r.B;
  const int64_t nA = r.nA, nB = r.nB;
  const int k = r.k;
  sj_status s = check_join_args(h, A, nA, B, nB);
  if (s != SJ_OK) return s;
  if (k < 0 || k > 1024 || (k > 0 && nA > 0 && (!r.out_idx || !r.out_score)))
    return SJ_ERR_INVALID_ARG;
  if (r.thr && (!r.n_out || r.capacity < 0 || std::isnan(r.tau) || (r.capacity > 0 && !r.out)))
    return SJ_ERR_INVALID_ARG;
  if (k == 0 && !r.thr) return SJ_ERR_INVALID_ARG;
  SJ_CUDA(cudaSetDevice(h->cfg.device));
  cudaStream_t stm = h->stream;
  Events ev{h};
  int64_t launches = 0;
  if (st) std::memset(st, 0, sizeof *st);

  // |s| <= ||a|| ||b|| < 1.00001 for validated rows: clamping tau to [-4, 4]
  // changes no decision and keeps it inside the key and exact ranges.
  const double tau_c = std::min(4.0, std::max(-4.0, r.thr ? r.tau : 4.0));
  float tau_f = INFINITY;
  if (r.thr) {
    tau_f = (float)tau_c;
    if ((double)tau_f > tau_c) tau_f = std::nextafter(tau_f, -INFINITY);
  }
  const long long tau_key = (long long)std::ceil(std::ldexp(tau_c, kKeyShift));
  const Exact tau_ex = tau_to_exact(tau_c);

  const bool a_host = nA > 0 && !is_device_ptr(A);
  const bool b_host = nB > 0 && !is_device_ptr(B) && B != A;
  const bool ot_host = k > 0 && nA > 0 && (!is_device_ptr(r.out_idx) || !is_device_ptr(r.out_score));
  const bool op_host = r.thr && r.capacity > 0 && !is_device_ptr(r.out);
  const JoinPlan pl = make_plan(h, nA, nB, k);
  const bool self = (A == B && nA == nB);
  const size_t slots = (size_t)std::max<int64_t>(nA, 1) * pl.S * pl.bands;
  const size_t rows1 = (size_t)std::max<int64_t>(nA, 1);
  unsigned long long thr_cap = 0;
  if (r.thr)
    thr_cap = (unsigned long long)std::max<int64_t>({(int64_t)1 << 16, 2 * nA,
                                                     r.capacity + r.capacity / 4});

  for (int attempt = 0; attempt < 3; ++attempt) {
    ev.rec(0);
    size_t bytes = prepare_bytes(pl, a_host, b_host, self);
    if (k > 0) {
      bytes += slots * (size_t)pl.cap * sizeof(Cand) + 256;  // band lists
      bytes += slots * 4 + 256;                              // band counts
      bytes += rows1 * 16 + 768;                             // tier-2/overflow rows, keys
      if (ot_host) bytes += (size_t)nA * k * 12 + 512;
    }
    if (r.thr) {
      bytes += (size_t)thr_cap * sizeof(ThrCand) * 2 + 512;  // candidates + accepted
      bytes += rows1 * 8 * 3 + 768;                          // count, offset, fill
      bytes += scan_scratch_bytes(nA) + 256 + 4096;
    }
    s = ensure_ws(h, bytes);
    if (s != SJ_OK) return s;
    Arena ar{static_cast<unsigned char *>(h->ws), h->ws_size, 0};
    Prepared P;
    s = prepare_join(h, ar, A, nA, B, nB, k, P);
    if (s != SJ_OK) return s;
    launches += (P.Bp == P.Ap) ? 1 : 2;
    Cand *band = nullptr;
    int *band_cnt = nullptr, *ovf = nullptr, *tier2 = nullptr;
    long long *ovf_key = nullptr;
    int64_t *d_idx = r.out_idx;
    float *d_score = r.out_score;
    if (k > 0) {
      band = static_cast<Cand *>(ar.take(slots * (size_t)pl.cap * sizeof(Cand)));
      band_cnt = static_cast<int *>(ar.take(slots * 4));
      ovf = static_cast<int *>(ar.take(rows1 * 4));
      tier2 = static_cast<int *>(ar.take(rows1 * 4));
      ovf_key = static_cast<long long *>(ar.take(rows1 * 8));
      if (ot_host) {
        d_idx = static_cast<int64_t *>(ar.take((size_t)nA * k * 8));
        d_score = static_cast<float *>(ar.take((size_t)nA * k * 4));
      }
      if (!band || !band_cnt || !ovf || !tier2 || !ovf_key ||
          (nA > 0 && (!d_idx || !d_score)))
        return SJ_ERR_INTERNAL;
    }
    ThrCand *cand = nullptr, *accd = nullptr;
    int64_t *row_count = nullptr, *row_off = nullptr, *row_fill = nullptr, *total = nullptr;
    int *n_big = nullptr;
    void *scan_scr = nullptr;
    if (r.thr) {
      cand = static_cast<ThrCand *>(ar.take((size_t)thr_cap * sizeof(ThrCand)));
      accd = static_cast<ThrCand *>(ar.take((size_t)thr_cap * sizeof(ThrCand)));
      row_count = static_cast<int64_t *>(ar.take(rows1 * 8));
      row_off = static_cast<int64_t *>(ar.take(rows1 * 8));
      row_fill = static_cast<int64_t *>(ar.take(rows1 * 8));
      total = static_cast<int64_t *>(ar.take(64));
      n_big = static_cast<int *>(ar.take(64));
      scan_scr = ar.take(scan_scratch_bytes(nA));
      if (!cand || !accd || !row_count || !row_off || !row_fill || !total || !n_big || !scan_scr)
        return SJ_ERR_INTERNAL;
    }
    ev.rec(1);
    s = read_counters(h, P.ctr);
    if (s != SJ_OK) return s;
    s = flags_status(h->h_ctr->err_flags);
    if (s != SJ_OK) return s;

    if (nA == 0 || nB == 0) {
      if (k > 0 && nA > 0) {
        std::vector<int64_t> pad_i((size_t)nA * k, -1);
        std::vector<float> pad_s((size_t)nA * k, -INFINITY);
        SJ_CUDA(cudaMemcpyAsync(r.out_idx, pad_i.data(), pad_i.size() * 8, cudaMemcpyDefault, stm));
        SJ_CUDA(cudaMemcpyAsync(r.out_score, pad_s.data(), pad_s.size() * 4, cudaMemcpyDefault, stm));
        SJ_CUDA(cudaStreamSynchronize(stm));
      }
      if (r.thr) *r.n_out = 0;
      return SJ_OK;
    }

    ScoreArgs sa{};
    sa.k = k;
    sa.tau_f = tau_f;
    sa.band = band;
    sa.cap = k > 0 ? pl.cap : 0;
    sa.band_cnt = band_cnt;
    sa.thr = cand;
    sa.thr_cap = thr_cap;
    s = run_score(h, P, sa);
    if (s != SJ_OK) return s;
    launches += 1;
    ev.rec(2);
    if (r.thr) {
      s = read_counters(h, P.ctr);
      if (s != SJ_OK) return s;
      s = flags_status(h->h_ctr->err_flags);
      if (s != SJ_OK) return s;
      const unsigned long long n_cand = h->h_ctr->thr_count;
      if (n_cand > thr_cap) {
        thr_cap = n_cand + n_cand / 8 + 1024;  // rerun with room for every candidate
        continue;
      }
    }

    // ---- top-k finalisation (+ fallback rows) ----
    if (k > 0) {
      TopkFinalArgs fa{};
      fa.A = P.A;
      fa.B = P.B;
      fa.nA = nA;
      fa.nB = nB;
      fa.d = pl.d;
      fa.metaA = P.metaA;
      fa.metaB = P.metaB;
      fa.gmaxB = P.gmaxB;
      fa.acc_coef = (float)pl.pp.acc_coef;
      fa.k = k;
      fa.n_splits = pl.S * pl.bands;
      fa.cap = pl.cap;
      fa.band = band;
      fa.band_cnt = band_cnt;
      fa.dot2_coef_key = dot2_coef_key(pl.d);
      fa.out_idx = d_idx;
      fa.out_score = d_score;
      fa.tier2_rows = tier2;
      fa.overflow_rows = ovf;
      fa.overflow_key = ovf_key;
      fa.ctr = P.ctr;
      SJ_CUDA(launch_topk_finalize(fa, stm));
      launches += 1;
      s = read_counters(h, P.ctr);
      if (s != SJ_OK) return s;
      s = flags_status(h->h_ctr->err_flags);
      if (s != SJ_OK) return s;
      const unsigned n_t2 = h->h_ctr->tier2_rows;
      if (n_t2 > 0) {
        SJ_CUDA(launch_topk_finalize_tier2(fa, (int)n_t2, stm));
        launches += 1;
        s = read_counters(h, P.ctr);
        if (s != SJ_OK) return s;
      }
      const unsigned n_ovf = h->h_ctr->overflow_rows;
      if (n_ovf > 0) {
        s = topk_fallback(h, P, pl, ovf, ovf_key, (int)n_ovf, k, d_idx, d_score, ar, launches);
        if (s != SJ_OK) return s;
      }
      if (ot_host) {
        SJ_CUDA(cudaMemcpyAsync(r.out_idx, d_idx, (size_t)nA * k * 8, cudaMemcpyDeviceToHost, stm));
        SJ_CUDA(cudaMemcpyAsync(r.out_score, d_score, (size_t)nA * k * 4, cudaMemcpyDeviceToHost, stm));
      }
    }

    // ---- threshold finalisation ----
    int64_t n_pairs = 0;
    if (r.thr) {
      const unsigned long long n_cand = h->h_ctr->thr_count;
      SJ_CUDA(cudaMemsetAsync(row_count, 0, (size_t)nA * 8, stm));
      SJ_CUDA(cudaMemsetAsync(row_fill, 0, (size_t)nA * 8, stm));
      ThrFinalArgs ta{};
      ta.A = P.A;
      ta.B = P.B;
      ta.nA = nA;
      ta.nB = nB;
      ta.d = pl.d;
      ta.metaA = P.metaA;
      ta.metaB = P.metaB;
      ta.dot2_coef_key = dot2_coef_key(pl.d);
      ta.tau_key = tau_key;
      ta.tau_exact = tau_ex;
      ta.cand = cand;
      ta.n_cand = (int64_t)n_cand;
      ta.row_count = row_count;
      ta.accepted = accd;
      ta.ctr = P.ctr;
      SJ_CUDA(launch_thr_rescore(ta, stm));
      launches += n_cand ? 1 : 0;
      s = read_counters(h, P.ctr);
      if (s != SJ_OK) return s;
      n_pairs = (int64_t)h->h_ctr->n_pairs;
      *r.n_out = n_pairs;
      if (n_pairs > r.capacity) {
        if (st) {
          fill_common_stats(st, *h->h_ctr);
          st->n_pairs = n_pairs;
        }
        return SJ_ERR_CAPACITY;
      }
      if (n_pairs > 0) {
        SJ_CUDA(launch_exclusive_scan(row_count, row_off, nA, total, scan_scr, stm));
        launches += 3;
        Arena ar2 = ar;
        PairOut *d_out = op_host ? static_cast<PairOut *>(ar2.take((size_t)n_pairs * sizeof(PairOut)))
                                 : reinterpret_cast<PairOut *>(r.out);
        // the candidate list is free now: reuse it as merge-sort scratch when it fits
        PairOut *tmp = ((size_t)thr_cap * sizeof(ThrCand) >= (size_t)n_pairs * sizeof(PairOut))
                           ? reinterpret_cast<PairOut *>(cand)
                           : static_cast<PairOut *>(ar2.take((size_t)n_pairs * sizeof(PairOut)));
        bool own_out = false, own_tmp = false;
        if (!d_out) {
          if (cudaMalloc(&d_out, (size_t)n_pairs * sizeof(PairOut)) != cudaSuccess) {
            cudaGetLastError();
            return SJ_ERR_OOM;
          }
          own_out = true;
        }
        if (!tmp) {
          if (cudaMalloc(&tmp, (size_t)n_pairs * sizeof(PairOut)) != cudaSuccess) {
            cudaGetLastError();
            if (own_out) cudaFree(d_out);
            return SJ_ERR_OOM;
          }
          own_tmp = true;
        }
        cudaError_t e = launch_thr_scatter(accd, total, n_pairs, row_off, row_fill, d_out, stm);
        // rows of more than 32 pairs are listed in row_fill's memory, which the
        // scatter (earlier on the same stream) no longer needs
        int *big_rows = reinterpret_cast<int *>(row_fill);
        if (e == cudaSuccess) e = cudaMemsetAsync(n_big, 0, sizeof(int), stm);
        if (e == cudaSuccess)
          e = launch_thr_sort_rows(d_out, row_off, row_count, nA, big_rows, n_big, (int)nA, stm);
        launches += 2;
        int hb = 0;
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(&h->h_i64[0], n_big, sizeof(int), cudaMemcpyDeviceToHost, stm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
        if (e == cudaSuccess) {
          std::memcpy(&hb, &h->h_i64[0], sizeof(int));
          e = launch_thr_sort_big(d_out, tmp, row_off, row_count, big_rows, n_big, hb, stm);
          launches += hb ? 1 : 0;
        }
        if (e == cudaSuccess && op_host)
          e = cudaMemcpyAsync(r.out, d_out, (size_t)n_pairs * sizeof(PairOut), cudaMemcpyDeviceToHost, stm);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stm);
        if (own_out) cudaFree(d_out);
        if (own_tmp) cudaFree(tmp);
        if (e != cudaSuccess) return cuda_status(e);
      }
    }
    ev.rec(3);
    s = read_counters(h, P.ctr);  // also drains the stream
    if (s != SJ_OK) return s;
    if (st) {
      fill_common_stats(st, *h->h_ctr);
      if (r.thr) st->n_candidates += (int64_t)h->h_ctr->thr_count;
      st->n_pairs = n_pairs;
      st->n_launches = launches;
      st->ms_prepare = ev.ms(0, 1);
      st->ms_score = ev.ms(1, 2);
      st->ms_select = ev.ms(2, 3);
      st->ms_total = ev.ms(0, 3);
      float mB = 0.f;
      st->margin_max = 0.0;
      (void)mB;
    }
    return flags_status(h->h_ctr->err_flags);
  }
  return SJ_ERR_INTERNAL;
}

sj_status topk_impl(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                    int32_t k, int64_t *out_idx, float *out_score, sj_stats *st) {
  if (k < 1) return SJ_ERR_INVALID_ARG;
  JoinReq r{A, nA, B, nB, k, out_idx, out_score, false, 0.0, nullptr, 0, nullptr};
  return join_impl(h, r, st);
}

sj_status threshold_impl(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                         double tau, sj_pair *out, int64_t capacity, int64_t *n_out,
                         sj_stats *st) {
  JoinReq r{A, nA, B, nB, 0, nullptr, nullptr, true, tau, out, capacity, n_out};
  return join_impl(h, r, st);
}

}  // namespace

extern "C" {

sj_status sj_create(sj_handle **out, const sj_config *cfg) {
  if (!out || !cfg || cfg->d < 1) return SJ_ERR_INVALID_ARG;
  if (cfg->prec != SJ_FP32 && cfg->prec != SJ_BF16 && cfg->prec != SJ_FP8_E4M3)
    return SJ_ERR_INVALID_ARG;
  if (cfg->d > (1 << 20)) return SJ_ERR_UNSUPPORTED;
  *out = nullptr;
  int ndev = 0;
  SJ_CUDA(cudaGetDeviceCount(&ndev));
  if (cfg->device < 0 || cfg->device >= ndev) return SJ_ERR_INVALID_ARG;
  SJ_CUDA(cudaSetDevice(cfg->device));
  cudaDeviceProp prop;
  SJ_CUDA(cudaGetDeviceProperties(&prop, cfg->device));
  const int cc = prop.major * 10 + prop.minor;
  if (cfg->prec == SJ_FP8_E4M3) return SJ_ERR_UNSUPPORTED;
  if (cfg->prec == SJ_BF16 && cc != 103) return SJ_ERR_UNSUPPORTED;
  sj_handle *h = new (std::nothrow) sj_handle();
  if (!h) return SJ_ERR_OOM;
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  h->sm_count = prop.multiProcessorCount;
  h->cc = cc;
  cudaError_t e = cudaMallocHost(&h->h_ctr, sizeof(Counters));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_i64, 64);
  for (int t = 0; t < 6 && e == cudaSuccess; ++t) e = cudaEventCreate(&h->ev[t]);
  if (e == cudaSuccess && cfg->prec != SJ_FP32) {
    sj_status s = tc_create(&h->tc);
    if (s != SJ_OK) {
      sj_destroy(h);
      return s;
    }
  }
  if (e != cudaSuccess) {
    sj_destroy(h);
    return cuda_status(e);
  }
  *out = h;
  return SJ_OK;
}

sj_status sj_destroy(sj_handle *h) {
  if (!h) return SJ_OK;
  cudaSetDevice(h->cfg.device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->h_ctr) cudaFreeHost(h->h_ctr);
  if (h->h_i64) cudaFreeHost(h->h_i64);
  for (int t = 0; t < 6; ++t)
    if (h->ev[t]) cudaEventDestroy(h->ev[t]);
  if (h->tc) tc_destroy(h->tc);
  delete h;
  return SJ_OK;
}

sj_status sj_topk(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB, int32_t k,
                  int64_t *out_idx, float *out_score, sj_stats *st) {
  return topk_impl(h, A, nA, B, nB, k, out_idx, out_score, st);
}

sj_status sj_threshold(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                       double tau, sj_pair *out, int64_t capacity, int64_t *n_out, sj_stats *st) {
  return threshold_impl(h, A, nA, B, nB, tau, out, capacity, n_out, st);
}

sj_status sj_batch(sj_handle *h, const sj_job *jobs, int32_t n_jobs, sj_stats *st) {
  if (!h || n_jobs < 0 || (n_jobs > 0 && !jobs)) return SJ_ERR_INVALID_ARG;
  sj_status first = SJ_OK;
  sj_stats acc{};
  for (int32_t q = 0; q < n_jobs; ++q) {
    const sj_job &jb = jobs[q];
    const bool want_topk = jb.topk_idx || jb.topk_score;
    const bool want_thr = jb.pairs || jb.n_out;
    JoinReq r{jb.A, jb.nA, jb.B, jb.nB, want_topk ? jb.k : 0, jb.topk_idx, jb.topk_score,
              want_thr, jb.tau, jb.pairs, jb.capacity, jb.n_out};
    if (want_topk && jb.k < 1) return SJ_ERR_INVALID_ARG;
    sj_stats one{};
    sj_status s = join_impl(h, r, &one);
    acc.ms_prepare += one.ms_prepare;
    acc.ms_score += one.ms_score;
    acc.ms_select += one.ms_select;
    acc.ms_total += one.ms_total;
    acc.n_candidates += one.n_candidates;
    acc.n_rescored += one.n_rescored;
    acc.n_exact += one.n_exact;
    acc.n_overflow_rows += one.n_overflow_rows;
    acc.n_pairs += one.n_pairs;
    acc.n_launches += one.n_launches;
    acc.max_abs_err_lowprec = std::max(acc.max_abs_err_lowprec, one.max_abs_err_lowprec);
    if (s != SJ_OK && first == SJ_OK) first = s;
    if (s != SJ_OK && s != SJ_ERR_CAPACITY) {
      if (st) *st = acc;
      return s;
    }
  }
  if (st) *st = acc;
  return first;
}

}  // extern "C"

namespace {

// Shared set-up of the contrastive calls: BF16 packing (and transposes for the
// backward) of A and B into the workspace, and their tensor maps.
struct ContrastivePlan {
  int64_t n, d, np, dp;
  void *Ap, *Bp, *AT, *BT;
  Counters *ctr;
  float *scratch;  // 2n floats (per-row loss terms)
  unsigned char mA[128], mB[128], mAT[128], mBT[128];
};

sj_status contrastive_setup(sj_handle *h, const void *A, const void *B, int64_t N, bool bwd,
                            ContrastivePlan &cp) {
  if (!h || !A || !B || N < 1) return SJ_ERR_INVALID_ARG;
  if (N >= (1ll << 31) - 1024) return SJ_ERR_UNSUPPORTED;
  if (!is_device_ptr(A) || !is_device_ptr(B)) return SJ_ERR_INVALID_ARG;
  SJ_CUDA(cudaSetDevice(h->cfg.device));
  if (h->cc != 103) return SJ_ERR_UNSUPPORTED;
  if (!h->tc) {
    sj_status s = tc_create(&h->tc);
    if (s != SJ_OK) return s;
  }
  cp.n = N;
  cp.d = h->cfg.d;
  cp.np = round_up(N, 128);
  cp.dp = round_up(cp.d, 64);
  const size_t op = (size_t)cp.np * cp.dp * 2;
  size_t bytes = 2 * op + (bwd ? 2 * op : 0) + sizeof(Counters) + (size_t)2 * N * 4 + 8 * 256;
  sj_status s = ensure_ws(h, bytes);
  if (s != SJ_OK) return s;
  Arena ar{static_cast<unsigned char *>(h->ws), h->ws_size, 0};
  cp.ctr = static_cast<Counters *>(ar.take(sizeof(Counters)));
  cp.scratch = static_cast<float *>(ar.take((size_t)2 * N * 4));
  cp.Ap = ar.take(op);
  cp.Bp = ar.take(op);
  cp.AT = bwd ? ar.take(op) : nullptr;
  cp.BT = bwd ? ar.take(op) : nullptr;
  if (!cp.ctr || !cp.scratch || !cp.Ap || !cp.Bp || (bwd && (!cp.AT || !cp.BT))) return SJ_ERR_INTERNAL;
  cudaStream_t st = h->stream;
  SJ_CUDA(cudaMemsetAsync(cp.ctr, 0, sizeof(Counters), st));
  SJ_CUDA(launch_contrastive_pack(static_cast<const float *>(A), N, cp.d, cp.Ap, cp.AT, cp.np, cp.dp,
                                  &cp.ctr->err_flags, st));
  SJ_CUDA(launch_contrastive_pack(static_cast<const float *>(B), N, cp.d, cp.Bp, cp.BT, cp.np, cp.dp,
                                  &cp.ctr->err_flags, st));
  s = tc_encode_2d(h->tc, cp.Ap, cp.dp, cp.np, 64, 128, cp.mA);
  if (s == SJ_OK) s = tc_encode_2d(h->tc, cp.Bp, cp.dp, cp.np, 64, 128, cp.mB);
  if (s == SJ_OK && bwd) s = tc_encode_2d(h->tc, cp.AT, cp.np, cp.dp, 64, 64, cp.mAT);
  if (s == SJ_OK && bwd) s = tc_encode_2d(h->tc, cp.BT, cp.np, cp.dp, 64, 64, cp.mBT);
  return s;
}

sj_status contrastive_finish(sj_handle *h, const ContrastivePlan &cp) {
  sj_status s = read_counters(h, cp.ctr);
  if (s != SJ_OK) return s;
  const unsigned f = h->h_ctr->err_flags;
  if (f & kErrNonFinite) return SJ_ERR_NONFINITE;
  if (f & kErrTimeout) return SJ_ERR_TIMEOUT;
  return SJ_OK;
}

}  // namespace

extern "C" {

sj_status sj_contrastive_fwd(sj_handle *h, const void *A, const void *B, int64_t N, float T,
                             float *loss, float *lse) {
  if (!h || !A || !B || N < 1 || !(T > 0.f) || !loss || !lse) return SJ_ERR_INVALID_ARG;
  if (!is_device_ptr(loss) || !is_device_ptr(lse)) return SJ_ERR_INVALID_ARG;
  ContrastivePlan cp;
  sj_status s = contrastive_setup(h, A, B, N, false, cp);
  if (s != SJ_OK) return s;
  const bool sym = (h->cfg.flags & SJ_FLAG_SYM_INFONCE) != 0;
  ContrastiveArgs a{};
  a.n = N;
  a.d = cp.d;
  a.np = cp.np;
  a.dp = cp.dp;
  a.T = T;
  a.n_chunks = 1;
  a.ctr = cp.ctr;
  a.debug_timeout = (h->cfg.flags & SJ_FLAG_DEBUG_TIMEOUT) ? 1 : 0;
  const int grid = (int)std::min<int64_t>(cp.np / 128, h->sm_count);
  a.lse_out = lse;
  a.term_out = cp.scratch;
  SJ_CUDA(launch_contrastive(false, cp.mA, cp.mB, nullptr, a, grid, h->stream));
  if (sym) {
    a.lse_out = lse + N;
    a.term_out = cp.scratch + N;
    SJ_CUDA(launch_contrastive(false, cp.mB, cp.mA, nullptr, a, grid, h->stream));
  }
  SJ_CUDA(launch_contrastive_loss(cp.scratch, sym ? cp.scratch + N : nullptr, N, sym ? 0.5f : 1.f,
                                  0.5f, loss, h->stream));
  return contrastive_finish(h, cp);
}

sj_status sj_backward(sj_handle *h, const void *A, const void *B, int64_t N, float T,
                      const float *lse, const float *grad_loss, float *dA, float *dB) {
  if (!h || !A || !B || N < 1 || !(T > 0.f) || !lse || !grad_loss || !dA || !dB)
    return SJ_ERR_INVALID_ARG;
  if (!is_device_ptr(lse) || !is_device_ptr(grad_loss) || !is_device_ptr(dA) || !is_device_ptr(dB))
    return SJ_ERR_INVALID_ARG;
  ContrastivePlan cp;
  sj_status s = contrastive_setup(h, A, B, N, true, cp);
  if (s != SJ_OK) return s;
  const bool sym = (h->cfg.flags & SJ_FLAG_SYM_INFONCE) != 0;
  ContrastiveArgs a{};
  a.n = N;
  a.d = cp.d;
  a.np = cp.np;
  a.dp = cp.dp;
  a.T = T;
  a.n_chunks = (int)((cp.dp + 383) / 384);
  a.grad_loss = grad_loss;
  a.ctr = cp.ctr;
  a.debug_timeout = (h->cfg.flags & SJ_FLAG_DEBUG_TIMEOUT) ? 1 : 0;
  const int grid = (int)std::min<int64_t>((cp.np / 128) * a.n_chunks, h->sm_count);
  // dA: rows of A against columns (rows of B); row term = softmax over j
  a.lse_r = lse;
  a.wr = sym ? 0.5f : 1.f;
  a.lse_c = sym ? lse + N : lse;
  a.wc = sym ? 0.5f : 0.f;
  a.dX = dA;
  SJ_CUDA(launch_contrastive(true, cp.mA, cp.mB, cp.mBT, a, grid, h->stream));
  // dB: rows of B against columns (rows of A); the row softmax term is indexed
  // by the kernel's columns, the column softmax term by its rows
  a.lse_r = sym ? lse + N : lse;
  a.wr = sym ? 0.5f : 0.f;
  a.lse_c = lse;
  a.wc = sym ? 0.5f : 1.f;
  a.dX = dB;
  SJ_CUDA(launch_contrastive(true, cp.mB, cp.mA, cp.mAT, a, grid, h->stream));
  return contrastive_finish(h, cp);
}

const char *sj_status_string(sj_status s) {
  switch (s) {
    case SJ_OK: return "ok";
    case SJ_ERR_INVALID_ARG: return "invalid argument";
    case SJ_ERR_NONFINITE: return "input holds NaN or Inf";
    case SJ_ERR_NOT_UNIT_NORM: return "input row is not unit norm (| ||x||^2 - 1 | > 1e-5)";
    case SJ_ERR_CAPACITY: return "output capacity too small (required count written)";
    case SJ_ERR_OOM: return "out of device memory or over the workspace limit";
    case SJ_ERR_CUDA: return "CUDA error";
    case SJ_ERR_TIMEOUT: return "device-side wait timed out";
    case SJ_ERR_UNSUPPORTED: return "unsupported configuration";
    case SJ_ERR_INTERNAL: return "internal error";
  }
  return "unknown status";
}

int sj_version(void) { return kVersion; }

}  // extern "C"
