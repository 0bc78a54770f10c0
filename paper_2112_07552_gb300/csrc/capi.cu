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
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
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

// Bump allocator over the handle's workspace.  A measuring arena hands out
// no memory and only counts the bytes a sequence of takes needs.
struct Arena {
  unsigned char *base = nullptr;
  size_t size = 0, used = 0;
  bool measure = false;
  void *take(size_t bytes) {
    size_t off = align_up(used, 256);
    if (measure) {
      used = off + bytes;
      return reinterpret_cast<void *>((uintptr_t)(off + 256));
    }
    if (off + bytes > size) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

// Where a caller's pointer lives.  Device memory of another GPU is neither
// usable in place (no peer access is assumed) nor host memory to stage from.
enum class PtrKind { kHost, kDevice, kOtherDevice };

PtrKind ptr_kind(const void *p, int device) {
  if (!p) return PtrKind::kHost;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PtrKind::kHost;
  }
  if (at.type == cudaMemoryTypeManaged) return PtrKind::kDevice;
  if (at.type == cudaMemoryTypeDevice)
    return at.device == device ? PtrKind::kDevice : PtrKind::kOtherDevice;
  return PtrKind::kHost;
}

bool is_device_ptr(const void *p, int device) { return p && ptr_kind(p, device) == PtrKind::kDevice; }
bool is_other_device_ptr(const void *p, int device) {
  return p && ptr_kind(p, device) == PtrKind::kOtherDevice;
}

// gamma_n = n u / (1 - n u)
double gamma_n(double n, double u) { return n * u / (1.0 - n * u); }

}  // namespace

// A join pipeline captured as a CUDA graph, replayed for groups of the same
// shape (the key) while the workspace and the pinned tables stay in place.
struct GraphEntry {
  std::vector<int64_t> key;
  cudaGraphExec_t exec = nullptr;
};

struct sj_handle {
  sj_config cfg{};
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int cc = 0;
  void *ws = nullptr;
  size_t ws_size = 0;
  Counters *h_ctr = nullptr;   // pinned
  void *h_tab = nullptr;       // pinned: job/segment/unit tables, then per-job pair counts
  size_t h_tab_size = 0;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  std::vector<GraphEntry> graphs;
  std::map<std::pair<int, int>, int> tile_width;  // (k, right-side size class) -> tile width
  int force_bn = 0;                               // autotuner: width under test
  int64_t force_tps = 0;                          // planner census: a full join's split plan
  cudaEvent_t ev[6]{};
  cudaEvent_t gev[4]{};  // stage events recorded only by captured graphs
  sj::TcContext *tc = nullptr;
  float *dbg_raw = nullptr;     // sj_debug_scores: armed for the next one-job call
  float *dbg_margin = nullptr;
  sj_handle *aux = nullptr;     // relational calls: a handle of their one-hot width;
                                // cascade re-joins: a handle of the next precision
  bool wide_lists = false;      // cascade stage: band lists sized by the columns they cover
  int64_t rejoin_rows = 0;      // this call: rows re-joined by the next precision
  int64_t rejoin_rows_next = 0; // of those, rows the next stage re-joined once more
};

sj_status sj::aux_handle(sj_handle *h, int64_t d, sj_precision prec, sj_handle **out,
                         uint32_t extra_flags) {
  const uint32_t flags = (h->cfg.flags & ~(uint32_t)SJ_FLAG_SYM_INFONCE) | extra_flags;
  if (h->aux && (h->aux->cfg.d != d || h->aux->cfg.prec != prec || h->aux->cfg.flags != flags)) {
    sj_destroy(h->aux);
    h->aux = nullptr;
  }
  if (!h->aux) {
    sj_config c = h->cfg;
    c.d = d;
    c.prec = prec;
    c.flags = flags;
    sj_status s = sj_create(&h->aux, &c);
    if (s != SJ_OK) return s;
  }
  *out = h->aux;
  return SJ_OK;
}

int sj::handle_device(const sj_handle *h) { return h->cfg.device; }
const sj_config *sj::handle_config(const sj_handle *h) { return &h->cfg; }

void *sj::handle_stream(const sj_handle *h) { return h->stream; }
int sj::handle_sm_count(const sj_handle *h) { return h->sm_count; }

namespace {

sj_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SJ_OK;
  if (e == cudaErrorMemoryAllocation) return SJ_ERR_OOM;
  return SJ_ERR_CUDA;
}

// Detail of the last CUDA failure seen by this thread (sj_last_error_detail).
thread_local char g_err_detail[320] = "";

}  // namespace

void sj::record_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  std::snprintf(g_err_detail, sizeof g_err_detail, "%s at %s:%d (%s): %s",
                cudaGetErrorName(e), file, line, what, cudaGetErrorString(e));
}

namespace {

void note_cuda_error(cudaError_t e, const char *what, int line) {
  sj::record_cuda_error(e, what, "capi.cu", line);
}

#define SJ_CUDA(call)                          \
  do {                                         \
    cudaError_t e__ = (call);                  \
    if (e__ != cudaSuccess) {                  \
      note_cuda_error(e__, #call, __LINE__);   \
      return cuda_status(e__);                 \
    }                                          \
  } while (0)

void drop_graphs(sj_handle *h) {
  for (GraphEntry &g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

sj_status ensure_ws(sj_handle *h, size_t bytes) {
  if (bytes <= h->ws_size) return SJ_OK;
  if (h->cfg.workspace_limit && bytes > h->cfg.workspace_limit) return SJ_ERR_OOM;
  drop_graphs(h);  // captured pipelines hold workspace addresses
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
  } else if (p == SJ_FP8_E4M3) {
    q.fmt = PackFormat::kFP8;
    q.elem = 1;
    q.BM = kTcBM;
    q.BN = kTcBN;
    q.dp = round_up(d, 128);
    // Exact E4M3 x E4M3 products (8-bit significands) summed by the tensor
    // core, whose FP8 accumulation precision is not documented (earlier FP8
    // tensor cores kept about 14 significant bits while adding).  Allow every
    // one of the d + 32 additions a relative error of 2^-13 of the sum of
    // |products| (<= ||a~|| ||b~||): (d + 32) 2^-13.
    q.acc_coef = ((double)d + 32.0) * std::ldexp(1.0, -13);
  } else if (p == SJ_BF16X3) {
    q.fmt = PackFormat::kBF16X3;
    q.elem = 2;
    q.BM = kTcBM;
    q.BN = kTcBN;
    q.dp = round_up(3 * d, 64);
    // The BF16 allowance below over the 3d products of the split.
    q.acc_coef = (3.0 * (double)d + 32.0) * std::ldexp(1.0, -21);
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

struct Events {
  sj_handle *h;
  cudaStream_t st;
  bool capturing = false;  // record the graph-owned events as record nodes
  // Inside a stream capture, external records become event record nodes, so
  // stage times stay measurable when the pipeline replays as a graph; those
  // events belong to the graphs alone.
  void rec(int t) {
    if (capturing) cudaEventRecordWithFlags(h->gev[t], st, cudaEventRecordExternal);
    else cudaEventRecord(h->ev[t], st);
  }
  double ms(int a, int b) {
    float v = 0.f;
    cudaEvent_t *e = capturing ? h->gev : h->ev;
    if (cudaEventElapsedTime(&v, e[a], e[b]) != cudaSuccess) {
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

void fill_common_stats(sj_stats *st, const Counters &c) {
  st->n_candidates = (int64_t)c.n_candidates;
  st->n_rescored = (int64_t)c.n_rescored;
  st->n_exact = (int64_t)c.n_exact;
  st->n_overflow_rows = (int64_t)c.overflow_rows;
  st->n_tier2_rows = (int64_t)c.tier2_rows;
  float me, mm;
  std::memcpy(&me, &c.max_err_bits, sizeof me);
  std::memcpy(&mm, &c.max_margin_bits, sizeof mm);
  st->max_abs_err_lowprec = me;
  st->margin_max = mm;
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

sj_status check_req(const JoinReq &r) {
  if (r.nA < 0 || r.nB < 0) return SJ_ERR_INVALID_ARG;
  if ((r.nA > 0 && !r.A) || (r.nB > 0 && !r.B)) return SJ_ERR_INVALID_ARG;
  if (r.k < 0 || r.k > 1024 || (r.k > 0 && r.nA > 0 && (!r.out_idx || !r.out_score)))
    return SJ_ERR_INVALID_ARG;
  if (r.thr && (!r.n_out || r.capacity < 0 || std::isnan(r.tau) || (r.capacity > 0 && !r.out)))
    return SJ_ERR_INVALID_ARG;
  if (r.k == 0 && !r.thr) return SJ_ERR_INVALID_ARG;
  if (r.nA >= (1ll << 31) - 1024 || r.nB >= (1ll << 31) - 1024) return SJ_ERR_UNSUPPORTED;
  return SJ_OK;
}

// Host side of one job: where its pointers live.
struct JobHost {
  bool a_host, b_host, self, ot_host, op_host, nout_dev;
};

// The batch as the kernels see it (device tables) plus host bookkeeping.
struct BatchPlan {
  PrecPlan pp;
  int64_t d = 0;
  int bands = 1;
  std::vector<JobDev> jobs;
  std::vector<JobHost> host;
  std::vector<PackSeg> segs;
  std::vector<UnitDev> units;
  int64_t rows = 0, prows = 0, slots = 0, band_entries = 0, topv_entries = 0;
  int64_t rows_thr = 0, cap_sum = 0;
  double padded_pairs = 0.0;  // pair-scores the score tiles compute (incl. padding)
  int occ_words = 0;          // block-sparse scoring: bitmap words per 128-row group (0: dense)
  bool any_topk = false, any_thr = false, any_op_host = false;
};

// Size class of a right side: nB in (2^(c-1), 2^c].
int size_class(int64_t n) {
  int c = 0;
  while (c < 62 && ((int64_t)1 << c) < n) ++c;
  return c;
}

// Column tile width of a job on the tensor-core pass: the width under test
// while autotuning, the test hook, the autotuned width of its (k, size
// class), else 128 columns for right sides of at most 128 rows and 256 above.
int tile_width(const sj_handle *h, int64_t nB, int k) {
  if (h->cfg.prec == SJ_FP32) return kSimtBN;
  if (h->force_bn) return h->force_bn;
  if (h->cfg.flags & SJ_FLAG_NARROW_TILES) return kTcBNNarrow;
  auto it = h->tile_width.find({k, size_class(nB)});
  if (it != h->tile_width.end()) return it->second;
  return nB <= kTcBNNarrow ? kTcBNNarrow : kTcBN;
}

// Column splits: a unit covers at most total_tiles / (2 SMs) column tiles, so
// a small batch still yields about two units per SM and a large one keeps
// units long (one band list per row and split).  At most 256 splits per job.
sj_status make_batch_plan(const sj_handle *h, const JoinReq *reqs, int n, BatchPlan &P) {
  P.d = h->cfg.d;
  P.pp = plan_prec(h->cfg.prec, P.d);
  P.bands = h->cfg.prec == SJ_FP32 ? 1 : 2;
  if ((h->cfg.flags & SJ_FLAG_BLOCK_SPARSE) && h->cfg.prec != SJ_FP32) {
    const int64_t nkb = P.pp.dp * P.pp.elem / 128;
    const int64_t words = (nkb + 31) / 32;
    if (words <= kOccMaxWords) P.occ_words = (int)words;
  }
  const int64_t BM = P.pp.BM, BN = P.pp.BN, edge = std::max(BM, BN);
  int64_t total_tiles = 0;
  for (int q = 0; q < n; ++q)
    if (reqs[q].nA > 0 && reqs[q].nB > 0)
      total_tiles += ((reqs[q].nA + BM - 1) / BM) * ((reqs[q].nB + BN - 1) / BN);
  const int64_t tps_target = std::max<int64_t>(1, total_tiles / (2 * (int64_t)h->sm_count));
  P.jobs.assign(n, JobDev{});
  P.host.assign(n, JobHost{});
  for (int q = 0; q < n; ++q) {
    const JoinReq &r = reqs[q];
    JobDev &jd = P.jobs[q];
    JobHost &hh = P.host[q];
    jd.nA = r.nA;
    jd.nB = r.nB;
    // a self-join shares one packed copy, except with the hi/lo split, whose
    // A and B rows are laid out differently
    hh.self = r.A == r.B && r.nA == r.nB && h->cfg.prec != SJ_BF16X3;
    const int dv = h->cfg.device;
    if (is_other_device_ptr(r.A, dv) || is_other_device_ptr(r.B, dv) ||
        is_other_device_ptr(r.out_idx, dv) || is_other_device_ptr(r.out_score, dv) ||
        is_other_device_ptr(r.out, dv) || is_other_device_ptr(r.n_out, dv))
      return SJ_ERR_INVALID_ARG;
    hh.a_host = r.nA > 0 && !is_device_ptr(r.A, dv);
    hh.b_host = !hh.self && r.nB > 0 && !is_device_ptr(r.B, dv);
    hh.ot_host = r.k > 0 && r.nA > 0 &&
                 (!is_device_ptr(r.out_idx, dv) || !is_device_ptr(r.out_score, dv));
    hh.op_host = r.thr && r.capacity > 0 && !is_device_ptr(r.out, dv);
    hh.nout_dev = r.thr && is_device_ptr(r.n_out, dv);
    jd.row0 = P.rows;
    P.rows += r.nA;
    // packed segments (zero-row segments are left out)
    if (hh.self) {
      jd.a_prow0 = jd.b_prow0 = P.prows;
      if (r.nA > 0) P.segs.push_back(PackSeg{nullptr, r.nA, P.prows, q, 2});
      P.prows += round_up(r.nA, edge);
    } else {
      jd.a_prow0 = P.prows;
      if (r.nA > 0) P.segs.push_back(PackSeg{nullptr, r.nA, P.prows, q, 0});
      P.prows += round_up(r.nA, BM);
      jd.b_prow0 = P.prows;
      if (r.nB > 0) P.segs.push_back(PackSeg{nullptr, r.nB, P.prows, q, 1});
      P.prows += round_up(r.nB, BN);
    }
    const int64_t bn = tile_width(h, r.nB, r.k);
    const int64_t rb = (r.nA + BM - 1) / BM, ct = (r.nB + bn - 1) / bn;
    jd.bn = (int32_t)bn;
    int64_t S = 0, tps = 1;
    if (rb > 0 && ct > 0) {
      // tps_target counts tiles of BN columns
      tps = (h->cfg.flags & SJ_FLAG_SINGLE_SPLIT) ? ct : std::min(ct, tps_target * (BN / bn));
      if (h->force_tps > 0) tps = std::min<int64_t>(ct, h->force_tps);
      if ((ct + tps - 1) / tps > 256) tps = (ct + 255) / 256;
      S = (ct + tps - 1) / tps;
    }
    jd.n_col_tiles = (int32_t)ct;
    P.padded_pairs += (double)(rb * BM) * (double)(ct * bn);
    jd.tiles_per_split = (int32_t)tps;
    jd.n_splits = (int32_t)S;
    jd.k = r.k;
    // Band list per (row, list): the k best plus the margin band plus room for
    // one round of visits (64).  With an exact running k-th (tensor-core path,
    // k <= 32) the margin band is the only slack: up to about k entries where
    // the k-th score lies in the bulk of a short row, and growing with the
    // columns a list covers (about 60-150 entries for 500k columns of d = 768
    // BF16 scores), so it is sized at k + columns / 2048, the latter within
    // [32, 192].  Lists are
    // kept short on purpose: the lists of the rows in flight (152 CTAs x 128
    // rows x 2) compete with the operand tiles for L2, and a list that still
    // overflows after compaction goes to the rescan fallback.  Otherwise the
    // running k-th is refreshed lazily and needs 4k + 256.
    // A cascade stage (wide_lists) re-joins rows whose bands overflowed the
    // lists of a coarser precision: its lists grow with the columns they
    // cover (1/8 of them, at most 2,048 more entries), as the dense band of
    // those rows does: each list tracks its own k-th best, below the row's, so
    // its band holds a fixed share of its columns (about 6% for the rows of
    // one tight cluster under the hi/lo split's margin).
    if (r.k > 0) {
      const int64_t cols = tps * bn / P.bands;
      const bool exact_running = h->cfg.prec != SJ_FP32 && r.k <= kTcExactMaxK;
      const int64_t slack =
          h->wide_lists ? std::min<int64_t>(2048, std::max<int64_t>(32, cols / 8))
                        : std::min<int64_t>(192, std::max<int64_t>(32, cols / 2048));
      jd.cap = (int32_t)(exact_running ? round_up(2 * (int64_t)r.k + 64 + slack, 32)
                                       : round_up(4 * (int64_t)r.k + 256 +
                                                      (h->wide_lists ? slack : 0), 32));
    } else {
      jd.cap = 0;
    }
    jd.lists = r.k > 0 ? (int32_t)(S * P.bands) : 0;
    jd.slot0 = P.slots;
    jd.band0 = P.band_entries;
    P.slots += r.nA * jd.lists;
    P.band_entries += r.nA * jd.lists * (int64_t)jd.cap;
    // exact per-list top-k values (tensor-core epilogue, k <= 32)
    jd.topv0 = -1;
    if (r.k > 0 && r.k <= kTcExactMaxK && h->cfg.prec != SJ_FP32) {
      jd.topv0 = P.topv_entries;
      P.topv_entries += r.nA * jd.lists * (int64_t)r.k;
    }
    for (int64_t b = 0; b < rb; ++b)
      for (int64_t sp = 0; sp < S; ++sp) P.units.push_back(UnitDev{q, (int32_t)b, (int32_t)sp, 0});
    // |s| <= ||a|| ||b|| < 1.00001 for validated rows: clamping tau to [-4, 4]
    // changes no decision and keeps it inside the key and exact ranges.
    jd.tau_f = INFINITY;
    if (r.thr) {
      const double tc = std::min(4.0, std::max(-4.0, r.tau));
      float tf = (float)tc;
      if ((double)tf > tc) tf = std::nextafter(tf, -INFINITY);
      jd.tau_f = tf;
      jd.tau_key = (long long)std::ceil(std::ldexp(tc, kKeyShift));
      jd.tau_exact = tau_to_exact(tc);
      P.rows_thr += r.nA;
      P.cap_sum += r.capacity;
      P.any_thr = true;
      P.any_op_host |= hh.op_host;
    }
    P.any_topk |= r.k > 0;
    jd.capacity = r.thr ? r.capacity : 0;
  }
  if (P.rows >= (1ll << 31) - 1024 || P.prows >= (1ll << 31) - 1024) return SJ_ERR_UNSUPPORTED;
  // Job-major unit order, jobs by decreasing unit length: the persistent grid
  // takes units round-robin, so CTAs running at the same time work on the same
  // job and share its B tiles in L2, and the schedule ends with the shortest
  // units.
  if (n > 1) {
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      return P.jobs[x].tiles_per_split > P.jobs[y].tiles_per_split;
    });
    std::vector<int64_t> first(n + 1, 0);
    for (int q = 0; q < n; ++q) {
      const JobDev &jd = P.jobs[q];
      first[q + 1] = first[q] + (jd.nA > 0 && jd.nB > 0 ? ((jd.nA + BM - 1) / BM) * jd.n_splits : 0);
    }
    std::vector<UnitDev> sorted;
    sorted.reserve(P.units.size());
    for (int q : order)
      sorted.insert(sorted.end(), P.units.begin() + first[q], P.units.begin() + first[q + 1]);
    P.units.swap(sorted);
  }
  return SJ_OK;
}

// Byte offsets of the job, segment and unit tables in one block.
struct TableLayout {
  size_t segs, units, bytes;
};
TableLayout table_layout(const BatchPlan &P) {
  TableLayout t;
  t.segs = align_up(sizeof(JobDev) * std::max<size_t>(P.jobs.size(), 1), 256);
  t.units = t.segs + align_up(sizeof(PackSeg) * std::max<size_t>(P.segs.size(), 1), 256);
  t.bytes = t.units + sizeof(UnitDev) * std::max<size_t>(P.units.size(), 1);
  return t;
}

// Device buffers of one call, carved from the workspace.  The same sequence of
// takes runs once on a measuring arena to size the workspace.
struct Bufs {
  Counters *ctr = nullptr;
  JobDev *jobs = nullptr;
  PackSeg *segs = nullptr;
  UnitDev *units = nullptr;
  RowMeta *meta = nullptr;
  void *packed = nullptr;
  std::vector<float *> stA, stB;
  uint32_t *occ = nullptr;
  Cand *band = nullptr;
  float *topv = nullptr;
  int *band_cnt = nullptr, *defer = nullptr, *tier2 = nullptr, *ovf = nullptr;
  int *ovf_band = nullptr;
  long long *ovf_key = nullptr;
  std::vector<int64_t *> st_idx;
  std::vector<float *> st_score;
  ThrCand *cand = nullptr, *acc = nullptr;
  int64_t *row_count = nullptr, *row_off = nullptr, *row_fill = nullptr, *total = nullptr;
  int *big_rows = nullptr, *n_big = nullptr;
  void *scan = nullptr;
  int64_t *job_info = nullptr;
  PairOut *staging = nullptr, *tmp = nullptr;
};

bool layout(Arena &ar, const BatchPlan &P, const JoinReq *reqs, unsigned long long thr_cap,
            Bufs &B) {
  const int n = (int)P.jobs.size();
  const int64_t rows1 = std::max<int64_t>(P.rows, 1);
  bool ok = true;
  auto take = [&](size_t bytes) {
    void *p = ar.take(bytes);
    ok = ok && p;
    return p;
  };
  B.ctr = static_cast<Counters *>(take(sizeof(Counters)));
  // job, segment and unit tables back to back (one copy from the pinned host
  // tables, same offsets)
  const TableLayout tl = table_layout(P);
  unsigned char *tab = static_cast<unsigned char *>(take(tl.bytes));
  B.jobs = reinterpret_cast<JobDev *>(tab);
  B.segs = reinterpret_cast<PackSeg *>(tab + tl.segs);
  B.units = reinterpret_cast<UnitDev *>(tab + tl.units);
  B.meta = static_cast<RowMeta *>(take(sizeof(RowMeta) * std::max<int64_t>(P.prows, 1)));
  B.packed = take((size_t)std::max<int64_t>(P.prows, 1) * P.pp.dp * P.pp.elem);
  if (P.occ_words > 0)
    B.occ = static_cast<uint32_t *>(take((size_t)(P.prows / 128 + 1) * P.occ_words * 4));
  B.stA.assign(n, nullptr);
  B.stB.assign(n, nullptr);
  B.st_idx.assign(n, nullptr);
  B.st_score.assign(n, nullptr);
  for (int q = 0; q < n; ++q) {
    if (P.host[q].a_host) B.stA[q] = static_cast<float *>(take((size_t)reqs[q].nA * P.d * 4));
    if (P.host[q].b_host) B.stB[q] = static_cast<float *>(take((size_t)reqs[q].nB * P.d * 4));
  }
  if (P.any_topk) {
    B.band = static_cast<Cand *>(take(sizeof(Cand) * std::max<int64_t>(P.band_entries, 1)));
    B.band_cnt = static_cast<int *>(take(4 * (size_t)std::max<int64_t>(P.slots, 1)));
    B.topv = static_cast<float *>(take(4 * (size_t)std::max<int64_t>(P.topv_entries, 1)));
    B.defer = static_cast<int *>(take(4 * (size_t)rows1));
    B.tier2 = static_cast<int *>(take(4 * (size_t)rows1));
    B.ovf = static_cast<int *>(take(4 * (size_t)rows1));
    B.ovf_key = static_cast<long long *>(take(8 * (size_t)rows1));
    B.ovf_band = static_cast<int *>(take(4 * (size_t)rows1));
    for (int q = 0; q < n; ++q)
      if (P.host[q].ot_host) {
        B.st_idx[q] = static_cast<int64_t *>(take((size_t)reqs[q].nA * reqs[q].k * 8));
        B.st_score[q] = static_cast<float *>(take((size_t)reqs[q].nA * reqs[q].k * 4));
      }
  }
  if (P.any_thr) {
    B.cand = static_cast<ThrCand *>(take((size_t)thr_cap * sizeof(ThrCand)));
    B.acc = static_cast<ThrCand *>(take((size_t)thr_cap * sizeof(ThrCand)));
    B.row_count = static_cast<int64_t *>(take(8 * (size_t)rows1));
    B.row_off = static_cast<int64_t *>(take(8 * (size_t)rows1));
    B.row_fill = static_cast<int64_t *>(take(8 * (size_t)rows1));
    B.total = static_cast<int64_t *>(take(64));
    B.big_rows = static_cast<int *>(take(4 * (size_t)rows1));
    B.n_big = static_cast<int *>(take(64));
    B.scan = take(scan_scratch_bytes(rows1));
    B.job_info = static_cast<int64_t *>(take(16 * (size_t)std::max(n, 1)));
    if (P.any_op_host) B.staging = static_cast<PairOut *>(take((size_t)thr_cap * sizeof(PairOut)));
    B.tmp = static_cast<PairOut *>(take((size_t)thr_cap * sizeof(PairOut)));
  }
  return ok;
}

// One rescan pass over rows[0 .. n) (local rows of one job; device arrays,
// with host copies of the rows in hrows) with lists of `cap` entries: rescan all of B
// with Dot2 against each row's key bound, then rank the lists (shared memory,
// or global memory for very long ones).  Rows whose list was cut off at `cap`
// are appended to redo_rows/redo_keys with the capacity they need.
sj_status topk_rescan_pass(sj_handle *h, Counters *ctr, const RowMeta *meta, const JobDev &jd,
                           int64_t d, const int *rows, const long long *keys, const int *hrows,
                           int n, int cap, const Cand *band, const int *band_cnt, Arena &ar,
                           int64_t &launches, std::vector<int> &redo_rows,
                           std::vector<long long> &redo_keys, int64_t &redo_cap) {
  cudaStream_t stm = h->stream;
  Scratch lists, count_s, redo_s, big_s, redo_k;
  SJ_CUDA(lists.get(ar, (size_t)n * cap * sizeof(KeyCand)));
  SJ_CUDA(count_s.get(ar, (size_t)n * 4 + 256));
  SJ_CUDA(redo_s.get(ar, (size_t)n * 4 + 256));
  SJ_CUDA(redo_k.get(ar, (size_t)n * 8 + 256));
  SJ_CUDA(big_s.get(ar, (size_t)n * 4 + 256));
  int *count = static_cast<int *>(count_s.p);
  SJ_CUDA(cudaMemsetAsync(count, 0, (size_t)n * 4, stm));
  SJ_CUDA(cudaMemsetAsync(&ctr->redo_rows, 0, 4 * sizeof(unsigned), stm));
  RescanArgs ra{};
  ra.A = jd.A;
  ra.B = jd.B;
  ra.nB = jd.nB;
  ra.d = d;
  ra.metaA = meta + jd.a_prow0;
  ra.metaB = meta + jd.b_prow0;
  ra.dot2_coef_key = dot2_coef_key(d);
  ra.rows = rows;
  ra.keys = keys;
  ra.n_rows = n;
  ra.lists = static_cast<KeyCand *>(lists.p);
  ra.count = count;
  ra.cap = cap;
  ra.ctr = ctr;
  if (band) {  // candidates from the rows' complete band lists
    ra.band = band + jd.band0;
    ra.band_cnt = band_cnt + jd.slot0;
    ra.band_lists = jd.lists;
    ra.band_cap = jd.cap;
  }
  SJ_CUDA(launch_topk_rescan(ra, stm));
  RankListArgs la{};
  la.A = jd.A;
  la.B = jd.B;
  la.d = d;
  la.k = jd.k;
  la.rows = rows;
  la.keys = keys;
  la.n_rows = n;
  la.lists = ra.lists;
  la.count = count;
  la.cap = cap;
  la.redo = static_cast<int *>(redo_s.p);
  la.redo_key = static_cast<long long *>(redo_k.p);
  la.big = static_cast<int *>(big_s.p);
  la.out_idx = jd.out_idx;
  la.out_score = jd.out_score;
  la.ctr = ctr;
  SJ_CUDA(launch_topk_rank_lists(la, stm));
  launches += 2;
  sj_status s = read_counters(h, ctr);
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
  if (n_redo > 0) {
    redo_cap = std::max<int64_t>(redo_cap, (int64_t)h->h_ctr->redo_cap);
    std::vector<int> slots(n_redo);
    std::vector<long long> tight(n_redo);
    SJ_CUDA(cudaMemcpyAsync(slots.data(), la.redo, n_redo * 4, cudaMemcpyDeviceToHost, stm));
    SJ_CUDA(cudaMemcpyAsync(tight.data(), la.redo_key, n_redo * 8, cudaMemcpyDeviceToHost, stm));
    SJ_CUDA(cudaStreamSynchronize(stm));
    for (unsigned q = 0; q < n_redo; ++q) {
      redo_rows.push_back(hrows[slots[q]]);
      redo_keys.push_back(tight[q]);
    }
  }
  return SJ_OK;
}

// Rows whose candidates did not fit (one job): rescan passes in chunks of
// rows whose lists fit in a bounded scratch (a list can hold all of B), first
// with 4,096-entry lists, then the cut-off rows once more with the capacity
// they need.  `rows`/`keys` are device arrays, hrows/hkeys their host copies.
// With `band` (rows whose band lists are complete) the candidates are the
// band entries instead of all of B.
sj_status topk_fallback(sj_handle *h, Counters *ctr, const RowMeta *meta, const JobDev &jd,
                        int64_t d, const int *rows, const long long *keys, const int *hrows,
                        const long long *hkeys, int n_rows, const Cand *band,
                        const int *band_cnt, Arena &ar, int64_t &launches) {
  cudaStream_t stm = h->stream;
  const size_t kScratch = (size_t)2 << 30;  // lists + global ranking per chunk
  const int64_t nB = jd.nB;
  std::vector<int> redo_rows;
  std::vector<long long> redo_keys;
  int64_t redo_cap = 0;
  auto run = [&](const int *dr, const long long *dk, const int *hr, const long long *hk, int n,
                 int cap, std::vector<int> &rr, std::vector<long long> &rk, int64_t &rc) {
    const size_t per_row = (size_t)cap * sizeof(KeyCand) + topk_rank_global_row_bytes(cap);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n, kScratch / per_row));
    for (int c0 = 0; c0 < n; c0 += chunk) {
      const int nc = std::min(chunk, n - c0);
      sj_status s = topk_rescan_pass(h, ctr, meta, jd, d, dr + c0, dk + c0, hr + c0, nc, cap,
                                     band, band_cnt, ar, launches, rr, rk, rc);
      if (s != SJ_OK) return s;
    }
    return SJ_OK;
  };
  // pass 1: lists of 4,096 entries; pass 2: the cut-off rows with their key
  // bounds tightened to the k-th best lower bound seen; pass 3: rows still cut
  // off (massive exact ties) with the capacity they need
  // a band scan's list cannot outgrow the row's band entries
  const int64_t most = band ? std::min<int64_t>(nB, (int64_t)jd.lists * jd.cap) : nB;
  const int cap0 = (int)std::min<int64_t>(most, 4096);
  sj_status s = run(rows, keys, hrows, hkeys, n_rows, cap0, redo_rows, redo_keys, redo_cap);
  std::vector<int> again;
  std::vector<long long> again_k;
  int64_t again_cap = 0;
  for (int pass = 2; pass <= 3 && s == SJ_OK && !redo_rows.empty(); ++pass) {
    const int n_redo = (int)redo_rows.size();
    Scratch rows2, keys2;
    SJ_CUDA(rows2.get(ar, (size_t)n_redo * 4 + 256));
    SJ_CUDA(keys2.get(ar, (size_t)n_redo * 8 + 256));
    SJ_CUDA(cudaMemcpyAsync(rows2.p, redo_rows.data(), (size_t)n_redo * 4, cudaMemcpyHostToDevice, stm));
    SJ_CUDA(cudaMemcpyAsync(keys2.p, redo_keys.data(), (size_t)n_redo * 8, cudaMemcpyHostToDevice, stm));
    SJ_CUDA(cudaStreamSynchronize(stm));
    again.clear();
    again_k.clear();
    again_cap = 0;
    const int cap = pass == 2 ? cap0 : (int)std::min<int64_t>(most, redo_cap);
    s = run(static_cast<int *>(rows2.p), static_cast<long long *>(keys2.p), redo_rows.data(),
            redo_keys.data(), n_redo, cap, again, again_k, again_cap);
    redo_rows.swap(again);
    redo_keys.swap(again_k);
    redo_cap = again_cap;
  }
  if (s != SJ_OK) return s;
  return redo_rows.empty() ? SJ_OK : SJ_ERR_INTERNAL;  // a list of all of B cannot be cut off
}

// The rows of one job to re-join, gathered into a dense matrix.
__global__ void gather_rows_kernel(const float *src, const int *rows, int n, int64_t d,
                                   float *dst) {
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const float *sr = src + (int64_t)rows[r] * d;
    float *o = dst + (int64_t)r * d;
    for (int64_t c = threadIdx.x; c < d; c += blockDim.x) o[c] = sr[c];
  }
}

// Top-k rows of the re-join back to their places in the job's outputs.
__global__ void scatter_topk_kernel(const int *rows, int n, int k, const int64_t *ii,
                                    const float *ss, int64_t *oi, float *os) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * k;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dst = (int64_t)rows[t / k] * k + t % k;
    oi[dst] = ii[t];
    os[dst] = ss[t];
  }
}

// Overflowed rows from this many up are re-joined by the next precision of
// the cascade instead of rescanned one by one (a 128-row tile serves them
// together).
constexpr int kRejoinMinRows = 64;

struct DevMem {
  void *p = nullptr;
  ~DevMem() {
    if (p) cudaFree(p);
  }
};

// Cascade step for rows whose band lists overflowed on a tensor-core pass:
// the dense band of near-ties below their k-th score, wider than the lists,
// comes from the margin of the low precision (BF16 (d + 32) 2^-21, E4M3
// (d + 32) 2^-13, the hi/lo split (3d + 32) 2^-21, times the norms and the
// quantisation terms).  The same rows re-joined against all of B in a
// precision with a narrower margin, or with longer lists, give complete
// candidate lists again:
//   * after a BF16, E4M3 or hi/lo-split pass with the usual lists, the BF16
//     hi/lo split on the tensor cores (quantisation terms near 2^-16 instead
//     of 2^-8 or 2^-4; three times the BF16 work) with band lists sized by
//     the columns they cover;
//   * after that, the FP32 form on the CUDA cores (2 gamma_d, about ten times
//     narrower again; 2 nB d flops per row on the FFMA tiles).
// Rows that overflow again go on down the cascade inside the re-join call.
// Either step replaces a Dot2 rescan of all of B per row.  The re-join runs
// through the handle's auxiliary handle (its own workspace: this call's
// buffers stay intact), in chunks of rows, and writes the rows' outputs in
// place.
sj_status rejoin_rows(sj_handle *h, const JobDev &jd, int64_t d, const int *rows, int n,
                      int64_t &launches) {
  const sj_precision next = h->cfg.prec == SJ_BF16X3 && h->wide_lists ? SJ_FP32 : SJ_BF16X3;
  sj_handle *ax = nullptr;
  sj_status s = sj::aux_handle(h, d, next, &ax);
  if (s != SJ_OK) return s;
  ax->wide_lists = next != SJ_FP32;
  cudaStream_t stm = h->stream;
  const int k = jd.k;
  const int chunk = std::min(n, 1 << 19);  // bounds the next stage's band lists
  DevMem ag, ii, ss;
  SJ_CUDA(cudaMalloc(&ag.p, (size_t)chunk * d * 4));
  SJ_CUDA(cudaMalloc(&ii.p, (size_t)chunk * k * 8));
  SJ_CUDA(cudaMalloc(&ss.p, (size_t)chunk * k * 4));
  for (int c0 = 0; c0 < n; c0 += chunk) {
    const int nc = std::min(chunk, n - c0);
    gather_rows_kernel<<<std::min(nc, 8192), 256, 0, stm>>>(jd.A, rows + c0, nc, d,
                                                          static_cast<float *>(ag.p));
    SJ_CUDA(cudaGetLastError());
    sj_stats st;
    s = sj_topk(ax, static_cast<const float *>(ag.p), nc, jd.B, jd.nB, k,
                static_cast<int64_t *>(ii.p), static_cast<float *>(ss.p), &st);
    if (s != SJ_OK) return s;
    const int64_t tot = (int64_t)nc * k;
    scatter_topk_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, stm>>>(
        rows + c0, nc, k, static_cast<int64_t *>(ii.p), static_cast<float *>(ss.p), jd.out_idx,
        jd.out_score);
    SJ_CUDA(cudaGetLastError());
    launches += 2 + st.n_launches;
    h->rejoin_rows += nc;
    h->rejoin_rows_next += st.n_rejoined_rows;
  }
  SJ_CUDA(cudaStreamSynchronize(stm));
  return SJ_OK;
}

// Fallback rows of the whole batch, grouped by job.
sj_status topk_fallback_all(sj_handle *h, const BatchPlan &P, const Bufs &B, unsigned n_ovf,
                            Arena &ar, int64_t &launches) {
  cudaStream_t stm = h->stream;
  std::vector<int> grow(n_ovf), gband(n_ovf);
  std::vector<long long> gkey(n_ovf);
  SJ_CUDA(cudaMemcpyAsync(grow.data(), B.ovf, (size_t)n_ovf * 4, cudaMemcpyDeviceToHost, stm));
  SJ_CUDA(cudaMemcpyAsync(gkey.data(), B.ovf_key, (size_t)n_ovf * 8, cudaMemcpyDeviceToHost, stm));
  SJ_CUDA(cudaMemcpyAsync(gband.data(), B.ovf_band, (size_t)n_ovf * 4, cudaMemcpyDeviceToHost,
                          stm));
  SJ_CUDA(cudaStreamSynchronize(stm));
  // (job * 2 + band-complete, index): rows of one job and kind are contiguous
  std::vector<std::pair<int, int>> by_job(n_ovf);
  for (unsigned t = 0; t < n_ovf; ++t) {
    auto it = std::upper_bound(P.jobs.begin(), P.jobs.end(), (int64_t)grow[t],
                               [](int64_t x, const JobDev &jd) { return x < jd.row0; });
    by_job[t] = {((int)(it - P.jobs.begin()) - 1) * 2 + (gband[t] ? 1 : 0), (int)t};
  }
  std::sort(by_job.begin(), by_job.end());
  Scratch rows_s, keys_s;
  SJ_CUDA(rows_s.get(ar, (size_t)n_ovf * 4 + 256));
  SJ_CUDA(keys_s.get(ar, (size_t)n_ovf * 8 + 256));
  std::vector<int> lrow(n_ovf);
  std::vector<long long> lkey(n_ovf);
  for (unsigned t = 0; t < n_ovf; ++t) {
    const int q = by_job[t].first / 2, src = by_job[t].second;
    lrow[t] = (int)(grow[src] - P.jobs[q].row0);
    lkey[t] = gkey[src];
  }
  SJ_CUDA(cudaMemcpyAsync(rows_s.p, lrow.data(), (size_t)n_ovf * 4, cudaMemcpyHostToDevice, stm));
  SJ_CUDA(cudaMemcpyAsync(keys_s.p, lkey.data(), (size_t)n_ovf * 8, cudaMemcpyHostToDevice, stm));
  SJ_CUDA(cudaStreamSynchronize(stm));
  for (unsigned t0 = 0; t0 < n_ovf;) {
    unsigned t1 = t0;
    while (t1 < n_ovf && by_job[t1].first == by_job[t0].first) ++t1;
    const JobDev &jd = P.jobs[by_job[t0].first / 2];
    const bool band = (by_job[t0].first & 1) != 0;
    sj_status s;
    if (!band && h->cfg.prec != SJ_FP32 && (int)(t1 - t0) >= kRejoinMinRows)
      s = rejoin_rows(h, jd, P.d, static_cast<int *>(rows_s.p) + t0, (int)(t1 - t0), launches);
    else
      s = topk_fallback(h, B.ctr, B.meta, jd, P.d, static_cast<int *>(rows_s.p) + t0,
                        static_cast<long long *>(keys_s.p) + t0, lrow.data() + t0,
                        lkey.data() + t0, (int)(t1 - t0), band ? B.band : nullptr, B.band_cnt,
                        ar, launches);
    if (s != SJ_OK) return s;
    t0 = t1;
  }
  return SJ_OK;
}

// All jobs of a batch share one validation/packing pass, one scoring launch
// and one finalisation pipeline.
// First size of the threshold candidate list (grown and rerun when exceeded).
unsigned long long initial_thr_cap(const BatchPlan &P) {
  if (!P.any_thr) return 0;
  return (unsigned long long)std::max<int64_t>(
      {(int64_t)1 << 16, 2 * P.rows_thr,
       std::min<int64_t>(P.cap_sum + P.cap_sum / 4, 32 * P.rows_thr + (1 << 20))});
}

// Pinned host tables: the job/segment/unit tables (table_layout offsets),
// then two int64 per job for the pair counts read back.
sj_status ensure_host_tables(sj_handle *h, size_t bytes) {
  if (bytes <= h->h_tab_size) return SJ_OK;
  drop_graphs(h);  // captured pipelines copy from this buffer
  if (h->h_tab) {
    SJ_CUDA(cudaStreamSynchronize(h->stream));
    cudaFreeHost(h->h_tab);
    h->h_tab = nullptr;
    h->h_tab_size = 0;
  }
  const size_t want = align_up(bytes + bytes / 4, 1 << 16);
  SJ_CUDA(cudaMallocHost(&h->h_tab, want));
  h->h_tab_size = want;
  return SJ_OK;
}

// Every device step of one group, asynchronous on `stm` and free of host
// reads, so that it can be captured as a graph: tables in, validation and
// packing, scoring with the fused filter, top-k finalisation (warp and CTA
// tiers), threshold rescoring, placement and ordering, then the counters and
// per-job pair counts back to pinned host memory.  Kernels skip their work
// once validation has flagged an input.
sj_status issue_group(sj_handle *h, cudaStream_t stm, bool capturing, const BatchPlan &P,
                      const Bufs &B, unsigned long long thr_cap, int64_t &launches) {
  const int n = (int)P.jobs.size();
  Events ev{h, stm, capturing};
  const TableLayout tl = table_layout(P);
  int64_t *h_info = reinterpret_cast<int64_t *>(static_cast<unsigned char *>(h->h_tab) +
                                                align_up(tl.bytes, 256));
  ev.rec(0);
  SJ_CUDA(cudaMemcpyAsync(B.jobs, h->h_tab, tl.bytes, cudaMemcpyHostToDevice, stm));
  SJ_CUDA(cudaMemsetAsync(B.ctr, 0, sizeof(Counters), stm));
  SJ_CUDA(launch_prepare(B.segs, (int)P.segs.size(), B.jobs, P.prows, P.d, P.pp.fmt, B.packed,
                         P.pp.dp, B.meta, B.ctr, stm));
  launches += P.prows > 0 ? (P.pp.fmt == PackFormat::kFP8 ? 2 : 1) : 0;
  if (B.occ && P.prows > 0) {
    SJ_CUDA(launch_occupancy(B.packed, P.prows, P.pp.dp * P.pp.elem, B.occ, P.occ_words, stm));
    launches += 1;
  }
  ev.rec(1);
  // ---- scoring pass with the fused filter ----
  if (P.any_topk && P.slots > 0) SJ_CUDA(cudaMemsetAsync(B.band_cnt, 0, (size_t)P.slots * 4, stm));
  if (!P.units.empty()) {
    ScoreArgs sa{};
    sa.jobs = B.jobs;
    sa.n_jobs = n;
    sa.units = B.units;
    sa.n_units = (int64_t)P.units.size();
    sa.Ap = B.packed;
    sa.Bp = B.packed;
    sa.dp = P.pp.dp;
    sa.metaA = B.meta;
    sa.acc_coef = (float)P.pp.acc_coef;
    sa.bands_per_split = P.bands;
    sa.band = B.band;
    sa.band_cnt = B.band_cnt;
    sa.topv = B.topv;
    sa.thr = B.cand;
    sa.thr_cap = thr_cap;
    sa.ctr = B.ctr;
    sa.raw = h->dbg_raw;
    sa.raw_m = h->dbg_margin;
    sa.occ = B.occ;
    sa.occ_words = P.occ_words;
    if (h->cfg.prec == SJ_FP32) {
      const int grid = (int)std::min<int64_t>(sa.n_units, (int64_t)h->sm_count * 2);
      SJ_CUDA(launch_score_simt(sa, grid, stm));
    } else {
      TcMaps maps;
      sj_status s = tc_make_maps(h->tc, B.packed, P.prows, B.packed, P.prows, P.pp.dp, &maps,
                                 P.pp.elem);
      if (s != SJ_OK) return s;
      const int grid = (int)std::min<int64_t>(sa.n_units, (int64_t)h->sm_count);
      SJ_CUDA(launch_score_tc(sa, grid, &maps, h->cfg.flags, h->cfg.prec == SJ_FP8_E4M3, stm));
    }
    launches += 1;
  }
  ev.rec(2);
  // ---- top-k finalisation (warp finaliser, two CTA tiers) ----
  if (P.any_topk) {
    TopkFinalArgs fa{};
    fa.jobs = B.jobs;
    fa.n_jobs = n;
    fa.rows = P.rows;
    fa.d = P.d;
    fa.metaA = B.meta;
    fa.metaB = B.meta;
    fa.acc_coef = (float)P.pp.acc_coef;
    fa.band = B.band;
    fa.band_cnt = B.band_cnt;
    fa.topv = B.topv;
    fa.dot2_coef_key = dot2_coef_key(P.d);
    fa.defer_rows = B.defer;
    fa.tier2_rows = B.tier2;
    fa.overflow_rows = B.ovf;
    fa.overflow_key = B.ovf_key;
    fa.overflow_band = B.ovf_band;
    fa.ctr = B.ctr;
    SJ_CUDA(launch_topk_finalize(fa, h->sm_count, stm));
    launches += P.rows > 0 ? 3 : 0;
  }
  // ---- threshold finalisation ----
  if (P.any_thr && P.rows > 0) {
    SJ_CUDA(cudaMemsetAsync(B.row_count, 0, (size_t)P.rows * 8, stm));
    SJ_CUDA(cudaMemsetAsync(B.row_fill, 0, (size_t)P.rows * 8, stm));
    SJ_CUDA(cudaMemsetAsync(B.n_big, 0, sizeof(int), stm));
    // candidates grouped by row into B.acc (counts in row_fill, offsets in
    // row_off; both are reset or rewritten below), then rescored from there
    // with the accepted pairs written over B.cand
    const int g_sc = (int)std::min<unsigned long long>((thr_cap + 255) / 256,
                                                       (unsigned long long)h->sm_count * 16);
    SJ_CUDA(launch_thr_bucket(B.cand, &B.ctr->thr_count, (int64_t)thr_cap, B.ctr, P.rows,
                              B.row_fill, B.row_off, B.total, B.scan, B.acc, g_sc, stm));
    SJ_CUDA(cudaMemsetAsync(B.row_fill, 0, (size_t)P.rows * 8, stm));
    ThrFinalArgs ta{};
    ta.jobs = B.jobs;
    ta.n_jobs = n;
    ta.d = P.d;
    ta.metaA = B.meta;
    ta.metaB = B.meta;
    ta.dot2_coef_key = dot2_coef_key(P.d);
    ta.cand = B.acc;
    ta.n_cand = &B.ctr->thr_count;
    ta.cand_cap = (int64_t)thr_cap;
    ta.row_count = B.row_count;
    ta.accepted = B.cand;
    ta.ctr = B.ctr;
    const int g_res = (int)std::min<unsigned long long>((thr_cap + 31) / 32,
                                                        (unsigned long long)h->sm_count * 16);
    SJ_CUDA(launch_thr_rescore(ta, g_res, stm));
    SJ_CUDA(launch_exclusive_scan(B.row_count, B.row_off, P.rows, B.total, B.scan, stm));
    SJ_CUDA(launch_job_pairs(B.jobs, n, P.rows, B.row_off, B.total, B.job_info, stm));
    SJ_CUDA(launch_thr_scatter(B.jobs, n, B.cand, &B.ctr->n_pairs, (int64_t)thr_cap, B.row_off,
                               B.row_fill, B.staging, g_sc, stm));
    SJ_CUDA(launch_thr_sort_rows(B.jobs, n, P.rows, B.row_off, B.row_count, B.staging,
                                 B.big_rows, B.n_big, stm));
    SJ_CUDA(launch_thr_sort_big(B.jobs, n, B.staging, B.tmp, B.row_off, B.row_count, B.big_rows,
                                B.n_big, 2 * h->sm_count, stm));
    launches += 14;
    SJ_CUDA(cudaMemcpyAsync(h_info, B.job_info, 16 * (size_t)n, cudaMemcpyDeviceToHost, stm));
  }
  SJ_CUDA(cudaMemcpyAsync(h->h_ctr, B.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, stm));
  ev.rec(3);
  return SJ_OK;
}

// Kernels issue_group launches for this plan.
void issue_count(const BatchPlan &P, int64_t &l) {
  l += P.prows > 0 ? (P.pp.fmt == PackFormat::kFP8 ? 2 : 1) : 0;
  l += P.prows > 0 && P.occ_words > 0 ? 1 : 0;
  l += P.units.empty() ? 0 : 1;
  l += P.any_topk && P.rows > 0 ? 3 : 0;
  l += P.any_thr && P.rows > 0 ? 9 : 0;
}

// Shape of a group as far as a captured pipeline depends on it.
std::vector<int64_t> graph_key(const sj_handle *h, const BatchPlan &P, const JoinReq *reqs,
                               unsigned long long thr_cap) {
  std::vector<int64_t> key;
  key.reserve(8 + 4 * P.jobs.size());
  key.push_back((int64_t)(uintptr_t)h->ws);
  key.push_back((int64_t)h->ws_size);
  key.push_back((int64_t)(uintptr_t)h->h_tab);
  key.push_back((int64_t)thr_cap);
  key.push_back((int64_t)h->cfg.flags);
  key.push_back((int64_t)P.jobs.size());
  for (size_t q = 0; q < P.jobs.size(); ++q) {
    key.push_back(reqs[q].nA);
    key.push_back(reqs[q].nB);
    key.push_back(((int64_t)reqs[q].k << 2) | (reqs[q].thr ? 2 : 0) | (P.host[q].self ? 1 : 0));
    key.push_back(P.jobs[q].bn);
  }
  return key;
}

// Launch the group's pipeline: a captured graph when every input and output
// is in device memory (captured on first use of the shape, then replayed),
// else the launches themselves.
sj_status run_group_device(sj_handle *h, const BatchPlan &P, const Bufs &B, const JoinReq *reqs,
                           unsigned long long thr_cap, bool graphable, int64_t &launches,
                           bool &used_graph) {
  used_graph = false;
  if (!graphable) return issue_group(h, h->stream, false, P, B, thr_cap, launches);
  std::vector<int64_t> key = graph_key(h, P, reqs, thr_cap);
  for (GraphEntry &g : h->graphs)
    if (g.key == key) {
      SJ_CUDA(cudaGraphLaunch(g.exec, h->stream));
      used_graph = true;
      int64_t l = 0;  // same launch count as the captured sequence
      issue_count(P, l);
      launches += l;
      return SJ_OK;
    }
  if (!h->cap_stream) SJ_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  // the captured copies read the pinned tables when the graph runs; the
  // tables are rewritten only after the previous call drained its stream
  cudaGraph_t graph = nullptr;
  SJ_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int64_t l = 0;
  sj_status s = issue_group(h, h->cap_stream, true, P, B, thr_cap, l);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (s != SJ_OK || e != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return issue_group(h, h->stream, false, P, B, thr_cap, launches);
  }
  GraphEntry ent;
  ent.key = std::move(key);
  e = cudaGraphInstantiate(&ent.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return issue_group(h, h->stream, false, P, B, thr_cap, launches);
  }
  if (h->graphs.size() >= 8) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(std::move(ent));
  SJ_CUDA(cudaGraphLaunch(h->graphs.back().exec, h->stream));
  used_graph = true;
  launches += l;
  return SJ_OK;
}

// One group of jobs as one pipeline (inputs already validated).
sj_status join_group(sj_handle *h, const JoinReq *reqs, int n, sj_stats *st) {
  if (st) std::memset(st, 0, sizeof *st);
  if (n == 0) return SJ_OK;
  h->rejoin_rows = h->rejoin_rows_next = 0;
  cudaStream_t stm = h->stream;
  Events ev{h, stm};
  int64_t launches = 0;
  BatchPlan P;
  sj_status s = make_batch_plan(h, reqs, n, P);
  if (s != SJ_OK) return s;
  unsigned long long thr_cap = initial_thr_cap(P);
  bool any_host = false;
  for (const JobHost &hh : P.host) any_host |= hh.a_host || hh.b_host || hh.ot_host || hh.op_host;
  const bool graphable = !any_host && !(h->cfg.flags & SJ_FLAG_NO_GRAPH) && !h->dbg_raw;
  const TableLayout tl = table_layout(P);
  s = ensure_host_tables(h, align_up(tl.bytes, 256) + 16 * (size_t)n);
  if (s != SJ_OK) return s;
  int64_t *h_info = reinterpret_cast<int64_t *>(static_cast<unsigned char *>(h->h_tab) +
                                                align_up(tl.bytes, 256));

  for (int attempt = 0; attempt < 3; ++attempt) {
    Bufs B;
    {
      Arena meas;
      meas.measure = true;
      layout(meas, P, reqs, thr_cap, B);
      s = ensure_ws(h, meas.used + 4096);
      if (s != SJ_OK) return s;
    }
    Arena ar{static_cast<unsigned char *>(h->ws), h->ws_size, 0};
    if (!layout(ar, P, reqs, thr_cap, B)) return SJ_ERR_INTERNAL;
    // device pointers of every job; host inputs staged into the workspace
    for (int q = 0; q < n; ++q) {
      const JoinReq &r = reqs[q];
      JobDev &jd = P.jobs[q];
      const JobHost &hh = P.host[q];
      jd.A = hh.a_host ? B.stA[q] : r.A;
      jd.B = hh.self ? jd.A : (hh.b_host ? B.stB[q] : r.B);
      jd.out_idx = hh.ot_host ? B.st_idx[q] : r.out_idx;
      jd.out_score = hh.ot_host ? B.st_score[q] : r.out_score;
      jd.out_pairs = (r.thr && !hh.op_host && r.capacity > 0) ? reinterpret_cast<PairOut *>(r.out)
                                                              : nullptr;
      jd.gmaxB[0] = jd.gmaxB[1] = jd.gmaxB[2] = jd.gmaxB[3] = 0.f;
      jd.bmax = 0.f;
      jd.eB = 0;
      jd.n_pairs = 0;
      if (hh.a_host)
        SJ_CUDA(cudaMemcpyAsync(B.stA[q], r.A, (size_t)r.nA * P.d * 4, cudaMemcpyHostToDevice, stm));
      if (hh.b_host)
        SJ_CUDA(cudaMemcpyAsync(B.stB[q], r.B, (size_t)r.nB * P.d * 4, cudaMemcpyHostToDevice, stm));
    }
    for (PackSeg &sg : P.segs) sg.src = sg.side == 1 ? P.jobs[sg.job].B : P.jobs[sg.job].A;
    unsigned char *tab = static_cast<unsigned char *>(h->h_tab);
    std::memcpy(tab, P.jobs.data(), sizeof(JobDev) * n);
    if (!P.segs.empty()) std::memcpy(tab + tl.segs, P.segs.data(), sizeof(PackSeg) * P.segs.size());
    if (!P.units.empty())
      std::memcpy(tab + tl.units, P.units.data(), sizeof(UnitDev) * P.units.size());
    std::memset(h_info, 0, 16 * (size_t)n);
    bool used_graph = false;
    s = run_group_device(h, P, B, reqs, thr_cap, graphable && attempt == 0, launches, used_graph);
    if (s != SJ_OK) return s;
    SJ_CUDA(cudaStreamSynchronize(stm));
    const Counters c1 = *h->h_ctr;
    s = flags_status(c1.err_flags);
    if (s != SJ_OK) return s;
    if (P.any_thr && c1.thr_count > thr_cap) {
      // rerun with room for every candidate (and without the captured graph)
      thr_cap = c1.thr_count + c1.thr_count / 8 + 1024;
      continue;
    }
    if (P.any_topk && c1.overflow_rows > 0) {
      s = topk_fallback_all(h, P, B, c1.overflow_rows, ar, launches);
      if (s != SJ_OK) return s;
    }
    for (int q = 0; q < n; ++q)
      if (P.host[q].ot_host) {
        const size_t e = (size_t)reqs[q].nA * reqs[q].k;
        SJ_CUDA(cudaMemcpyAsync(reqs[q].out_idx, B.st_idx[q], e * 8, cudaMemcpyDeviceToHost, stm));
        SJ_CUDA(cudaMemcpyAsync(reqs[q].out_score, B.st_score[q], e * 4, cudaMemcpyDeviceToHost, stm));
      }
    int64_t n_pairs_all = 0;
    bool over_cap = false;
    for (int q = 0; q < n; ++q) {
      const JoinReq &r = reqs[q];
      if (!r.thr) continue;
      const int64_t np = h_info[2 * q], off = h_info[2 * q + 1];
      n_pairs_all += np;
      if (P.host[q].nout_dev) {
        SJ_CUDA(cudaMemcpyAsync(r.n_out, &h_info[2 * q], 8, cudaMemcpyHostToDevice, stm));
      } else {
        *r.n_out = np;
      }
      if (np > r.capacity) {
        over_cap = true;
      } else if (np > 0 && P.host[q].op_host) {
        SJ_CUDA(cudaMemcpyAsync(r.out, B.staging + off, (size_t)np * sizeof(PairOut),
                                cudaMemcpyDeviceToHost, stm));
      }
    }
    s = read_counters(h, B.ctr);  // drains the stream; counters after any fallback
    if (s != SJ_OK) return s;
    if (st) {
      fill_common_stats(st, *h->h_ctr);
      st->n_candidates += (int64_t)c1.thr_count;
      st->n_pairs = n_pairs_all;
      st->n_launches = launches;
      ev.capturing = used_graph;  // read the graph-owned events after a replay
      st->ms_prepare = ev.ms(0, 1);
      st->ms_score = ev.ms(1, 2);
      st->ms_select = ev.ms(2, 3);
      st->ms_total = ev.ms(0, 3);
      st->graph_replayed = used_graph ? 1 : 0;
      st->padded_pair_scores = P.padded_pairs;
      st->n_rejoined_rows = h->rejoin_rows;
      st->n_rejoined_again = h->rejoin_rows_next;
    }
    s = flags_status(h->h_ctr->err_flags);
    if (s != SJ_OK) return s;
    return over_cap ? SJ_ERR_CAPACITY : SJ_OK;
  }
  return SJ_ERR_INTERNAL;
}

// Workspace bytes of one group of jobs as planned.
size_t group_bytes(const sj_handle *h, const JoinReq *reqs, int n, sj_status &s) {
  BatchPlan P;
  s = make_batch_plan(h, reqs, n, P);
  if (s != SJ_OK) return 0;
  Arena meas;
  meas.measure = true;
  Bufs B;
  layout(meas, P, reqs, initial_thr_cap(P), B);
  return meas.used + 4096;
}

void add_stats(sj_stats *acc, const sj_stats &one) {
  acc->ms_prepare += one.ms_prepare;
  acc->ms_score += one.ms_score;
  acc->ms_select += one.ms_select;
  acc->ms_total += one.ms_total;
  acc->n_candidates += one.n_candidates;
  acc->n_rescored += one.n_rescored;
  acc->n_exact += one.n_exact;
  acc->n_overflow_rows += one.n_overflow_rows;
  acc->n_pairs += one.n_pairs;
  acc->n_launches += one.n_launches;
  acc->n_tier2_rows += one.n_tier2_rows;
  acc->graph_replayed += one.graph_replayed;
  acc->padded_pair_scores += one.padded_pair_scores;
  acc->n_rejoined_rows += one.n_rejoined_rows;
  acc->n_rejoined_again += one.n_rejoined_again;
  acc->max_abs_err_lowprec = std::max(acc->max_abs_err_lowprec, one.max_abs_err_lowprec);
  acc->margin_max = std::max(acc->margin_max, one.margin_max);
}

// Jobs [lo, hi) in as few groups as the workspace budget allows: a range
// that does not fit is halved by rows (nA + nB) until it does.  A single job
// over the budget runs alone (and may fail with SJ_ERR_OOM).
sj_status run_range(sj_handle *h, const JoinReq *reqs, int lo, int hi, size_t budget,
                    sj_stats *acc) {
  if (hi - lo > 1) {
    sj_status s = SJ_OK;
    const size_t bytes = group_bytes(h, reqs + lo, hi - lo, s);
    if (s != SJ_OK) return s;
    if (bytes > budget) {
      int64_t tot = 0;
      for (int q = lo; q < hi; ++q) tot += reqs[q].nA + reqs[q].nB + 1;
      int mid = lo + 1;
      for (int64_t run = 0; mid < hi - 1; ++mid) {
        run += reqs[mid - 1].nA + reqs[mid - 1].nB + 1;
        if (2 * run >= tot) break;
      }
      sj_status s1 = run_range(h, reqs, lo, mid, budget, acc);
      if (s1 != SJ_OK && s1 != SJ_ERR_CAPACITY) return s1;
      sj_status s2 = run_range(h, reqs, mid, hi, budget, acc);
      if (s2 != SJ_OK) return s2;
      return s1;
    }
  }
  sj_stats one;
  sj_status s = join_group(h, reqs + lo, hi - lo, &one);
  add_stats(acc, one);
  return s;
}

sj_status join_batch(sj_handle *h, const JoinReq *reqs, int n, sj_stats *st) {
  if (!h || n < 0 || (n > 0 && !reqs)) return SJ_ERR_INVALID_ARG;
  for (int q = 0; q < n; ++q) {
    sj_status s = check_req(reqs[q]);
    if (s != SJ_OK) return s;
  }
  sj_stats acc{};
  if (n == 0) {
    if (st) *st = acc;
    return SJ_OK;
  }
  SJ_CUDA(cudaSetDevice(h->cfg.device));
  size_t budget = h->cfg.workspace_limit;
  if (!budget) {
    size_t free_b = 0, total_b = 0;
    SJ_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t reserve = std::max<size_t>((size_t)1 << 30, total_b / 50);
    const size_t avail = free_b + h->ws_size;
    budget = avail > reserve ? avail - reserve : 0;
  }
  sj_status s = (h->dbg_raw && n != 1) ? SJ_ERR_INVALID_ARG
                                       : run_range(h, reqs, 0, n, budget, &acc);
  h->dbg_raw = h->dbg_margin = nullptr;  // the test hook arms one call
  if (st) *st = acc;
  return s;
}

sj_status topk_impl(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                    int32_t k, int64_t *out_idx, float *out_score, sj_stats *st) {
  if (!h) return SJ_ERR_INVALID_ARG;
  if (k < 1) return SJ_ERR_INVALID_ARG;
  JoinReq r{A, nA, B, nB, k, out_idx, out_score, false, 0.0, nullptr, 0, nullptr};
  return join_batch(h, &r, 1, st);
}

sj_status threshold_impl(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                         double tau, sj_pair *out, int64_t capacity, int64_t *n_out,
                         sj_stats *st) {
  if (!h) return SJ_ERR_INVALID_ARG;
  JoinReq r{A, nA, B, nB, 0, nullptr, nullptr, true, tau, out, capacity, n_out};
  return join_batch(h, &r, 1, st);
}

// ---------------------------------------------------------------------------
// Autotuner of the column tile width per right-side size class.

// Unit-norm rows for timing only: uniform entries from a 64-bit mix of
// (seed, row, column), normalised in double.  One thread per row.
__global__ void tune_rows_kernel(float *X, int64_t n, int64_t d, uint64_t seed) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  auto mix = [](uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    return x ^ (x >> 31);
  };
  double s = 0.0;
  for (int64_t c = 0; c < d; ++c) {
    const double u = (double)(mix(seed ^ mix((uint64_t)r * 0x9e3779b97f4a7c15ull + c)) >> 11) *
                         0x1p-53 * 2.0 - 1.0;
    s += u * u;
  }
  const double inv = 1.0 / sqrt(s > 0.0 ? s : 1.0);
  for (int64_t c = 0; c < d; ++c) {
    const double u = (double)(mix(seed ^ mix((uint64_t)r * 0x9e3779b97f4a7c15ull + c)) >> 11) *
                         0x1p-53 * 2.0 - 1.0;
    X[r * d + c] = (float)(u * inv);
  }
}

constexpr int kTuneClassLo = 6, kTuneClassHi = 16;  // right sides of 48 .. 49,152 rows
constexpr int64_t kTuneRowsA = 8192;

// Table file: one "d precision k class width" line per entry.
sj_status write_tile_table(const sj_handle *h, const char *path) {
  std::vector<std::string> keep;
  if (FILE *f = std::fopen(path, "r")) {
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
      long long d;
      int prec, k, c, w;
      if (std::sscanf(line, "%lld %d %d %d %d", &d, &prec, &k, &c, &w) != 5) continue;
      if (d == h->cfg.d && prec == (int)h->cfg.prec && h->tile_width.count({k, c})) continue;
      keep.push_back(line);
    }
    std::fclose(f);
  }
  FILE *f = std::fopen(path, "w");
  if (!f) return SJ_ERR_INVALID_ARG;
  for (const std::string &l : keep) std::fputs(l.c_str(), f);
  for (const auto &e : h->tile_width)
    std::fprintf(f, "%lld %d %d %d %d\n", (long long)h->cfg.d, (int)h->cfg.prec, e.first.first,
                 e.first.second, e.second);
  return std::fclose(f) == 0 ? SJ_OK : SJ_ERR_INVALID_ARG;
}

}  // namespace

extern "C" {

sj_status sj_autotune(sj_handle *h, int32_t k, const char *path) {
  if (!h || k < 1 || k > 1024) return SJ_ERR_INVALID_ARG;
  if (h->cfg.prec == SJ_FP32) return SJ_ERR_UNSUPPORTED;
  SJ_CUDA(cudaSetDevice(h->cfg.device));
  const int64_t d = h->cfg.d, nB_max = (int64_t)3 << (kTuneClassHi - 2);
  float *A = nullptr, *B = nullptr;
  int64_t *idx = nullptr;
  float *sc = nullptr;
  cudaError_t e = cudaMalloc(&A, (size_t)kTuneRowsA * d * 4);
  if (e == cudaSuccess) e = cudaMalloc(&B, (size_t)nB_max * d * 4);
  if (e == cudaSuccess) e = cudaMalloc(&idx, (size_t)kTuneRowsA * k * 8);
  if (e == cudaSuccess) e = cudaMalloc(&sc, (size_t)kTuneRowsA * k * 4);
  sj_status s = SJ_OK;
  if (e == cudaSuccess) {
    tune_rows_kernel<<<(unsigned)((kTuneRowsA + 127) / 128), 128, 0, h->stream>>>(A, kTuneRowsA,
                                                                                d, 1);
    tune_rows_kernel<<<(unsigned)((nB_max + 127) / 128), 128, 0, h->stream>>>(B, nB_max, d, 2);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    note_cuda_error(e, "autotune buffers", __LINE__);
    s = cuda_status(e);
  }
  for (int c = kTuneClassLo; c <= kTuneClassHi && s == SJ_OK; ++c) {
    const int64_t nB = (int64_t)3 << (c - 2);  // three quarters of the class's upper end
    double best = 1e300;
    int best_w = kTcBN;
    for (int w : {kTcBNNarrow, kTcBN}) {
      h->force_bn = w;
      double t = 1e300;
      for (int rep = 0; rep < 3 && s == SJ_OK; ++rep) {
        JoinReq r{A, kTuneRowsA, B, nB, k, idx, sc, false, 0.0, nullptr, 0, nullptr};
        sj_stats st{};
        s = join_batch(h, &r, 1, &st);
        if (rep > 0) t = std::min(t, st.ms_total);
      }
      if (t < best) {
        best = t;
        best_w = w;
      }
    }
    h->force_bn = 0;
    h->tile_width[{k, c}] = best_w;
  }
  h->force_bn = 0;
  cudaStreamSynchronize(h->stream);
  cudaFree(A);
  cudaFree(B);
  cudaFree(idx);
  cudaFree(sc);
  if (s == SJ_OK && path) s = write_tile_table(h, path);
  return s;
}

sj_status sj_autotune_load(sj_handle *h, const char *path) {
  if (!h || !path) return SJ_ERR_INVALID_ARG;
  FILE *f = std::fopen(path, "r");
  if (!f) return SJ_ERR_INVALID_ARG;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    long long d;
    int prec, k, c, w;
    if (std::sscanf(line, "%lld %d %d %d %d", &d, &prec, &k, &c, &w) != 5) continue;
    if (d != h->cfg.d || prec != (int)h->cfg.prec) continue;
    if (w != kTcBN && w != kTcBNNarrow) continue;
    h->tile_width[{k, c}] = w;
  }
  std::fclose(f);
  return SJ_OK;
}

sj_status sj_create(sj_handle **out, const sj_config *cfg) {
  if (!out || !cfg || cfg->d < 1) return SJ_ERR_INVALID_ARG;
  if (cfg->prec != SJ_FP32 && cfg->prec != SJ_BF16 && cfg->prec != SJ_FP8_E4M3 &&
      cfg->prec != SJ_BF16X3)
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
  if (cfg->prec != SJ_FP32 && cc != 103) return SJ_ERR_UNSUPPORTED;
  sj_handle *h = new (std::nothrow) sj_handle();
  if (!h) return SJ_ERR_OOM;
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  h->sm_count = prop.multiProcessorCount;
  h->cc = cc;
  cudaError_t e = cudaMallocHost(&h->h_ctr, sizeof(Counters));
  for (int t = 0; t < 6 && e == cudaSuccess; ++t) e = cudaEventCreate(&h->ev[t]);
  for (int t = 0; t < 4 && e == cudaSuccess; ++t) e = cudaEventCreate(&h->gev[t]);
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
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->ws) cudaFree(h->ws);
  if (h->h_ctr) cudaFreeHost(h->h_ctr);
  if (h->h_tab) cudaFreeHost(h->h_tab);
  for (int t = 0; t < 6; ++t)
    if (h->ev[t]) cudaEventDestroy(h->ev[t]);
  for (int t = 0; t < 4; ++t)
    if (h->gev[t]) cudaEventDestroy(h->gev[t]);
  if (h->tc) tc_destroy(h->tc);
  if (h->aux) sj_destroy(h->aux);
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
  std::vector<JoinReq> reqs;
  reqs.reserve((size_t)n_jobs);
  for (int32_t q = 0; q < n_jobs; ++q) {
    const sj_job &jb = jobs[q];
    if (jb.k < 0) return SJ_ERR_INVALID_ARG;
    const bool want_topk = jb.k > 0;
    const bool want_thr = jb.n_out != nullptr;
    if ((jb.topk_idx || jb.topk_score) && !want_topk) return SJ_ERR_INVALID_ARG;
    if (jb.pairs && !want_thr) return SJ_ERR_INVALID_ARG;
    if (!want_topk && !want_thr) continue;  // nothing requested
    reqs.push_back(JoinReq{jb.A, jb.nA, jb.B, jb.nB, jb.k, jb.topk_idx, jb.topk_score, want_thr,
                           jb.tau, jb.pairs, jb.capacity, jb.n_out});
  }
  return join_batch(h, reqs.data(), (int)reqs.size(), st);
}

}  // extern "C"

namespace {

// Shared set-up of the contrastive calls: BF16 packing (and transposes for the
// backward) of A and B into the workspace, and their tensor maps.
struct ContrastivePlan {
  int64_t nx, ny, d, npx, npy, dp;  // rows of A (the call's row operand) and of B, padded
  void *Ap, *Bp, *AT, *BT;
  void *G;       // materialised backward: dL/dS (npx x npy BF16)
  float *part;   // forward: partial row states (3 x 2 n_splits x npx) and S_ii (npx)
  int n_splits, tiles_per_split;
  Counters *ctr;
  float *scratch;  // nx + ny floats (per-row loss terms)
  unsigned char mA[128], mB[128], mAT[128], mBT[128], mG[128];
};

// `gmat`: also reserve and map G (fails with SJ_ERR_OOM before any launch
// when the workspace cannot hold it).  A has nx rows, B ny rows.
sj_status contrastive_setup(sj_handle *h, const void *A, int64_t nx, const void *B, int64_t ny,
                            bool bwd, ContrastivePlan &cp, bool gmat = false) {
  if (!h || !A || !B || nx < 1 || ny < 1) return SJ_ERR_INVALID_ARG;
  if (nx >= (1ll << 31) - 1024 || ny >= (1ll << 31) - 1024) return SJ_ERR_UNSUPPORTED;
  if (!is_device_ptr(A, h->cfg.device) || !is_device_ptr(B, h->cfg.device))
    return SJ_ERR_INVALID_ARG;
  SJ_CUDA(cudaSetDevice(h->cfg.device));
  if (h->cc != 103) return SJ_ERR_UNSUPPORTED;
  if (!h->tc) {
    sj_status s = tc_create(&h->tc);
    if (s != SJ_OK) return s;
  }
  cp.nx = nx;
  cp.ny = ny;
  cp.d = h->cfg.d;
  cp.npx = round_up(nx, 256);
  cp.npy = round_up(ny, 256);
  cp.dp = round_up(cp.d, 64);
  contrastive_splits(cp.npy, &cp.n_splits, &cp.tiles_per_split);
  const size_t opa = (size_t)cp.npx * cp.dp * 2, opb = (size_t)cp.npy * cp.dp * 2;
  const size_t gsz = (size_t)cp.npx * cp.npy * 2;
  const size_t psz = ((size_t)6 * cp.n_splits + 1) * std::max(cp.npx, cp.npy) * 4;
  size_t bytes = (opa + opb) * (bwd ? 2 : 1) + sizeof(Counters) + (size_t)(nx + ny) * 4 +
                 8 * 256 + (gmat ? gsz + 256 : 0) + (bwd ? 0 : psz + 256);
  sj_status s = ensure_ws(h, bytes);
  if (s != SJ_OK) return s;
  Arena ar{static_cast<unsigned char *>(h->ws), h->ws_size, 0};
  cp.ctr = static_cast<Counters *>(ar.take(sizeof(Counters)));
  cp.scratch = static_cast<float *>(ar.take((size_t)(nx + ny) * 4));
  cp.Ap = ar.take(opa);
  cp.Bp = ar.take(opb);
  cp.AT = bwd ? ar.take(opa) : nullptr;
  cp.BT = bwd ? ar.take(opb) : nullptr;
  cp.G = gmat ? ar.take(gsz) : nullptr;
  cp.part = bwd ? nullptr : static_cast<float *>(ar.take(psz));
  if (!cp.ctr || !cp.scratch || !cp.Ap || !cp.Bp || (bwd && (!cp.AT || !cp.BT)) ||
      (gmat && !cp.G) || (!bwd && !cp.part))
    return SJ_ERR_INTERNAL;
  cudaStream_t st = h->stream;
  SJ_CUDA(cudaMemsetAsync(cp.ctr, 0, sizeof(Counters), st));
  SJ_CUDA(launch_contrastive_pack(static_cast<const float *>(A), nx, cp.d, cp.Ap, cp.AT, cp.npx,
                                  cp.dp, &cp.ctr->err_flags, st));
  SJ_CUDA(launch_contrastive_pack(static_cast<const float *>(B), ny, cp.d, cp.Bp, cp.BT, cp.npy,
                                  cp.dp, &cp.ctr->err_flags, st));
  s = tc_encode_2d(h->tc, cp.Ap, cp.dp, cp.npx, 64, 128, cp.mA);
  if (s == SJ_OK) s = tc_encode_2d(h->tc, cp.Bp, cp.dp, cp.npy, 64, 128, cp.mB);
  if (s == SJ_OK && bwd) s = tc_encode_2d(h->tc, cp.AT, cp.npx, cp.dp, 64, 64, cp.mAT);
  if (s == SJ_OK && bwd) s = tc_encode_2d(h->tc, cp.BT, cp.npy, cp.dp, 64, 64, cp.mBT);
  if (s == SJ_OK && gmat) s = tc_encode_2d(h->tc, cp.G, cp.npy, cp.npx, 64, 128, cp.mG);
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

int64_t sj::planned_tiles_per_split(sj_handle *h, int64_t nA, int64_t nB, int k, bool thr) {
  JoinReq r{nullptr, nA, nullptr, nB, k, nullptr, nullptr, thr, 0.5, nullptr, 0, nullptr};
  BatchPlan P;
  if (make_batch_plan(h, &r, 1, P) != SJ_OK || P.jobs.empty()) return 0;
  return P.jobs[0].tiles_per_split;
}

void sj::set_tiles_per_split(sj_handle *h, int64_t tps) { h->force_tps = tps; }

extern "C" {

}  // extern "C"

namespace {

// Forward over rows [r0, r0 + nx) of a paired set of N rows: A holds those nx
// rows, B all N; the positive of local row i is B row r0 + i; the loss is
// normalised by N.  With r0 = 0 and nx = N it is the whole join (and the
// symmetric flag adds the column term).
sj_status contrastive_fwd_impl(sj_handle *h, const void *A, int64_t nx, int64_t r0,
                               const void *B, int64_t N, float T, bool sym, float *loss,
                               float *lse) {
  ContrastivePlan cp;
  sj_status s = contrastive_setup(h, A, nx, B, N, false, cp);
  if (s != SJ_OK) return s;
  ContrastiveArgs a{};
  a.n = nx;
  a.d = cp.d;
  a.np = cp.npx;
  a.ny = N;
  a.npy = cp.npy;
  a.diag_off = r0;
  a.n_norm = N;
  a.dp = cp.dp;
  a.T = T;
  a.n_chunks = 1;
  a.ctr = cp.ctr;
  a.debug_timeout = (h->cfg.flags & SJ_FLAG_DEBUG_TIMEOUT) ? 1 : 0;
  // units = (row block, column split) for balance across the SMs; the
  // partial row states are merged by a second launch
  a.n_splits = cp.n_splits;
  a.tiles_per_split = cp.tiles_per_split;
  const size_t pn = (size_t)2 * cp.n_splits * cp.npx;
  a.part_m = cp.part;
  a.part_l = cp.part + pn;
  a.part_c = cp.part + 2 * pn;
  a.diag_out = cp.part + 3 * pn;
  const int grid = (int)std::min<int64_t>((cp.npx / 128) * cp.n_splits, h->sm_count);
  a.lse_out = lse;
  a.term_out = cp.scratch;
  SJ_CUDA(launch_contrastive(kContrastiveFwd, cp.mA, cp.mB, nullptr, a, grid, h->stream));
  if (sym) {  // square only: rows of B against the columns of A
    a.lse_out = lse + N;
    a.term_out = cp.scratch + N;
    SJ_CUDA(launch_contrastive(kContrastiveFwd, cp.mB, cp.mA, nullptr, a, grid, h->stream));
  }
  SJ_CUDA(launch_contrastive_loss(cp.scratch, sym ? cp.scratch + N : nullptr, nx, N,
                                  sym ? 0.5f : 1.f, 0.5f, loss, h->stream));
  return contrastive_finish(h, cp);
}

// Backward of contrastive_fwd_impl: dA (nx x d) for the call's rows and dB
// (N x d), the rows' contribution to the gradient of B (the whole of it when
// nx = N).
sj_status backward_impl(sj_handle *h, const void *A, int64_t nx, int64_t r0, const void *B,
                        int64_t N, float T, bool sym, const float *lse, const float *grad_loss,
                        float *dA, float *dB) {
  ContrastivePlan cp;
  // materialise G when the workspace allows, else the fused path
  bool gmat = (h->cfg.flags & SJ_FLAG_FUSED_BACKWARD) == 0;
  sj_status s = gmat ? contrastive_setup(h, A, nx, B, N, true, cp, true) : SJ_ERR_OOM;
  if (s == SJ_ERR_OOM) {
    gmat = false;
    s = contrastive_setup(h, A, nx, B, N, true, cp, false);
  }
  if (s != SJ_OK) return s;
  ContrastiveArgs a{};
  a.n = nx;
  a.d = cp.d;
  a.np = cp.npx;
  a.ny = N;
  a.npy = cp.npy;
  a.diag_off = r0;
  a.n_norm = N;
  a.dp = cp.dp;
  a.T = T;
  a.n_chunks = (int)((cp.dp + 383) / 384);
  a.n_splits = 1;
  a.tiles_per_split = (int)(cp.npy / 128);
  a.grad_loss = grad_loss;
  a.ctr = cp.ctr;
  a.debug_timeout = (h->cfg.flags & SJ_FLAG_DEBUG_TIMEOUT) ? 1 : 0;
  // G = w_r (P - I) + w_c (Q - I): the row softmax P of A's rows, the column
  // softmax Q (symmetric loss only)
  a.lse_r = lse;
  a.wr = sym ? 0.5f : 1.f;
  a.lse_c = sym ? lse + N : lse;
  a.wc = sym ? 0.5f : 0.f;
  const int64_t n_rb = cp.npx / 128;
  if (gmat) {
    // G pass: units = (row block, column split) for balance; G written
    // through its tensor map (TMA stores)
    a.n_splits = cp.n_splits;
    a.tiles_per_split = cp.tiles_per_split;
    const int grid = (int)std::min<int64_t>(n_rb * a.n_splits, h->sm_count);
    SJ_CUDA(launch_contrastive(kContrastiveGprime, cp.mA, cp.mB, cp.mG, a, grid, h->stream));
    ContrastiveGemmArgs g{};
    g.d = cp.d;
    g.dp = cp.dp;
    g.n_norm = N;
    g.T = T;
    g.n_chunks = a.n_chunks;
    g.grad_loss = grad_loss;
    g.ctr = cp.ctr;
    g.n = nx;  // dA = G B / T: rows of A, K over the rows of B
    g.np = cp.npx;
    g.kp = cp.npy;
    g.dX = dA;
    SJ_CUDA(launch_contrastive_gemm(false, cp.mG, cp.mBT, g,
                                    (int)std::min<int64_t>(n_rb * g.n_chunks, h->sm_count),
                                    h->stream));
    g.n = N;  // dB = G^T A / T: rows of B, K over the rows of A
    g.np = cp.npy;
    g.kp = cp.npx;
    g.dX = dB;
    // G^T as an MN-major operand: boxes of 64 columns x 64 rows of G
    unsigned char mG64[128];
    sj_status ms = tc_encode_2d(h->tc, cp.G, cp.npy, cp.npx, 64, 64, mG64);
    if (ms != SJ_OK) return ms;
    SJ_CUDA(launch_contrastive_gemm(true, mG64, cp.mAT, g,
                                    (int)std::min<int64_t>((cp.npy / 128) * g.n_chunks,
                                                           h->sm_count),
                                    h->stream));
    return contrastive_finish(h, cp);
  }
  // dA: rows of A against columns (rows of B); row term = softmax over j
  a.dX = dA;
  SJ_CUDA(launch_contrastive(kContrastiveBwdFused, cp.mA, cp.mB, cp.mBT, a,
                             (int)std::min<int64_t>(n_rb * a.n_chunks, h->sm_count), h->stream));
  // dB: rows of B against columns (rows of A); the row softmax term is indexed
  // by the kernel's columns, the column softmax term by its rows; B row j's
  // positive is A row j - r0
  a.n = N;
  a.np = cp.npy;
  a.ny = nx;
  a.npy = cp.npx;
  a.diag_off = -r0;
  a.tiles_per_split = (int)(cp.npx / 128);
  a.lse_r = sym ? lse + N : lse;
  a.wr = sym ? 0.5f : 0.f;
  a.lse_c = lse;
  a.wc = sym ? 0.5f : 1.f;
  a.dX = dB;
  SJ_CUDA(launch_contrastive(kContrastiveBwdFused, cp.mB, cp.mA, cp.mAT, a,
                             (int)std::min<int64_t>((cp.npy / 128) * a.n_chunks, h->sm_count),
                             h->stream));
  return contrastive_finish(h, cp);
}

}  // namespace

extern "C" {

sj_status sj_contrastive_fwd(sj_handle *h, const void *A, const void *B, int64_t N, float T,
                             float *loss, float *lse) {
  if (!h || !A || !B || N < 1 || !(T > 0.f) || !loss || !lse) return SJ_ERR_INVALID_ARG;
  if (!is_device_ptr(loss, h->cfg.device) || !is_device_ptr(lse, h->cfg.device))
    return SJ_ERR_INVALID_ARG;
  return contrastive_fwd_impl(h, A, N, 0, B, N, T, (h->cfg.flags & SJ_FLAG_SYM_INFONCE) != 0,
                              loss, lse);
}

sj_status sj_backward(sj_handle *h, const void *A, const void *B, int64_t N, float T,
                      const float *lse, const float *grad_loss, float *dA, float *dB) {
  if (!h || !A || !B || N < 1 || !(T > 0.f) || !lse || !grad_loss || !dA || !dB)
    return SJ_ERR_INVALID_ARG;
  const int dv = h->cfg.device;
  if (!is_device_ptr(lse, dv) || !is_device_ptr(grad_loss, dv) || !is_device_ptr(dA, dv) ||
      !is_device_ptr(dB, dv))
    return SJ_ERR_INVALID_ARG;
  return backward_impl(h, A, N, 0, B, N, T, (h->cfg.flags & SJ_FLAG_SYM_INFONCE) != 0, lse,
                       grad_loss, dA, dB);
}

sj_status sj_contrastive_fwd_rows(sj_handle *h, const void *A_rows, int64_t n_rows, int64_t r0,
                                  const void *B, int64_t N, float T, float *loss_part,
                                  float *lse_rows) {
  if (!h || !A_rows || !B || n_rows < 1 || r0 < 0 || r0 + n_rows > N || !(T > 0.f) ||
      !loss_part || !lse_rows)
    return SJ_ERR_INVALID_ARG;
  if (h->cfg.flags & SJ_FLAG_SYM_INFONCE) return SJ_ERR_UNSUPPORTED;
  if (!is_device_ptr(loss_part, h->cfg.device) || !is_device_ptr(lse_rows, h->cfg.device))
    return SJ_ERR_INVALID_ARG;
  return contrastive_fwd_impl(h, A_rows, n_rows, r0, B, N, T, false, loss_part, lse_rows);
}

sj_status sj_backward_rows(sj_handle *h, const void *A_rows, int64_t n_rows, int64_t r0,
                           const void *B, int64_t N, float T, const float *lse_rows,
                           const float *grad_loss, float *dA_rows, float *dB_part) {
  if (!h || !A_rows || !B || n_rows < 1 || r0 < 0 || r0 + n_rows > N || !(T > 0.f) ||
      !lse_rows || !grad_loss || !dA_rows || !dB_part)
    return SJ_ERR_INVALID_ARG;
  if (h->cfg.flags & SJ_FLAG_SYM_INFONCE) return SJ_ERR_UNSUPPORTED;
  const int dv = h->cfg.device;
  if (!is_device_ptr(lse_rows, dv) || !is_device_ptr(grad_loss, dv) ||
      !is_device_ptr(dA_rows, dv) || !is_device_ptr(dB_part, dv))
    return SJ_ERR_INVALID_ARG;
  return backward_impl(h, A_rows, n_rows, r0, B, N, T, false, lse_rows, grad_loss, dA_rows,
                       dB_part);
}

sj_status sj_debug_scores(sj_handle *h, float *raw, float *margin) {
  if (!h || !raw || !margin) return SJ_ERR_INVALID_ARG;
  if (!is_device_ptr(raw, h->cfg.device) || !is_device_ptr(margin, h->cfg.device))
    return SJ_ERR_INVALID_ARG;
  h->dbg_raw = raw;
  h->dbg_margin = margin;
  return SJ_OK;
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

const char *sj_last_error_detail(void) { return g_err_detail; }

}  // extern "C"
