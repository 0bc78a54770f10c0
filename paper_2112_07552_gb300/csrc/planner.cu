// planner.cu -- sj_plan: choose the scoring precision of a join from a census.
//
// The paper's optimizer (Sec. 4.2) tests which compact type represents the
// data exactly (the feasibility test) and ranks plans with the cost model
// Eq. (cost), CT ~ 2 M N K / peak.  For real-valued embeddings no low
// precision is exact; exactness comes from rescoring instead, and what a
// precision costs is its tensor-core time plus the rescoring its error
// margin lets through -- a property of the data.  So the planner measures
// the second on a census (a sample of left rows against all of B, through
// the same kernels) and models the first with Eq. (cost).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/sj.h"
#include "sj_internal.h"

namespace sj {
namespace {

// flop per clock per SM of each scoring precision's pipe, and the fraction of
// it the scoring kernels of this library reached on GB300 (headline BF16
// join, E4M3 threshold join, the hi/lo split on the Zipf top-50 join, the
// CUDA-core FP32 form), indexed by sj_precision.
constexpr double kFlopPerClk[4] = {256.0, 8192.0, 16384.0, 8192.0};
constexpr double kEff[4] = {0.31, 0.71, 0.74, 0.65};

sj_status pl_fail(cudaError_t e, const char *what, int line) {
  record_cuda_error(e, what, "planner.cu", line);
  return e == cudaErrorMemoryAllocation ? SJ_ERR_OOM : SJ_ERR_CUDA;
}
#define PL_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return pl_fail(e__, #call, __LINE__); \
  } while (0)

struct PlBuf {
  void *p = nullptr;
  ~PlBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace
}  // namespace sj

using namespace sj;

extern "C" sj_status sj_plan(sj_handle *h, const float *A, int64_t nA, const float *B,
                             int64_t nB, int32_t k, double tau, int64_t sample_rows,
                             sj_plan_info *info) {
  const bool thr = !std::isnan(tau);
  if (!h || !info || nA < 1 || nB < 1 || !A || !B || k < 0 || k > 1024 || (k == 0 && !thr) ||
      sample_rows < 0)
    return SJ_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof *info);
  const sj_config cfg0 = *handle_config(h);
  const int dev = cfg0.device;
  const int64_t d = cfg0.d;
  cudaStream_t stm = static_cast<cudaStream_t>(handle_stream(h));
  PL_CUDA(cudaSetDevice(dev));
  const int64_t s = std::min<int64_t>(nA, sample_rows ? sample_rows : 512);
  info->sample_rows = s;
  // evenly spaced rows of A, gathered where A lives
  cudaPointerAttributes at;
  bool a_dev = false;
  if (cudaPointerGetAttributes(&at, A) == cudaSuccess)
    a_dev = at.type == cudaMemoryTypeManaged || at.type == cudaMemoryTypeDevice;
  else
    cudaGetLastError();
  if (a_dev && at.type == cudaMemoryTypeDevice && at.device != dev) return SJ_ERR_INVALID_ARG;
  const int64_t stride = nA / s;
  PlBuf sample_d, idx_d, sc_d;
  std::vector<float> sample_h;
  const float *As = nullptr;
  if (a_dev) {
    PL_CUDA(cudaMalloc(&sample_d.p, (size_t)s * d * 4));
    PL_CUDA(cudaMemcpy2DAsync(sample_d.p, (size_t)d * 4, A, (size_t)stride * d * 4,
                              (size_t)d * 4, (size_t)s, cudaMemcpyDeviceToDevice, stm));
    As = static_cast<const float *>(sample_d.p);
  } else {
    sample_h.resize((size_t)s * d);
    for (int64_t r = 0; r < s; ++r)
      std::memcpy(&sample_h[(size_t)r * d], A + (size_t)r * stride * d, (size_t)d * 4);
    As = sample_h.data();
  }
  if (k > 0) {
    PL_CUDA(cudaMalloc(&idx_d.p, (size_t)s * k * 8));
    PL_CUDA(cudaMalloc(&sc_d.p, (size_t)s * k * 4));
  }
  int clock_khz = 0, sms = 0;
  PL_CUDA(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
  PL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const double flops = 2.0 * (double)nA * (double)nB * (double)d;
  double best = INFINITY;
  double sel_dev[4] = {0, 0, 0, 0}, host[4] = {0, 0, 0, 0};
  bool ran[4] = {false, false, false, false};
  info->choice = SJ_BF16;
  for (int p = 0; p < 4; ++p) {
    info->est_ms[p] = INFINITY;
    sj_config c = cfg0;
    c.prec = (sj_precision)p;
    c.flags &= (uint32_t)(SJ_FLAG_SINGLE_SPLIT | SJ_FLAG_NO_GRAPH);
    sj_handle *hp = nullptr;
    sj_status st = sj_create(&hp, &c);
    if (st == SJ_ERR_UNSUPPORTED) continue;  // no tensor-core path on this device
    if (st != SJ_OK) return st;
    // the sample gets the full join's split plan (lists of the same length)
    set_tiles_per_split(hp, planned_tiles_per_split(hp, nA, nB, k, thr));
    sj_job jb;
    std::memset(&jb, 0, sizeof jb);
    jb.A = As;
    jb.nA = s;
    jb.B = B;
    jb.nB = nB;
    jb.k = k;
    jb.tau = thr ? tau : 0.0;
    jb.topk_idx = static_cast<int64_t *>(idx_d.p);
    jb.topk_score = static_cast<float *>(sc_d.p);
    int64_t n_out = 0;
    jb.pairs = nullptr;
    jb.capacity = 0;  // count the pairs only
    jb.n_out = thr ? &n_out : nullptr;
    // The first call sizes the handle's workspace.  Then s rows and one row
    // are timed: T(s) - T(1) over s - 1 rows is the cost that grows with rows
    // (the fixed costs of a call cancel; a sample too small to fill the GPU
    // errs high, not low).  Device time of the finalisation from its events;
    // host time (the rescan fallback of overflowed rows runs after those
    // events) from the wall clock.
    const int64_t q = 1;
    sj_stats stt, stq;
    double wall_s = 0.0, wall_q = 0.0;
    for (int rep = 0; rep < 3 && (st == SJ_OK || st == SJ_ERR_CAPACITY); ++rep) {
      jb.nA = rep == 2 ? q : s;
      const auto t0 = std::chrono::steady_clock::now();
      st = sj_batch(hp, &jb, 1, rep == 2 ? &stq : &stt);
      const double w = std::chrono::duration<double, std::milli>(
                           std::chrono::steady_clock::now() - t0).count();
      (rep == 2 ? wall_q : wall_s) = w;
    }
    sj_destroy(hp);
    if (st != SJ_OK && st != SJ_ERR_CAPACITY) return st;
    const double peak = (double)sms * kFlopPerClk[p] * (double)clock_khz * 1e3;
    const double work = flops * (p == SJ_BF16X3 ? 3.0 : 1.0);
    info->score_ms[p] = work / (kEff[p] * peak) * 1e3;
    const double rows = (double)(s - q);
    sel_dev[p] = s > q ? std::max(0.0, stt.ms_select - stq.ms_select) / rows
                       : stt.ms_select / (double)s;
    host[p] = s > q ? std::max(0.0, (wall_s - stt.ms_total) - (wall_q - stq.ms_total)) / rows
                    : 0.0;
    ran[p] = true;
    info->cand_per_row[p] = (double)stt.n_rescored / (double)s;
    info->overflow_frac[p] = (double)stt.n_overflow_rows / (double)s;
  }
  PL_CUDA(cudaStreamSynchronize(stm));
  // per-row costs times nA; host time per row counts only where rows fell
  // back to rescans (otherwise it is noise of the fixed host work)
  for (int p = 0; p < 4; ++p) {
    if (!ran[p]) continue;
    const double fallback = info->overflow_frac[p] > 0.0 ? host[p] : 0.0;
    info->select_ms[p] = (sel_dev[p] + fallback) * (double)nA;
    info->est_ms[p] = info->score_ms[p] + info->select_ms[p];
    if (info->est_ms[p] < best) {
      best = info->est_ms[p];
      info->choice = (sj_precision)p;
    }
  }
  return best < INFINITY ? SJ_OK : SJ_ERR_UNSUPPORTED;
}
