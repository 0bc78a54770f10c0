// sj_internal.h -- host-side declarations shared by the library's translation
// units (launchers and plan structures).  Not part of the public ABI.
//
// Every join kernel works on a batch of independent joins described by a job
// table in device memory; a single join is a batch of one.  Rows are numbered
// three ways: local (within a job), global (A rows of all jobs in job order,
// unpadded) and packed (rows of the packed operand buffers, each job padded
// to the tile edge).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sj.h"
#include "sj_device.cuh"

namespace sj {

// A second handle inside h with the same device, stream and workspace limit
// but width d, precision prec and h's flags plus extra_flags (created on
// first use, replaced when any of them change, destroyed with h): the
// relational calls run their one-hot joins through it, the cascade its FP32
// re-joins.
sj_status aux_handle(sj_handle *h, int64_t d, sj_precision prec, sj_handle **out,
                     uint32_t extra_flags = 0);
int handle_device(const sj_handle *h);
const sj_config *handle_config(const sj_handle *h);
// Column tiles per split the planner gives a one-job join of these sizes on h,
// and an override of it for h's later calls (0: none): the precision
// planner's census runs a sample of rows with the full join's split plan, so
// its candidate lists cover as many columns as the real join's.
int64_t planned_tiles_per_split(sj_handle *h, int64_t nA, int64_t nB, int k, bool thr);
void set_tiles_per_split(sj_handle *h, int64_t tps);
void *handle_stream(const sj_handle *h);
int handle_sm_count(const sj_handle *h);

// Record the CUDA failure behind an SJ_ERR_CUDA / SJ_ERR_OOM status for
// sj_last_error_detail() (thread-local; error name, file:line, call, message).
void record_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// kBF16X3: rows of 3d bfloat16, [hi | hi | lo] for A rows and [hi | lo | hi]
// for B rows (x = hi + lo + r, hi = bf16(x), lo = bf16(x - hi)).
enum class PackFormat { kF32, kBF16, kFP8, kBF16X3 };

struct PairOut {  // layout of sj_pair
  int64_t i, j;
  float score;
  int32_t pad;
};

// One join of a batch as the kernels see it.
struct JobDev {
  const float *A, *B;        // float32 rows on the device (staged copies of host inputs)
  int64_t nA, nB;
  int64_t a_prow0, b_prow0;  // first packed row of A / B (multiples of the tile edges)
  int64_t row0;              // first global row
  int64_t slot0;             // first band-list slot (row-major: local row * lists + list)
  int64_t band0;             // first band-list entry (slots of this job hold cap entries)
  int64_t topv0;             // first exact top-k value per slot (k per slot), -1: none
  int32_t k;                 // 0: no top-k part
  int32_t cap;               // band-list capacity
  int32_t lists;             // band lists per row = n_splits * bands per split
  int32_t n_splits;          // column splits
  int32_t tiles_per_split;   // column tiles per split
  int32_t n_col_tiles;       // column tiles of the job
  int32_t bn;                // column tile width of the job (tensor-core pass: 128 or 256)
  int32_t eB;                // E4M3 packing: the job's B rows are stored as x 2^eB
  float bmax;                // E4M3 packing: max |x| over the job's B rows (device-written)
  int32_t pad_e;
  float tau_f;               // tau rounded down to float (+inf: no threshold part)
  float gmaxB[4];            // max over the job's B rows of {nrm, qnrm, qerr, lonrm}
                             // (device-written)
  long long tau_key;         // ceil(tau 2^60)
  Exact tau_exact;           // ceil(tau 2^298)
  int64_t *out_idx;          // device top-k outputs (nA x k)
  float *out_score;
  PairOut *out_pairs;        // device pair outputs
  int64_t capacity;
  int64_t n_pairs;           // device-written: pairs of the job
};

// One work unit of the scoring kernels: a 128-row block of a job's A against
// one column split of its B.
struct UnitDev {
  int32_t job, rb, split, pad;
};

// Index of the job whose global rows hold x (row0 ascending, jobs[0].row0 = 0).
__device__ __forceinline__ int find_job_row0(const JobDev *jobs, int n_jobs, int64_t x) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].row0 <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One range of the packed operand buffer: rows [prow0, next segment's prow0)
// hold src's n rows followed by zero rows.  Both sides of every job live in
// one packed buffer (a self-join shares one segment between its two sides).
struct PackSeg {
  const float *src;
  int64_t n;
  int64_t prow0;
  int32_t job;
  int32_t side;      // 0: A rows, 1: B rows, 2: both (self-join, not with kBF16X3);
                     // B rows feed jobs[job].gmaxB
};
// Job of global row x given a job q0 <= the answer (rows visited in
// increasing order): walks forward from q0.
__device__ __forceinline__ int advance_job_row0(const JobDev *jobs, int n_jobs, int q0, int64_t x) {
  int q = q0;
  while (q + 1 < n_jobs && jobs[q + 1].row0 <= x) ++q;
  return q;
}

// Job of global row x, trying the hint first.
__device__ __forceinline__ int find_job_row0_hint(const JobDev *jobs, int n_jobs, int hint,
                                                  int64_t x) {
  const JobDev &h = jobs[hint];
  if (h.row0 <= x && x < h.row0 + h.nA) return hint;
  return find_job_row0(jobs, n_jobs, x);
}

// For E4M3 (kFP8) two launches: the B-side maxima, then the packing; an A
// row is stored as q = RNE_sat(x 2^e) with its own e (largest with max|x| 2^e
// <= 448), a B row with its job's common eB (from the maxima), a self-join
// segment with eB in both roles.  meta.sexp holds the row's exponent.
// Occupancy bitmaps of a packed buffer (prows rows of row_bytes bytes, prows
// a multiple of 128): occ[g * words + kb / 32] bit kb % 32 for 128-row group g
// and 128-byte k-block kb.
constexpr int kOccMaxWords = 128;  // k-blocks tracked: up to 4,096 (wider rows run dense)
cudaError_t launch_occupancy(const void *Xp, int64_t prows, int64_t row_bytes, uint32_t *occ,
                             int words, cudaStream_t st);

cudaError_t launch_prepare(const PackSeg *segs, int n_segs, JobDev *jobs, int64_t prows,
                           int64_t d, PackFormat fmt, void *Xp, int64_t dp, RowMeta *meta,
                           Counters *ctr, cudaStream_t st);

// Everything the scoring kernels need.
struct ScoreArgs {
  const JobDev *jobs;
  int n_jobs;
  const UnitDev *units;
  int64_t n_units;
  const void *Ap, *Bp;       // packed operands (stride dp elements)
  int64_t dp;
  const RowMeta *metaA;      // per packed row
  float acc_coef;            // accumulation error allowance per unit norm product
  int bands_per_split;       // band lists per (row, split): epilogue column groups
  Cand *band;
  int *band_cnt;             // per slot; -(cnt + 1) marks an overflowed list
  float *topv;               // per slot: the list's k best s~, descending (jobs with topv0 >= 0)
  ThrCand *thr;              // threshold candidates
  unsigned long long thr_cap;
  Counters *ctr;
  // block-sparse scoring (SJ_FLAG_BLOCK_SPARSE): per 128-row group of the
  // packed buffer, occ_words words of bits, bit kb set when a row of the
  // group has a nonzero byte in 128-byte k-block kb; null: dense
  const uint32_t *occ;
  int occ_words;
  // test hook (sj_debug_scores; one job): every raw score s~_ij of the job,
  // row-major nA x nB, and each row's margin m_i; null in normal calls
  float *raw;
  float *raw_m;
};

// Tile sizes of the scoring kernels (rows x columns of one score tile).
constexpr int kSimtBM = 128, kSimtBN = 128, kSimtBK = 16;
constexpr int kTcBM = 128, kTcBN = 256, kTcBNNarrow = 128;
constexpr int kTcExactMaxK = 32;  // k tracked exactly by the tensor-core epilogue (registers)
constexpr int kTcQueue = 15;      // tensor-core epilogue: queued visits per thread

cudaError_t launch_score_simt(const ScoreArgs &a, int grid, cudaStream_t st);

// Top-k finalisation over global rows.
struct TopkFinalArgs {
  const JobDev *jobs;
  int n_jobs;
  int64_t rows;            // global rows
  int64_t d;
  const RowMeta *metaA, *metaB;  // per packed row
  float acc_coef;
  const Cand *band;
  const int *band_cnt;
  const float *topv;       // per-slot exact k best s~ (jobs with topv0 >= 0)
  float dot2_coef_key;     // Dot2 error bound per unit norm product, key units
  int *defer_rows;         // rows the warp finaliser leaves to the CTA tiers
  int *tier2_rows;         // rows with more candidates than the first tier holds
  int *overflow_rows;      // rows for the fallback (global)
  long long *overflow_key; // their key bounds
  int *overflow_band;      // per fallback row: 1 when its band lists are complete
                           // (more candidates than the block tiers take), 0 when
                           // a list overflowed
  Counters *ctr;
};
// Three launches (warp finaliser, two CTA tiers) with device-side row counts;
// rows left for the fallback are counted in ctr->overflow_rows.
cudaError_t launch_topk_finalize(const TopkFinalArgs &a, int sm_count, cudaStream_t st);

// Fallback of the top-k finalisation: rescan B for rows whose candidates did
// not fit, then rank the resulting short lists.  One job per launch.
struct KeyCand {
  long long U, L;  // key interval of the exact score
  int32_t j, pad;
};
struct RescanArgs {
  const float *A, *B;      // the job's float32 rows
  int64_t nB, d;
  const RowMeta *metaA, *metaB;  // offset to the job's packed rows
  float dot2_coef_key;
  const int *rows;         // local left rows to rescan
  const long long *keys;   // per row: keep j when its upper key >= keys[r]
  int n_rows;
  KeyCand *lists;          // n_rows x cap
  int *count;              // n_rows (zeroed by the caller)
  int cap;
  Counters *ctr;
  // band scan (band != nullptr): the candidates are the rows' band-list
  // entries (lists complete) instead of all of B
  const Cand *band;        // the job's band lists (job offset applied)
  const int *band_cnt;     // the job's list counts (job offset applied)
  int band_lists, band_cap;  // lists per row, entries per list
};
// Rescan (all of B) or band scan, by a.band.
cudaError_t launch_topk_rescan(const RescanArgs &a, cudaStream_t st);

struct RankListArgs {
  const float *A, *B;      // the job's float32 rows
  int64_t d;
  int k;
  const int *rows;         // local left rows
  const long long *keys;   // their rescan key bounds
  int n_rows;
  const KeyCand *lists;
  const int *count;
  int cap;
  int *redo;               // list slots cut off at cap
  long long *redo_key;     // their tightened key bounds
  int *big;                // list slots longer than the shared-memory ranker takes
  int64_t *out_idx;        // the job's outputs
  float *out_score;
  Counters *ctr;
};
cudaError_t launch_topk_rank_lists(const RankListArgs &a, cudaStream_t st);
size_t topk_rank_global_row_bytes(int64_t n);
cudaError_t launch_topk_rank_global(const RankListArgs &a, const int *big, int n_big,
                                    void *scratch, size_t per_row, cudaStream_t st);

// Threshold finalisation over the batch's candidate list.
struct ThrFinalArgs {
  const JobDev *jobs;
  int n_jobs;
  int64_t d;
  const RowMeta *metaA, *metaB;
  float dot2_coef_key;
  const ThrCand *cand;
  const unsigned long long *n_cand;  // device count (clamped to cand_cap)
  int64_t cand_cap;
  int64_t *row_count;      // [rows], zeroed by the caller
  ThrCand *accepted;       // accepted pairs (score in v), capacity cand_cap
  Counters *ctr;
};
cudaError_t launch_thr_rescore(const ThrFinalArgs &a, int grid, cudaStream_t st);
// Candidates cand[0 .. min(*n_cand, cap)) placed into `out` grouped by left
// row (rows in increasing order): counts into cnt (zeroed by the caller), an
// exclusive scan into off (off[i] ends as the end of row i's group), then
// placement.  Skips its work once an input was flagged.
cudaError_t launch_thr_bucket(const ThrCand *cand, const unsigned long long *n_cand,
                              int64_t cap, const Counters *ctr, int64_t rows, int64_t *cnt,
                              int64_t *off, int64_t *total, void *scan_scratch, ThrCand *out,
                              int grid, cudaStream_t st);


// Exclusive scan of n int64 values (in place allowed); total written to *total.
size_t scan_scratch_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                                  void *scratch, cudaStream_t st);

// Per-job pair totals from the scanned row counts: jobs[q].n_pairs and
// job_info[2q] = n_pairs, job_info[2q + 1] = offset of the job's first pair
// in the concatenated (global row) order.
cudaError_t launch_job_pairs(JobDev *jobs, int n_jobs, int64_t rows, const int64_t *row_off,
                             const int64_t *total, int64_t *job_info, cudaStream_t st);
// Pairs of a job within capacity go to jobs[q].out_pairs, or (out_pairs null)
// to `staging` in the concatenated order; a job over capacity writes nothing.
cudaError_t launch_thr_scatter(const JobDev *jobs, int n_jobs, const ThrCand *accepted,
                               const unsigned long long *n_acc, int64_t acc_cap,
                               const int64_t *row_off, int64_t *row_fill, PairOut *staging,
                               int grid, cudaStream_t st);
cudaError_t launch_thr_sort_rows(const JobDev *jobs, int n_jobs, int64_t rows,
                                 const int64_t *row_off, const int64_t *row_count,
                                 PairOut *staging, int *big_rows, int *n_big, cudaStream_t st);
cudaError_t launch_thr_sort_big(const JobDev *jobs, int n_jobs, PairOut *staging, PairOut *tmp,
                                const int64_t *row_off, const int64_t *row_count,
                                const int *big_rows, const int *n_big, int grid, cudaStream_t st);

}  // namespace sj
