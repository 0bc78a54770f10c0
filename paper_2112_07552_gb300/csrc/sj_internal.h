// sj_internal.h -- host-side declarations shared by the library's translation
// units (launchers and plan structures).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "sj_device.cuh"

namespace sj {

enum class PackFormat { kF32, kBF16 };

cudaError_t launch_prepare(const float *X, int64_t n, int64_t d, PackFormat fmt, void *Xp,
                           int64_t n_pad, int64_t dp, RowMeta *meta, float *gmax,
                           Counters *ctr, cudaStream_t st);

// Everything the scoring kernels need for one join.
struct ScoreArgs {
  const void *Ap;          // packed A rows (stride dp elements), rows padded
  const void *Bp;          // packed B rows
  int64_t nA, nB, dp;      // true row counts, padded width
  const RowMeta *metaA;    // per-row bounds of A
  const float *gmaxB;      // device: max over B of {nrm, qnrm, qerr}
  float acc_coef;          // accumulation error allowance per unit norm product
  int k;                   // top-k (0: no top-k)
  float tau_f;             // float tau rounded down (+inf: no threshold)
  int n_splits;            // column splits per row block
  int bands_per_split;     // band lists per (row, split): one per epilogue column group
  int64_t tiles_per_split; // column tiles per split
  int64_t n_units;         // row blocks x splits
  Cand *band;              // [nA][n_splits * bands_per_split][cap]
  int cap;
  int *band_cnt;           // [nA][n_splits * bands_per_split]; -(cnt + 1): overflowed
  ThrCand *thr;            // threshold candidates
  unsigned long long thr_cap;
  Counters *ctr;
};

// Tile sizes of the scoring kernels (rows x columns of one score tile).
constexpr int kSimtBM = 128, kSimtBN = 128, kSimtBK = 16;
constexpr int kTcBM = 128, kTcBN = 256;

cudaError_t launch_score_simt(const ScoreArgs &a, int grid, cudaStream_t st);

// Finalisation.
struct TopkFinalArgs {
  const float *A;          // original float32 rows (stride d)
  const float *B;
  int64_t nA, nB, d;
  const RowMeta *metaA, *metaB;
  const float *gmaxB;
  float acc_coef;
  int k, n_splits, cap;    // n_splits here counts band lists per row
  const Cand *band;
  const int *band_cnt;
  float dot2_coef_key;     // Dot2 error bound per unit norm product, key units
  int64_t *out_idx;
  float *out_score;
  int *tier2_rows;         // rows with more candidates than the first tier holds
  int *overflow_rows;      // rows whose band list overflowed (rescan fallback)
  long long *overflow_key; // their rescan key bounds
  Counters *ctr;
};
cudaError_t launch_topk_finalize(const TopkFinalArgs &a, cudaStream_t st);
cudaError_t launch_topk_finalize_tier2(const TopkFinalArgs &a, int n_rows, cudaStream_t st);

// Fallback of the top-k finalisation: rescan B for rows whose candidates did
// not fit, then rank the resulting short lists.
struct KeyCand {
  long long U, L;  // key interval of the exact score
  int32_t j, pad;
};
struct RescanArgs {
  const float *A, *B;
  int64_t nB, d;
  const RowMeta *metaA, *metaB;
  float dot2_coef_key;
  const int *rows;         // left rows to rescan
  const long long *keys;   // per row: keep j when its upper key >= keys[r]
  int n_rows;
  KeyCand *lists;          // n_rows x cap
  int *count;              // n_rows (zeroed by the caller)
  int cap;
  Counters *ctr;
};
cudaError_t launch_topk_rescan(const RescanArgs &a, cudaStream_t st);

struct RankListArgs {
  const float *A, *B;
  int64_t d;
  int k;
  const int *rows;
  int n_rows;
  const KeyCand *lists;
  const int *count;
  int cap;
  int *redo;               // list slots cut off at cap
  int *big;                // list slots longer than the shared-memory ranker takes
  int64_t *out_idx;
  float *out_score;
  Counters *ctr;
};
cudaError_t launch_topk_rank_lists(const RankListArgs &a, cudaStream_t st);
size_t topk_rank_global_row_bytes(int64_t n);
cudaError_t launch_topk_rank_global(const RankListArgs &a, const int *big, int n_big,
                                    void *scratch, size_t per_row, cudaStream_t st);

struct ThrFinalArgs {
  const float *A, *B;
  int64_t nA, nB, d;
  const RowMeta *metaA, *metaB;
  float dot2_coef_key;
  long long tau_key;       // ceil(tau 2^60)
  Exact tau_exact;         // ceil(tau 2^298) in the exact format
  const ThrCand *cand;
  int64_t n_cand;
  int64_t *row_count;      // [nA], zeroed by the caller
  ThrCand *accepted;       // accepted pairs (score in v), capacity n_cand
  Counters *ctr;
};
cudaError_t launch_thr_rescore(const ThrFinalArgs &a, cudaStream_t st);

// Exclusive scan of n int64 values (in place allowed); total written to *total.
size_t scan_scratch_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *total,
                                  void *scratch, cudaStream_t st);

struct PairOut {  // layout of sj_pair
  int64_t i, j;
  float score;
  int32_t pad;
};
cudaError_t launch_thr_scatter(const ThrCand *accepted, const int64_t *n_acc_dev,
                               int64_t n_acc_cap, const int64_t *row_off, int64_t *row_fill,
                               PairOut *out, cudaStream_t st);
cudaError_t launch_thr_sort_rows(PairOut *out, const int64_t *row_off, const int64_t *row_count,
                                 int64_t nA, int *big_rows, int *n_big, int big_cap,
                                 cudaStream_t st);
cudaError_t launch_thr_sort_big(PairOut *out, PairOut *tmp, const int64_t *row_off,
                                const int64_t *row_count, const int *big_rows, const int *n_big,
                                int n_big_host, cudaStream_t st);

}  // namespace sj
