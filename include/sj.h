/*
 * sj.h -- C ABI of the GB300 embedding similarity join library (libsj.so).
 *
 * The operation.  The paper (Sec. 3.1, "Two-way natural join") evaluates a
 * join of tables A and B as the matrix product C = mat(A) mat(B)^T and keeps
 * (a_i, b_j) exactly when C_ij > 0; its Sec. 3.2 turns C back into pairs with
 * nonzero(C).  This library evaluates that product over real-valued,
 * unit-norm embeddings: C_ij = s_ij = <a_i, b_j>, the exact real dot product
 * of the stored float32 rows, and returns
 *
 *   top-k   : for every left row i, the k right rows j with the largest s_ij,
 *             ordered by (s_ij desc, j asc), padded with (-1, -inf) when
 *             k > nB;
 *   threshold: every pair with s_ij >= tau, ordered by (i asc, j asc).
 *
 * Every emitted index set and order is the one the exact scores define, and
 * every emitted score is s_ij rounded to nearest-even float32, whatever
 * precision the tensor-core scoring runs in (cfg.prec): candidates near a
 * decision are rescored with a compensated FP32 dot product and, where even
 * that cannot decide, with an exact fixed-point accumulation.
 *
 * Memory.  Row-major float32 matrices, row i at A + i*d.  Every array pointer
 * may be DEVICE memory (used in place) or HOST memory (pageable or pinned;
 * staged through the handle's workspace with copies inside the call).  The
 * caller owns all arrays; the handle owns only its workspace, grown on demand
 * up to cfg.workspace_limit bytes and kept between calls.
 *
 * Synchronisation.  Work is queued on cfg.stream; every call returns after
 * that stream has drained the call's work (so status codes that depend on
 * device-side checks, and the stats, are final on return).  One handle must
 * not be used by two host threads at once.
 *
 * Errors.  Calls return a status code and never abort, trap or print.  Input
 * validation (finite values, |  ||x||^2 - 1 | <= 1e-5 per row) runs on the
 * device inside the call.  Device-side waits are bounded; a wait that gives up
 * returns SJ_ERR_TIMEOUT and leaves the context usable.
 */
#ifndef SJ_H_
#define SJ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SJ_OK = 0,
  SJ_ERR_INVALID_ARG = 1,   /* null pointer, bad size, k < 1, d < 1, NaN tau */
  SJ_ERR_NONFINITE = 2,     /* an input row holds NaN or Inf */
  SJ_ERR_NOT_UNIT_NORM = 3, /* an input row has | ||x||^2 - 1 | > 1e-5 */
  SJ_ERR_CAPACITY = 4,      /* output buffer too small; *n_out = required count */
  SJ_ERR_OOM = 5,           /* workspace allocation failed or over the limit */
  SJ_ERR_CUDA = 6,          /* a CUDA runtime/driver call failed */
  SJ_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  SJ_ERR_UNSUPPORTED = 8,   /* configuration not supported on this device */
  SJ_ERR_INTERNAL = 9       /* internal consistency check failed */
} sj_status;

/* Precision of the tensor-core scoring pass.  The emitted results do not
 * depend on it (see above); only speed and candidate counts do. */
typedef enum {
  SJ_FP32 = 0,     /* CUDA-core FP32 FMA tiles (no tensor cores) */
  SJ_BF16 = 1,     /* bfloat16 operands, FP32 accumulation in TMEM */
  SJ_FP8_E4M3 = 2, /* E4M3 with power-of-two scales: per row for A, per job for B */
  SJ_BF16X3 = 3    /* each float32 split into bfloat16 hi + lo; the tensor cores
                      sum hi.hi + hi.lo + lo.hi (one 3d-wide product): a proven
                      score error near 2^-16 plus accumulation instead of
                      2^-8, for data whose near-ties crowd the k-th score;
                      three times the BF16 work */
} sj_precision;

/* cfg.flags */
#define SJ_FLAG_SYM_INFONCE 0x1u   /* contrastive: add the column (B->A) term */
#define SJ_FLAG_SINGLE_SPLIT 0x2u  /* one column split per row block (each row's
                                      candidates collected in one list; lowers
                                      parallelism when nA is small) */
#define SJ_FLAG_NO_GRAPH 0x4u      /* never replay joins from a captured CUDA graph */
#define SJ_FLAG_NARROW_TILES 0x8u  /* test hook: 128-column score tiles for every job */
#define SJ_FLAG_FUSED_BACKWARD 0x10u /* sj_backward: never materialise dL/dS (see there) */
#define SJ_FLAG_BLOCK_SPARSE 0x20u  /* tensor-core scoring skips zero blocks: the packing
                                       pass records which 128-byte k-blocks of each
                                       128-row group hold a nonzero; a score tile loads
                                       and multiplies only the k-blocks nonzero on both
                                       sides (exact: a zero block adds exactly 0), and a
                                       threshold-only job skips the epilogue of an
                                       all-zero tile when tau exceeds its margin (the
                                       paper's block-sparse path for low density,
                                       Sec. 4.3).  Pays off for one-hot or sparse rows
                                       clustered by key; dense rows only pay the
                                       occupancy pass */
#define SJ_FLAG_DEBUG_TIMEOUT 0x100u /* test hook: device waits give up at once */

typedef struct {
  int device;             /* CUDA device ordinal */
  void *stream;           /* cudaStream_t; NULL = the legacy default stream */
  sj_precision prec;      /* scoring precision */
  int64_t d;              /* embedding width, >= 1 */
  uint32_t flags;         /* SJ_FLAG_* */
  size_t workspace_limit; /* bytes; 0 = no limit */
} sj_config;

/* One threshold result. 24 bytes; _pad is written as 0. */
typedef struct {
  int64_t i;
  int64_t j;
  float score;
  int32_t _pad;
} sj_pair;

/* Per-call statistics (optional; pass NULL to skip).  Times come from CUDA
 * events on cfg.stream. */
typedef struct {
  double ms_prepare;         /* validation + quantisation/packing (+ staging) */
  double ms_score;           /* tensor-core / FFMA scoring with fused filter */
  double ms_select;          /* rescoring, exact resolution, ordering, output */
  double ms_total;           /* whole call */
  int64_t n_candidates;      /* pairs that passed the low-precision filter */
  int64_t n_rescored;        /* pairs rescored with the compensated FP32 dot */
  int64_t n_exact;           /* pairs evaluated with the exact accumulator */
  int64_t n_overflow_rows;   /* rows whose band lists overflowed (re-joined, or re-ranked
                                against all of B) */
  int64_t n_pairs;           /* threshold: pairs emitted */
  double margin_max;         /* max proven bound m_i >= |s~ - s| over the rows whose
                                top-k were finalised (0 without a top-k part) */
  double max_abs_err_lowprec;/* max |s~ - s| seen over rescored top-k candidates */
  int64_t n_launches;        /* kernels this call launched */
  int64_t n_tier2_rows;      /* rows finalised with the large candidate tier */
  int64_t graph_replayed;    /* job groups run from a captured CUDA graph */
  double padded_pair_scores; /* pair-scores the score tiles computed, padding included */
  int64_t n_rejoined_rows;   /* overflowed rows (64 or more of a job) re-joined against
                                all of B by the next stage of the cascade: the BF16
                                hi/lo split with band lists sized by the columns they
                                cover, then FP32 */
  int64_t n_rejoined_again;  /* of those, rows whose lists overflowed there as well and
                                were re-joined by the stage after it (rows whose lists
                                were complete but long are ranked within the stage) */
} sj_stats;

typedef struct sj_handle sj_handle;

/* Create a handle bound to cfg->device.  Allocates no workspace yet.
 * Errors: SJ_ERR_INVALID_ARG (null, d < 1), SJ_ERR_UNSUPPORTED (device is not
 * compute capability 10.3 for SJ_BF16/SJ_FP8_E4M3), SJ_ERR_CUDA. */
sj_status sj_create(sj_handle **h, const sj_config *cfg);

/* Free the handle and its workspace.  NULL is accepted. */
sj_status sj_destroy(sj_handle *h);

/* Top-k join.  A: nA x d, B: nB x d float32 (device or host).  Outputs
 * out_idx[nA*k] (int64) and out_score[nA*k] (float32), row i at i*k, ordered
 * (score desc, j asc) with (-1, -inf) padding.  nA == 0 or nB == 0 is valid.
 * A == B (self-join) is allowed; the diagonal is included.
 * Errors: SJ_ERR_INVALID_ARG, SJ_ERR_NONFINITE, SJ_ERR_NOT_UNIT_NORM,
 * SJ_ERR_OOM, SJ_ERR_CUDA, SJ_ERR_TIMEOUT.  Outputs are undefined on error. */
sj_status sj_topk(sj_handle *h, const float *A, int64_t nA, const float *B,
                  int64_t nB, int32_t k, int64_t *out_idx, float *out_score,
                  sj_stats *st);

/* Threshold join: all (i, j) with s_ij >= tau, sorted by (i, j), written to
 * out[0 .. *n_out).  If more than `capacity` pairs qualify the call returns
 * SJ_ERR_CAPACITY with *n_out = the required count and out undefined.
 * Same input rules and errors as sj_topk. */
sj_status sj_threshold(sj_handle *h, const float *A, int64_t nA, const float *B,
                       int64_t nB, double tau, sj_pair *out, int64_t capacity,
                       int64_t *n_out, sj_stats *st);

/* One job of a batch: an independent join with its own sizes and outputs.
 * k > 0 requests the top-k part (topk_idx/topk_score required when nA > 0);
 * a non-NULL n_out requests the threshold part at tau (pairs required when
 * capacity > 0).  A job requesting neither is skipped.  All pointers follow
 * the same device/host rule as sj_topk. */
typedef struct {
  const float *A;
  int64_t nA;
  const float *B;
  int64_t nB;
  int32_t k;
  double tau;
  int64_t *topk_idx;
  float *topk_score;
  sj_pair *pairs;
  int64_t capacity;
  int64_t *n_out;
} sj_job;

/* Run n_jobs independent joins of the same d and precision as ONE pipeline:
 * one validation/packing launch over all rows, one persistent scoring launch
 * over every job's (row block, column split) units, and one finalisation.
 * Sec. 3.1 states one join as one matrix product; batching many uneven
 * products into one launch is this library's own addition.  A job that asks for both parts gets them from
 * the same scoring pass.  Results per job are exactly those of sj_topk /
 * sj_threshold.  Input checks cover the whole batch: a non-finite or
 * non-unit row in any job fails the call.  A job whose pairs exceed its
 * capacity writes no pairs and sets *n_out to the required count; the other
 * jobs complete and the call returns SJ_ERR_CAPACITY. */
sj_status sj_batch(sj_handle *h, const sj_job *jobs, int32_t n_jobs, sj_stats *st);

/* Autotuner of the score tile shape per size class of the right side (the
 * paper has no counterpart: its joins are single products).  For every class
 * c = 6..16 (nB in (2^(c-1), 2^c]) it times a synthetic top-k join of 8,192
 * unit rows against 0.75 * 2^c rows with 128- and 256-column tiles, and
 * keeps the faster width for later jobs of this handle with the same k and
 * class (untuned jobs use 128 columns up to nB = 128, else 256).  If `path`
 * is non-NULL the table is merged into that text file (one
 * "d precision k class width" line per entry).  Results never depend on the
 * width; only speed does.  Takes about a second.
 * Errors: SJ_ERR_INVALID_ARG (k outside 1..1024, unwritable path),
 * SJ_ERR_UNSUPPORTED (SJ_FP32: one tile shape), SJ_ERR_CUDA, SJ_ERR_OOM. */
sj_status sj_autotune(sj_handle *h, int32_t k, const char *path);

/* Load the widths that sj_autotune wrote to `path` for this handle's d and
 * precision.  Errors: SJ_ERR_INVALID_ARG (null or unreadable path). */
sj_status sj_autotune_load(sj_handle *h, const char *path);

/* Contrastive (InfoNCE) join over N paired rows, positives on the diagonal:
 * S = A B^T / T, l_i = logsumexp_j S_ij, loss = (1/N) sum_i (l_i - S_ii)
 * (with SJ_FLAG_SYM_INFONCE also the column term, averaged).  A, B: N x d
 * float32 rows in DEVICE memory, rounded to bfloat16 (nearest even) inside;
 * FP32 accumulation.  Writes loss[0] (device float) and lse[N] (2N with the
 * symmetric flag: rows then columns).
 * Errors: SJ_ERR_INVALID_ARG, SJ_ERR_UNSUPPORTED, SJ_ERR_CUDA, SJ_ERR_OOM. */
sj_status sj_contrastive_fwd(sj_handle *h, const void *A, const void *B, int64_t N,
                             float T, float *loss, float *lse);

/* Backward of sj_contrastive_fwd: given lse from the forward and the upstream
 * gradient grad_loss[0] (device float), writes dA, dB (N x d float32, device).
 * With G = dloss/dS rounded to bfloat16 (N x N, padded to multiples of 128):
 * dA = G B / T and dB = G^T A / T.  When the workspace can hold G (2 Np^2
 * bytes, Np = N rounded up to 256) one pass over the score tiles writes it
 * and two GEMMs read it (three products of 2 N^2 d flops);
 * otherwise, or with SJ_FLAG_FUSED_BACKWARD, G is recomputed per output chunk
 * of 384 dimensions and direction and never stored.  Both give the same G and
 * differ only in FP32 summation order.
 * Errors: SJ_ERR_INVALID_ARG, SJ_ERR_UNSUPPORTED, SJ_ERR_CUDA, SJ_ERR_OOM,
 * SJ_ERR_NONFINITE, SJ_ERR_TIMEOUT. */
sj_status sj_backward(sj_handle *h, const void *A, const void *B, int64_t N, float T,
                      const float *lse, const float *grad_loss, float *dA, float *dB);

/* Joins whose right table B stays in HOST memory (larger than the device's,
 * or simply not resident): B is streamed through the device in chunks of
 * `chunk_rows` rows (0: 1,048,576), the copy of the next chunk overlapping
 * the join of the current one on a second stream; the paper's pipelined
 * blocking for data larger than device memory (Sec. 4.3, MSplitGEMM).
 * Results are exactly those of sj_topk / sj_threshold on the whole of B:
 * threshold pairs are the chunks' pairs (columns offset by the chunk start)
 * merged by row; the top-k of a row is ranked exactly from the union of the
 * chunks' top-k lists (Dot2 intervals and the fixed-point accumulator, which
 * settles equal float32 scores of different chunks), reading those B rows
 * through B's mapped host address.  B is page-locked for the call
 * (cudaHostRegister) unless it already is.  A: device or host; top-k
 * outputs: device memory; threshold outputs: device or host.
 * Errors: SJ_ERR_INVALID_ARG (B not host memory, null, sizes), those of
 * sj_topk / sj_threshold. */
sj_status sj_topk_streamed(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                           int32_t k, int64_t chunk_rows, int64_t *out_idx, float *out_score,
                           sj_stats *st);
sj_status sj_threshold_streamed(sj_handle *h, const float *A, int64_t nA, const float *B,
                                int64_t nB, double tau, int64_t chunk_rows, sj_pair *out,
                                int64_t capacity, int64_t *n_out, sj_stats *st);

/* Row shard of the contrastive join, for data parallelism over rows (one
 * GPU per shard): A_rows are rows [r0, r0 + n_rows) of A (n_rows x d, DEVICE
 * float32), B all N rows of B, the positive of local row i is B row r0 + i,
 * and the loss keeps the global 1/N.  Writes lse_rows[n_rows] and
 * loss_part[0] = (1/N) sum_i (lse_i - S_i,r0+i): the shards' loss_part sum to
 * the loss of sj_contrastive_fwd (an all-reduce of one float).
 * One-directional loss only (SJ_FLAG_SYM_INFONCE: SJ_ERR_UNSUPPORTED).
 * Errors: SJ_ERR_INVALID_ARG (r0 + n_rows > N, ...) and those of
 * sj_contrastive_fwd. */
sj_status sj_contrastive_fwd_rows(sj_handle *h, const void *A_rows, int64_t n_rows, int64_t r0,
                                  const void *B, int64_t N, float T, float *loss_part,
                                  float *lse_rows);

/* Backward of sj_contrastive_fwd_rows: dA_rows (n_rows x d) is the gradient of
 * the shard's rows, dB_part (N x d) the shard's contribution to the gradient
 * of B (G_rows^T A_rows / T); the shards' dB_part sum to sj_backward's dB (an
 * all-reduce of N x d floats).  Same two paths (materialised or fused) as
 * sj_backward.  Errors as sj_backward, plus those of the forward's rows. */
sj_status sj_backward_rows(sj_handle *h, const void *A_rows, int64_t n_rows, int64_t r0,
                           const void *B, int64_t N, float T, const float *lse_rows,
                           const float *grad_loss, float *dA_rows, float *dB_part);

/* Exact top-k join that allocates nothing, for callers that cannot allocate
 * device memory at call time (their HBM is reserved in full by another
 * allocator's pool, or they must not call cudaMalloc/cudaFree, which can
 * synchronise the device).  The paper has no counterpart: this is a
 * deployment variant of sj_topk.  No handle is needed; the work runs on
 * `stream` (cudaStream_t, NULL = legacy default stream) of the current device.
 * Results equal sj_topk's.
 *
 * A, B: nA x d and nB x d float32 rows, out_idx/out_score: nA x k, all memory
 * of the CURRENT device (or managed memory) owned by the caller.  Limits:
 * nB <= 2048 (larger nB returns SJ_ERR_UNSUPPORTED), 1 <= k <= 1024 (k > nB
 * pads with (-1, -inf)).  Cost: one compensated FP32 dot product per pair on
 * 32 blocks, far slower than sj_topk when nA is large.
 * Scratch: one fixed device array of about 5.2 MB inside the library, held by
 * every GPU that loads it until the process exits.  The first call on each
 * device resolves that array's device address (cudaGetSymbolAddress).  All
 * calls on a device share the array and it keeps the previous call's contents
 * (the call clears its status area first): calls that overlap on the GPU
 * (other threads or streams) race and must be serialised by the caller.
 * The call is synchronous: it reads its status back and returns after
 * `stream` has drained its work, so it must not be called while `stream` is
 * being captured into a CUDA graph (it then returns SJ_ERR_INVALID_ARG
 * without enqueuing anything).
 * Errors: SJ_ERR_INVALID_ARG (null, host or other-device pointers, bad sizes,
 * stream under capture), SJ_ERR_UNSUPPORTED, SJ_ERR_NONFINITE,
 * SJ_ERR_NOT_UNIT_NORM, SJ_ERR_CUDA (sj_last_error_detail() names the
 * failing call).  Outputs are undefined on error. */
sj_status sj_topk_noalloc(const float *A, int64_t nA, const float *B, int64_t nB,
                          int64_t d, int32_t k, int64_t *out_idx, float *out_score,
                          void *stream);

/* ---- Precision planner (the paper's cost-based optimizer idea, Sec. 4.2:
 * feasibility test and cost estimation with Eq. (cost), CT ~ 2MNK / peak) ---- */

/* What sj_plan found.  Arrays are indexed by sj_precision. */
typedef struct {
  sj_precision choice;    /* the precision with the smallest est_ms */
  int32_t _pad;
  double est_ms[4];       /* predicted milliseconds of the whole join */
  double score_ms[4];     /* its scoring part: 2 nA nB d_p / (eff_p peak_p), Eq. (cost) */
  double select_ms[4];    /* its rescoring part, from the census (scaled by rows) */
  double cand_per_row[4]; /* census: candidates per sampled row that were rescored */
  double overflow_frac[4];/* census: sampled rows that took the rescan fallback */
  int64_t sample_rows;    /* rows of A in the census */
} sj_plan_info;

/* Choose the scoring precision of a join before running it.  Every precision
 * gives the same results (exact rescoring); they differ in tensor-core
 * cost (E4M3 issues twice the BF16 rate, the BF16 hi/lo split three times
 * the BF16 work, FP32 runs on the CUDA cores) and in how many candidates
 * their error margin lets through, which the data decides (a dense band
 * near the k-th score can overflow the candidate lists into a rescan of all
 * of B).  sj_plan runs a census: `sample_rows` evenly spaced rows of A
 * (0: 512) joined against all of B in each precision (k and/or tau as the
 * real join; k = 0 for none, tau = NaN for none), then predicts
 *   est_ms[p] = 2 nA nB d_p / (eff_p peak_p) + select_ms_sample[p] nA / s,
 * with peak_p = SMs x (8,192 BF16 | 16,384 E4M3 | 256 FP32) flop per clock
 * x the device's clock and eff_p the fraction of it this library's scoring
 * kernels reached on GB300 (bf16 0.71, e4m3 0.74, bf16x3 0.65, fp32 0.31).
 * A, B follow the sj_topk rules.  The handle's precision is not used.
 * Errors: SJ_ERR_INVALID_ARG (null, k < 0, neither k nor tau), the errors of
 * sj_batch. */
sj_status sj_plan(sj_handle *h, const float *A, int64_t nA, const float *B, int64_t nB,
                  int32_t k, double tau, int64_t sample_rows, sj_plan_info *info);

/* ---- Relational join patterns (Sec. 3.1 "Two-way natural join", Sec. 3.3
 * "Group-by aggregates over joins"; the entity-matching blocking of
 * Sec. 6.3.2) ---- */

/* Blocking / equi-join on key attributes.  Rows of A and B carry n_attr int64
 * key attributes (row-major: ka[i*n_attr + a], nA x n_attr and nB x n_attr;
 * device or host memory).  As in Sec. 3.1 every row becomes a one-hot row,
 * one block per attribute over that attribute's shared domain (values seen on
 * one side only get a column of their own side), scaled by
 * c = fl32(1/sqrt(n_attr)) so rows have unit norm, and C = mat(A) mat(B)^T
 * runs through the tensor-core threshold join of this library (bfloat16
 * scoring, exact rescoring) at tau = (min_match - 1/2) / n_attr.
 * Result: every (i, j) whose keys agree in at least min_match attributes
 * (n_attr = min_match = 1: the equi-join Q1, C_ij > 0), sorted by (i, j),
 * score = RN_fp32(matches * c^2) (= matches / n_attr for n_attr = 1 and 4).
 * Outputs and capacity rules as sj_threshold (out may be device or host).
 * The handle's d and precision are not used: the call runs through an
 * internal handle of the one-hot width, kept in h between calls.
 * Errors: SJ_ERR_INVALID_ARG (null, n_attr outside 1..64, min_match outside
 * 1..n_attr), SJ_ERR_CAPACITY, SJ_ERR_OOM, SJ_ERR_CUDA. */
sj_status sj_block(sj_handle *h, const int64_t *ka, int64_t nA, const int64_t *kb, int64_t nB,
                   int32_t n_attr, int32_t min_match, sj_pair *out, int64_t capacity,
                   int64_t *n_out, sj_stats *st);

/* One group of a join aggregate: its value, the exact SUM as a two's
 * complement 128-bit integer (sum_lo + 2^64 sum_hi) and COUNT(*). */
typedef struct {
  int64_t group;
  uint64_t sum_lo;
  int64_t sum_hi;
  int64_t count;
} sj_group;

/* Q3 of Sec. 3.3: SELECT B.G, SUM(A.Val), COUNT(*) FROM A, B
 * WHERE A.ID = B.ID GROUP BY B.G.  Every pair of the join counts (bag
 * semantics; the paper's 0/1 mat(B) gives the same result when B holds no
 * duplicate (ID, G) tuple).  Evaluated as the paper's product
 * 1 x mat(A) x mat(B)^T in its cheap association order: the per-key sums
 * 1 x mat(A) first, then one scatter per row of B; on GB300 both are atomic,
 * memory-bound kernels (a matrix product of one-hot operands would multiply
 * the work), with exact integer accumulation.  a_id, a_val (int32), b_id,
 * b_group: device or host arrays.  Writes the groups that have at least one
 * join pair, ordered by value, to out[0 .. *n_groups); with more groups than
 * `capacity` returns SJ_ERR_CAPACITY with *n_groups = the required count.
 * Errors: SJ_ERR_INVALID_ARG, SJ_ERR_CAPACITY, SJ_ERR_OOM, SJ_ERR_CUDA. */
sj_status sj_join_groupby_sum(sj_handle *h, const int64_t *a_id, const int32_t *a_val,
                              int64_t nA, const int64_t *b_id, const int64_t *b_group,
                              int64_t nB, sj_group *out, int64_t capacity, int64_t *n_groups);

/* Q4 of Sec. 3.3: SELECT SUM(A.Val * B.Val), COUNT(*) FROM A, B
 * WHERE A.ID = B.ID, i.e. 1 x mat(A) mat(B)^T x 1, evaluated as the per-key
 * sums of A dotted with B's values; exact 128-bit result in out->sum_lo /
 * out->sum_hi, the pair count in out->count (out->group = 0).
 * Errors: SJ_ERR_INVALID_ARG, SJ_ERR_OOM, SJ_ERR_CUDA. */
sj_status sj_join_sum_product(sj_handle *h, const int64_t *a_id, const int32_t *a_val,
                              int64_t nA, const int64_t *b_id, const int32_t *b_val, int64_t nB,
                              sj_group *out);

/* Test hook: arm the next sj_topk / sj_threshold / one-job sj_batch call of
 * this handle to also write what its scoring pass computed, so that the
 * margin argument can be checked pair by pair: raw[i*nB + j] = s~_ij, the
 * low-precision score of every pair of the join (float32, in score units,
 * i.e. E4M3 accumulators already scaled back), and margin[i] = m_i, the
 * proven bound |s~_ij - s_ij| <= m_i the fused filter relies on.  Both are
 * DEVICE buffers of the handle's device with room for nA*nB and nA floats.
 * The armed call runs without graph capture and fails with
 * SJ_ERR_INVALID_ARG if it holds more than one job; any call disarms the
 * hook.  Meant for small joins (it writes the whole score matrix).
 * Errors: SJ_ERR_INVALID_ARG (null, host or other-device buffers). */
sj_status sj_debug_scores(sj_handle *h, float *raw, float *margin);

/* Static description of a status code. */
const char *sj_status_string(sj_status s);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int sj_version(void);

/* Detail of the last CUDA failure behind an SJ_ERR_CUDA / SJ_ERR_OOM status
 * returned to the calling thread (error name, location, message); "" if none.
 * The string is owned by the library and valid until the thread's next call. */
const char *sj_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* SJ_H_ */
