// contrastive.h -- host-side declarations of the contrastive (InfoNCE) kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sj_device.cuh"

namespace sj {

struct ContrastiveArgs {
  int64_t n;            // rows of the kernel's row operand X
  int64_t d;            // embedding width
  int64_t np, dp;       // padded rows of X (multiple of 256) and width (multiple of 64)
  int64_t ny, npy;      // rows of the column operand Y (score columns), padded
  int64_t diag_off;     // the positive of X row i is column i + diag_off (if in range)
  int64_t n_norm;       // N of the loss (1/N scale): all paired rows, over every shard
  float T;              // temperature
  int n_chunks;         // fused backward: output-dimension chunks of <= 384
  int n_splits;         // forward and G' pass: column splits of a row block
  int tiles_per_split;  // forward and G' pass: 256-column tiles per split
  // forward outputs
  float *lse_out;       // [n] natural-log logsumexp of the kernel's rows
  float *term_out;      // [n] lse - S_ii
  float *part_m, *part_l, *part_c;  // [2 n_splits][np] partial max / sum / sum
                                    // compensation (log2 domain) per (split, half)
  float *diag_out;      // [n] S_ii * T (accumulator units)
  // backward inputs / outputs
  const float *lse_r;   // row-indexed logsumexp used by the w_r term
  const float *lse_c;   // column-indexed logsumexp used by the w_c term
  float wr, wc;         // weights of the two softmax terms
  const float *grad_loss;  // device scalar
  float *dX;            // [n][d] gradient of the kernel's row operand
  Counters *ctr;
  int debug_timeout;
};

// Kernel modes of launch_contrastive.
constexpr int kContrastiveFwd = 0;       // lse and loss terms of the kernel's rows
constexpr int kContrastiveBwdFused = 1;  // dX with G' recomputed per output chunk
constexpr int kContrastiveGprime = 2;    // G' written to memory through tmZ

// dX = (g / (N T)) G Z from a materialised G (np x np BF16) and Z^T (dp x np).
struct ContrastiveGemmArgs {
  int64_t n, d, np, dp;    // output rows (valid, padded) and width
  int64_t kp;              // padded K (rows of Z)
  int64_t n_norm;          // N of the 1/N scale
  float T;
  int n_chunks;            // output-dimension chunks of <= 384
  const float *grad_loss;  // device scalar
  float *dX;               // [n][d]
  Counters *ctr;
};

size_t contrastive_smem_bytes(int mode);
// Column splits of the forward and the G' pass for np padded rows.
void contrastive_splits(int64_t np, int *n_splits, int *tiles_per_split);
size_t contrastive_gemm_smem_bytes();
cudaError_t launch_contrastive_pack(const float *X, int64_t n, int64_t d, void *Xp, void *XT,
                                    int64_t np, int64_t dp, unsigned *err, cudaStream_t st);
// loss = (w1 sum t1 + w2 sum t2) / n_norm over n terms each
cudaError_t launch_contrastive_loss(const float *t1, const float *t2, int64_t n, int64_t n_norm,
                                    float w1, float w2, float *loss, cudaStream_t st);
// tmX/tmY/tmZ: 128-byte CUtensorMap objects (X, Y: box 64 x 128; Z: Z^T with
// box 64 x 64 in the fused backward, the G' map with box 64 x 128 in the G'
// pass, null in the forward).  The forward also launches the merge of its
// partial row states into lse_out and term_out.
cudaError_t launch_contrastive(int mode, const void *tmX, const void *tmY, const void *tmZ,
                               const ContrastiveArgs &a, int grid, cudaStream_t st);
// dX = P Z * g / (N T) with P = G (trans false; tmG box 64 x 128) or P = G^T
// (trans true; tmG over the same G with box 64 x 64); tmZ: Z^T (box 64 x 64)
cudaError_t launch_contrastive_gemm(bool trans, const void *tmG, const void *tmZ,
                                    const ContrastiveGemmArgs &a, int grid, cudaStream_t st);

}  // namespace sj
