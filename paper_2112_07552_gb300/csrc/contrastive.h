// contrastive.h -- host-side declarations of the contrastive (InfoNCE) kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sj_device.cuh"

namespace sj {

struct ContrastiveArgs {
  int64_t n;            // paired rows
  int64_t d;            // embedding width
  int64_t np, dp;       // padded rows (multiple of 128) and width (multiple of 64)
  float T;              // temperature
  int n_chunks;         // backward: output-dimension chunks of <= 384
  // forward outputs
  float *lse_out;       // [n] natural-log logsumexp of the kernel's rows
  float *term_out;      // [n] lse - S_ii
  // backward inputs / outputs
  const float *lse_r;   // row-indexed logsumexp used by the w_r term
  const float *lse_c;   // column-indexed logsumexp used by the w_c term
  float wr, wc;         // weights of the two softmax terms
  const float *grad_loss;  // device scalar
  float *dX;            // [n][d] gradient of the kernel's row operand
  Counters *ctr;
  int debug_timeout;
};

size_t contrastive_smem_bytes(bool bwd);
cudaError_t launch_contrastive_pack(const float *X, int64_t n, int64_t d, void *Xp, void *XT,
                                    int64_t np, int64_t dp, unsigned *err, cudaStream_t st);
cudaError_t launch_contrastive_loss(const float *t1, const float *t2, int64_t n, float w1,
                                    float w2, float *loss, cudaStream_t st);
// tmX/tmY/tmZ: 128-byte CUtensorMap objects (X, Y: box 64 x 128; Z: box 64 x 64)
cudaError_t launch_contrastive(bool bwd, const void *tmX, const void *tmY, const void *tmZ,
                               const ContrastiveArgs &a, int grid, cudaStream_t st);

}  // namespace sj
