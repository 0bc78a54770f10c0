// tc_host.h -- host side of the tensor-core scoring pass: TMA descriptors.
#pragma once

#include <cstdint>

#include "../../include/sj.h"
#include "sj_internal.h"

namespace sj {

struct TcContext;

// TMA tensor maps (opaque 128-byte CUtensorMap objects) for the packed
// operands: A tiles (128 rows), B tiles of 256 and of 128 rows.
struct TcMaps {
  alignas(64) unsigned char a[128];
  alignas(64) unsigned char b[128];
  alignas(64) unsigned char b128[128];
};

sj_status tc_create(TcContext **out);
void tc_destroy(TcContext *ctx);
// Maps over packed operands of `elem` bytes per element (2: BF16, 1: E4M3);
// every box is 128 bytes wide (one swizzle row).
sj_status tc_make_maps(TcContext *ctx, const void *Ap, int64_t nA_pad, const void *Bp,
                       int64_t nB_pad, int64_t dp, TcMaps *out, int elem = 2);
// fp8: E4M3 operands (tcgen05.mma kind::f8f6f4), else BF16 (kind::f16).
cudaError_t launch_score_tc(const ScoreArgs &a, int grid, const TcMaps *maps, uint32_t flags,
                            bool fp8, cudaStream_t st);
// Generic 2-D tensor map with 128-byte swizzle: `rows` rows of `inner`
// elements of `elem` bytes (2: BF16, 1: 8-bit), row stride = inner, box of
// box_inner x box_rows.
sj_status tc_encode_2d(TcContext *ctx, const void *base, int64_t inner, int64_t rows,
                       int box_inner, int box_rows, unsigned char out[128], int elem = 2);

}  // namespace sj
