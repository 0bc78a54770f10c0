// score_simt.cu -- plain FP32 scoring pass on the CUDA cores (no tensor cores).
//
// The comparison form of the join: s~_ij is the FP32 FMA chain
// acc <- fma(a_k, b_k, acc), k = 0..d-1, of the stored rows, so
// |s~ - s| <= gamma_d sum|a_k b_k| <= gamma_d ||a|| ||b|| (one rounding per
// step).  A persistent grid walks (row block, column split) units; per unit
// it computes 128 x 128 tiles with 8 x 8 register micro-tiles and hands each
// tile to the fused row filter through shared memory.
#include "epilogue.cuh"

namespace sj {

namespace {

constexpr int BM = kSimtBM, BN = kSimtBN, BK = kSimtBK;
constexpr int kThreads = 256;
constexpr int kSStride = BN + 1;

struct SimtSmem {
  float As[2][BK][BM];
  float Bs[2][BK][BN];
  float S[BM][kSStride];
};

__global__ void __launch_bounds__(kThreads, 2) score_simt_kernel(ScoreArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SimtSmem &sm = *reinterpret_cast<SimtSmem *>(smem_raw);
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const float *Ap = static_cast<const float *>(a.Ap);
  const float *Bp = static_cast<const float *>(a.Bp);
  const int64_t dp = a.dp;
  const int64_t nkt = dp / BK;
  if (*(volatile unsigned *)&a.ctr->err_flags & (kErrNonFinite | kErrNotUnit)) return;

  for (int64_t unit = blockIdx.x; unit < a.n_units; unit += gridDim.x) {
    const UnitDev un = a.units[unit];
    const JobDev &jb = a.jobs[un.job];
    const int64_t row0 = jb.a_prow0 + (int64_t)un.rb * BM;  // packed rows of A
    const int64_t lrow = (int64_t)un.rb * BM + tid;         // local row of this thread
    RowCtx rc;
    rc.cnt = 0;
    rc.overflow = 0;
    rc.k = jb.k;
    rc.theta = INFINITY;
    rc.tau_lo = INFINITY;
    rc.exact = false;  // theta refreshed lazily from the band list
    const bool owner = tid < BM && lrow < jb.nA;
    if (owner) row_begin(rc, a, jb, lrow, un.split);
    if (a.raw_m != nullptr && owner)
      a.raw_m[lrow] = row_margin(a.metaA[jb.a_prow0 + lrow], jb.gmaxB, a.acc_coef);
    const int64_t nB = jb.nB;
    const int64_t ct0 = (int64_t)un.split * jb.tiles_per_split;
    const int64_t ct1 = min64(jb.n_col_tiles, ct0 + jb.tiles_per_split);
    for (int64_t ct = ct0; ct < ct1; ++ct) {
      const int64_t col0 = ct * BN;                  // local column
      const int64_t bcol0 = jb.b_prow0 + col0;       // packed rows of B
      float acc[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

      // global -> register staging: thread loads rows r and r+64, 4 floats each
      const int lr = tid / 4, lc = (tid % 4) * 4;
      float4 ra[2], rb4[2];
      auto gload = [&](int64_t kt) {
        const int64_t k0 = kt * BK + lc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          ra[h] = *reinterpret_cast<const float4 *>(Ap + (row0 + lr + 64 * h) * dp + k0);
          rb4[h] = *reinterpret_cast<const float4 *>(Bp + (bcol0 + lr + 64 * h) * dp + k0);
        }
      };
      auto sstore = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          sm.As[buf][lc + 0][lr + 64 * h] = ra[h].x;
          sm.As[buf][lc + 1][lr + 64 * h] = ra[h].y;
          sm.As[buf][lc + 2][lr + 64 * h] = ra[h].z;
          sm.As[buf][lc + 3][lr + 64 * h] = ra[h].w;
          sm.Bs[buf][lc + 0][lr + 64 * h] = rb4[h].x;
          sm.Bs[buf][lc + 1][lr + 64 * h] = rb4[h].y;
          sm.Bs[buf][lc + 2][lr + 64 * h] = rb4[h].z;
          sm.Bs[buf][lc + 3][lr + 64 * h] = rb4[h].w;
        }
      };
      gload(0);
      sstore(0);
      __syncthreads();
      for (int64_t kt = 0; kt < nkt; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nkt) gload(kt + 1);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          float4 a0 = *reinterpret_cast<const float4 *>(&sm.As[buf][kk][ty * 4]);
          float4 a1 = *reinterpret_cast<const float4 *>(&sm.As[buf][kk][64 + ty * 4]);
          float4 b0 = *reinterpret_cast<const float4 *>(&sm.Bs[buf][kk][tx * 4]);
          float4 b1 = *reinterpret_cast<const float4 *>(&sm.Bs[buf][kk][64 + tx * 4]);
          float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < nkt) sstore(buf ^ 1);
        __syncthreads();
      }
      // tile -> shared memory
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
          sm.S[r][c] = acc[i][j];
        }
      }
      __syncthreads();
      if (tid < BM) {
        // the whole of warps 0-3 (the row owners) refreshes and compacts
        if (rc.k > 0) warp_compact<true>(rc, owner, rc.k, jb.cap - BN);
        if (owner) {
          const int ncol = (int)min64(BN, nB - col0);
          const float tmin = fminf(rc.theta, rc.tau_lo);
          for (int c = 0; c < ncol; ++c) {
            const float v = sm.S[tid][c];
            if (a.raw != nullptr) a.raw[lrow * nB + col0 + c] = v;
            if (v >= tmin) row_push(rc, a, v, (int32_t)(col0 + c));
          }
        }
      }
      __syncthreads();
    }
    if (owner) row_end(rc, a);
  }
}

}  // namespace

cudaError_t launch_score_simt(const ScoreArgs &a, int grid, cudaStream_t st) {
  if (a.n_units == 0) return cudaSuccess;
  const size_t smem = sizeof(SimtSmem);
  cudaError_t e = cudaFuncSetAttribute(score_simt_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  score_simt_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace sj
