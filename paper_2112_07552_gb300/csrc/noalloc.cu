// noalloc.cu -- exact top-k join for small right tables that allocates nothing.
//
// Some callers cannot allocate device memory at call time: a serving process
// whose HBM is already reserved in full by another allocator's pool, or a
// latency-critical caller that must not trigger cudaMalloc / cudaFree (those
// calls can synchronise the whole device).  sj_topk_noalloc serves them: it
// needs no handle and no workspace; its scratch memory is one file-scope
// device array of fixed size, loaded with the library and kept by every GPU
// that loads it until the process exits.
//
// Computation: a first launch validates every right row once and stores an
// upper bound on its norm in the scratch; then, for every left row i, a block
// validates the row, computes the compensated FP32 (Dot2) score interval of
// every right row j, and ranks all nB candidates exactly with the same block
// ranker as the main path (rank.cuh), so results equal sj_topk's bit for bit.
// Rows are validated as in sj_topk.  Cost: one Dot2 per pair on 32 blocks,
// about nA * nB * d * 2 FP32 FMAs plus the ranking, far slower than sj_topk
// for large nA; the variant is for small right tables only.
//
// Limits: nB <= kNoAllocMaxB right rows (any nA), 1 <= k <= 1024, device
// pointers only.  The scratch is shared by every call on a device and keeps
// the last call's contents; calls whose work overlaps on the GPU (other host
// threads, other streams) race on it and must be serialised by the caller.
#include <mutex>

#include "../../include/sj.h"
#include "rank.cuh"
#include "sj_device.cuh"
#include "sj_internal.h"

namespace sj {
namespace {

constexpr int kNoAllocMaxB = 2048;  // right rows
constexpr int kNoAllocBlocks = 32;  // one scratch slot per block
constexpr int kNoAllocThreads = 256;
// per slot: U, L (8 B), Exact (40 B), j, v, perm, perm2, grp, sc (4 B), flag (1 B)
constexpr size_t kSlotBytes = (size_t)kNoAllocMaxB * (8 + 8 + sizeof(Exact) + 6 * 4 + 1);
constexpr size_t kStatusBytes = 256;  // Counters of the current call, cleared per call
static_assert(sizeof(Counters) <= kStatusBytes, "status area too small");
constexpr size_t kNormBytes = (size_t)kNoAllocMaxB * sizeof(float);  // right-row norm bounds
constexpr size_t kScratchBytes =
    kStatusBytes + kNormBytes + (size_t)kNoAllocBlocks * kSlotBytes;  // ~5.2 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch, resolved once per device (host code
// sees only a host-side stand-in for the symbol).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_addr[dev]);
  return cudaSuccess;
}

__device__ __forceinline__ void warp_sumsq(const float *x, int64_t d, float &s, float &c) {
  const int lane = threadIdx.x & 31;
  s = 0.f;
  c = 0.f;
  for (int64_t k = lane; k < d; k += 32) dot2_step(x[k], x[k], s, c);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    float s2 = __shfl_xor_sync(0xffffffffu, s, off);
    float c2 = __shfl_xor_sync(0xffffffffu, c, off);
    float t, q;
    two_sum(s, s2, t, q);
    s = t;
    c = __fadd_rn(__fadd_rn(c, c2), q);
  }
}

// Validation of one row (finite, | ||x||^2 - 1 | <= 1e-5) and an upper bound
// on its norm; the result is the same on every lane.
__device__ __forceinline__ float check_row(const float *x, int64_t d, Counters *ctr) {
  bool bad = false;
  for (int64_t k = threadIdx.x & 31; k < d; k += 32) bad |= !isfinite(x[k]);
  bad = __any_sync(0xffffffffu, bad);
  float s, c;
  warp_sumsq(x, d, s, c);
  const float n2 = __fadd_rn(s, c);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&ctr->err_flags, kErrNonFinite);
    else if (!(fabsf(n2 - 1.0f) <= 1e-5f)) atomicOr(&ctr->err_flags, kErrNotUnit);
  }
  return __fsqrt_ru(__fmul_ru(fmaxf(n2, 0.f), 1.0f + 0x1p-20f));
}

// Validation and norm bound of every right row, once per call (warp per row).
__global__ void __launch_bounds__(kNoAllocThreads)
    noalloc_norms_kernel(const float *B, int64_t nB, int64_t d, unsigned char *scratch) {
  Counters *ctr = reinterpret_cast<Counters *>(scratch);
  float *nrm = reinterpret_cast<float *>(scratch + kStatusBytes);
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < nB; j += nw) {
    const float nb = check_row(B + j * d, d, ctr);
    if ((threadIdx.x & 31) == 0) nrm[j] = nb;
  }
}

__global__ void __launch_bounds__(kNoAllocThreads)
    topk_noalloc_kernel(const float *A, int64_t nA, const float *B, int64_t nB, int64_t d, int k,
                        float dot2_coef_key, int64_t *out_idx, float *out_score,
                        unsigned char *scratch) {
  Counters *ctr = reinterpret_cast<Counters *>(scratch);
  const float *nrm_bs = reinterpret_cast<const float *>(scratch + kStatusBytes);
  unsigned char *base = scratch + kStatusBytes + kNormBytes + (size_t)blockIdx.x * kSlotBytes;
  const int n_pad = next_pow2(nB > 0 ? (int)nB : 1);
  CandArrays c;
  c.U = reinterpret_cast<long long *>(base);
  c.L = c.U + n_pad;
  c.ex = reinterpret_cast<Exact *>(c.L + n_pad);
  c.j = reinterpret_cast<int32_t *>(c.ex + n_pad);
  c.v = reinterpret_cast<float *>(c.j + n_pad);
  c.perm = reinterpret_cast<int32_t *>(c.v + n_pad);
  c.perm2 = c.perm + n_pad;
  c.grp = c.perm2 + n_pad;
  c.sc = reinterpret_cast<float *>(c.grp + n_pad);
  c.flag = reinterpret_cast<uint8_t *>(c.sc + n_pad);
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
  __shared__ float s_nrm_a;
  __shared__ unsigned s_bad;
  for (int64_t i = blockIdx.x; i < nA; i += gridDim.x) {
    const float *a = A + i * d;
    if (warp == 0) {
      float na = check_row(a, d, ctr);
      if (lane == 0) {
        s_nrm_a = na;
        s_bad = *(volatile unsigned *)&ctr->err_flags & (kErrNonFinite | kErrNotUnit);
      }
    }
    __syncthreads();
    // an input failed validation: the call returns an error and its outputs
    // are undefined, so no row is ranked any more (uniform over the block)
    if (s_bad) break;
    const float nrm_a = s_nrm_a;
    for (int64_t j = warp; j < nB; j += nwarps) {
      const float *b = B + j * d;
      const float nrm_b = nrm_bs[j];
      float hi, lo;
      dot2_warp(a, b, d, hi, lo);
      if (lane == 0) {
        long long K = dot2_key(hi, lo);
        long long D = dot2_halfwidth(dot2_coef_key, nrm_a, nrm_b);
        c.U[j] = K + D;
        c.L[j] = K - D;
        c.j[j] = (int32_t)j;
        c.v[j] = NAN;
      }
    }
    __syncthreads();
    rank_and_emit(c, (int)nB, k, a, B, d, out_idx + i * k, out_score + i * k, ctr);
  }
}

// Memory the current device `dev` can use in place: its own device memory or
// managed memory (device memory of another GPU is refused: no peer access is
// assumed).
bool is_device_memory(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Returns SJ_ERR_CUDA (or SJ_ERR_OOM) with sj_last_error_detail() set.
sj_status cuda_fail(cudaError_t e, const char *what, int line) {
  record_cuda_error(e, what, "noalloc.cu", line);
  return e == cudaErrorMemoryAllocation ? SJ_ERR_OOM : SJ_ERR_CUDA;
}
#define NA_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call, __LINE__); \
  } while (0)

}  // namespace
}  // namespace sj

using namespace sj;

extern "C" sj_status sj_topk_noalloc(const float *A, int64_t nA, const float *B, int64_t nB,
                                     int64_t d, int32_t k, int64_t *out_idx, float *out_score,
                                     void *stream) {
  if (nA < 0 || nB < 0 || d < 1 || k < 1 || k > 1024) return SJ_ERR_INVALID_ARG;
  if (nB > kNoAllocMaxB) return SJ_ERR_UNSUPPORTED;  // the fixed scratch holds kNoAllocMaxB rows
  if (d > (1 << 20) || nA >= (1ll << 31)) return SJ_ERR_UNSUPPORTED;
  if (nA == 0) return SJ_OK;
  if (!A || !out_idx || !out_score || (nB > 0 && !B)) return SJ_ERR_INVALID_ARG;
  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SJ_ERR_UNSUPPORTED;
  if (!is_device_memory(A, dev) || !is_device_memory(out_idx, dev) ||
      !is_device_memory(out_score, dev) || (nB > 0 && !is_device_memory(B, dev)))
    return SJ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The call reads its status back and synchronises: it cannot be captured.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NA_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return SJ_ERR_INVALID_ARG;
  unsigned char *scratch = nullptr;
  NA_CUDA(scratch_address(dev, &scratch));
  // Dot2 error coefficient in key units (as in the main path): lane chains of
  // n = ceil(d/32) products plus a 5-level combination.
  const double u = 0x1p-24;
  const double n = (double)((d + 31) / 32) + 1.0;
  const double g = n * u / (1.0 - n * u);
  const double coef = 2.0 * (g * g + 10.0 * u * (g + 5.0 * u)) * (1.0 + 1e-6) * 0x1p60;
  float coef_key = (float)coef;
  if ((double)coef_key < coef) coef_key = nextafterf(coef_key, INFINITY);
  NA_CUDA(cudaMemsetAsync(scratch, 0, kStatusBytes, st));
  if (nB > 0) {
    const int ngrid = (int)((nB + kNoAllocThreads / 32 - 1) / (kNoAllocThreads / 32));
    noalloc_norms_kernel<<<ngrid, kNoAllocThreads, 0, st>>>(B, nB, d, scratch);
    NA_CUDA(cudaGetLastError());
  }
  const int grid = (int)(nA < kNoAllocBlocks ? nA : kNoAllocBlocks);
  topk_noalloc_kernel<<<grid, kNoAllocThreads, 0, st>>>(A, nA, B, nB, d, k, coef_key, out_idx,
                                                        out_score, scratch);
  NA_CUDA(cudaGetLastError());
  Counters hc;
  NA_CUDA(cudaMemcpyAsync(&hc, scratch, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
  if (hc.err_flags & kErrNonFinite) return SJ_ERR_NONFINITE;
  if (hc.err_flags & kErrNotUnit) return SJ_ERR_NOT_UNIT_NORM;
  return SJ_OK;
}
