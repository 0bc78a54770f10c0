// relational.cu -- the paper's relational join patterns on this library.
//
// sj_block (Sec. 3.1 "Two-way natural join", the entity-matching blocking of
// Sec. 6.3.2): key attributes become one-hot rows (one block per attribute,
// scaled to unit norm) and the join C = mat(A) mat(B)^T runs through the
// tensor-core threshold join at tau = (min_match - 1/2) / n_attr, with the
// block-sparse scoring of SJ_FLAG_BLOCK_SPARSE (tables clustered by key leave
// most k-blocks and tiles without a common nonzero).
//
// sj_join_groupby_sum / sj_join_sum_product (Sec. 3.3, Q3 and Q4): the
// paper writes them as 1 x mat(A) x mat(B)^T (x 1).  Associated from the
// left, 1 x mat(A) is a per-key sum over A and the product with mat(B)^T a
// per-row scatter over B: memory-bound, atomic kernels on GB300 (a one-hot
// matrix product would multiply the work by the key domain).  Sums are exact
// 128-bit integers (int32 values; per-key sums stay below 2^62 for fewer than
// 2^31 rows, group sums below 2^93, the Q4 total below 2^125).
//
// Keys are dictionary-encoded on the host (hash maps over the key columns),
// the step the paper calls converting the tables into matrix format.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "../../include/sj.h"
#include "sj_internal.h"

namespace sj {
namespace {

sj_status rl_fail(cudaError_t e, const char *what, int line) {
  record_cuda_error(e, what, "relational.cu", line);
  return e == cudaErrorMemoryAllocation ? SJ_ERR_OOM : SJ_ERR_CUDA;
}
#define RL_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return rl_fail(e__, #call, __LINE__); \
  } while (0)

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
  template <class T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

// 0: host memory, 1: memory of device `dev` (or managed), -1: another GPU's.
int where(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (at.type == cudaMemoryTypeManaged) return 1;
  if (at.type == cudaMemoryTypeDevice) return at.device == dev ? 1 : -1;
  return 0;
}

template <class T>
sj_status to_host(const T *p, int64_t n, int dev, cudaStream_t st, std::vector<T> &out) {
  out.resize((size_t)n);
  if (n == 0) return SJ_OK;
  const int w = where(p, dev);
  if (w < 0) return SJ_ERR_INVALID_ARG;
  if (w == 1) {
    RL_CUDA(cudaMemcpyAsync(out.data(), p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, st));
    RL_CUDA(cudaStreamSynchronize(st));
  } else {
    std::memcpy(out.data(), p, (size_t)n * sizeof(T));
  }
  return SJ_OK;
}

// Copy host bytes to dst, which may be host or device memory.
sj_status store(void *dst, const void *src, size_t bytes, int dev, cudaStream_t st) {
  if (bytes == 0) return SJ_OK;
  const int w = where(dst, dev);
  if (w < 0) return SJ_ERR_INVALID_ARG;
  if (w == 1) {
    RL_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    RL_CUDA(cudaStreamSynchronize(st));
  } else {
    std::memcpy(dst, src, bytes);
  }
  return SJ_OK;
}

template <class T>
sj_status to_device(const std::vector<T> &v, DevBuf &b, cudaStream_t st) {
  RL_CUDA(b.alloc(v.size() * sizeof(T)));
  if (!v.empty())
    RL_CUDA(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return SJ_OK;
}

int grid_for(int64_t n, int threads, int sm_count) {
  const int64_t g = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sm_count * 8));
}

// ---------------------------------------------------------------------------
// Kernels

// X (zeroed, n x d) gets `scale` at every entry's column: entry t belongs to
// row t / n_attr.
__global__ void onehot_scatter_kernel(const int32_t *cols, int64_t n_entries, int n_attr,
                                      int64_t d, float scale, float *X) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_entries;
       t += (int64_t)gridDim.x * blockDim.x)
    X[(t / n_attr) * d + cols[t]] = scale;
}

constexpr int kKeyPriv = 2048;  // keys summed in shared memory first (per block)
constexpr int kGrpPriv = 1024;  // groups summed in shared memory first

// 128-bit two's complement add of (plo, phi) into (*lo, *hi): the carry out of
// the low word comes from the value the atomic returned, so concurrent adds
// compose.
__device__ __forceinline__ void add128(unsigned long long *lo, unsigned long long *hi,
                                       unsigned long long plo, unsigned long long phi) {
  const unsigned long long old = atomicAdd(lo, plo);
  atomicAdd(hi, phi + (old + plo < old ? 1ull : 0ull));
}

// Per-key SUM (two's complement in 64 bits, exact below 2^63) and COUNT of
// A's values: 1 x mat(A) of Sec. 3.3.
__global__ void key_agg_kernel(const int32_t *code, const int32_t *val, int64_t n, int K,
                               unsigned long long *sum, unsigned long long *cnt) {
  __shared__ unsigned long long s_sum[kKeyPriv], s_cnt[kKeyPriv];
  const bool priv = K <= kKeyPriv;
  if (priv) {
    for (int t = threadIdx.x; t < K; t += blockDim.x) s_sum[t] = s_cnt[t] = 0ull;
    __syncthreads();
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = code[t];
    const unsigned long long v = (unsigned long long)(long long)val[t];
    atomicAdd(priv ? &s_sum[c] : &sum[c], v);
    atomicAdd(priv ? &s_cnt[c] : &cnt[c], 1ull);
  }
  if (priv) {
    __syncthreads();
    for (int t = threadIdx.x; t < K; t += blockDim.x)
      if (s_cnt[t]) {
        atomicAdd(&sum[t], s_sum[t]);
        atomicAdd(&cnt[t], s_cnt[t]);
      }
  }
}

// Q3: every row of B with a key of A adds its key's SUM (sign-extended to 128
// bits) and COUNT to its group.
__global__ void group_agg_kernel(const int32_t *code, const int32_t *grp, int64_t n, int G,
                                 const unsigned long long *sum, const unsigned long long *cnt,
                                 unsigned long long *g_lo, unsigned long long *g_hi,
                                 unsigned long long *g_cnt) {
  __shared__ unsigned long long s_lo[kGrpPriv], s_hi[kGrpPriv], s_cnt[kGrpPriv];
  const bool priv = G <= kGrpPriv;
  if (priv) {
    for (int t = threadIdx.x; t < G; t += blockDim.x) s_lo[t] = s_hi[t] = s_cnt[t] = 0ull;
    __syncthreads();
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = code[t];
    if (c < 0) continue;
    const int g = grp[t];
    const unsigned long long s = sum[c];
    const unsigned long long sh = (long long)s < 0 ? ~0ull : 0ull;
    if (priv) {
      add128(&s_lo[g], &s_hi[g], s, sh);
      atomicAdd(&s_cnt[g], cnt[c]);
    } else {
      add128(&g_lo[g], &g_hi[g], s, sh);
      atomicAdd(&g_cnt[g], cnt[c]);
    }
  }
  if (priv) {
    __syncthreads();
    for (int t = threadIdx.x; t < G; t += blockDim.x)
      if (s_cnt[t]) {
        add128(&g_lo[t], &g_hi[t], s_lo[t], s_hi[t]);
        atomicAdd(&g_cnt[t], s_cnt[t]);
      }
  }
}

// Q4: SUM over B's rows of key SUM x B.Val (128-bit products and total) and
// the pair count; per-thread partials, then one atomic pair per warp.
__global__ void dot_agg_kernel(const int32_t *code, const int32_t *val, int64_t n,
                               const unsigned long long *sum, const unsigned long long *cnt,
                               unsigned long long *tot) {
  __int128 acc = 0;
  unsigned long long c_acc = 0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = code[t];
    if (c < 0) continue;
    acc += (__int128)(long long)sum[c] * (__int128)val[t];
    c_acc += cnt[c];
  }
  unsigned long long lo = (unsigned long long)acc;
  unsigned long long hi = (unsigned long long)(acc >> 64);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const unsigned long long lo2 = __shfl_down_sync(0xffffffffu, lo, off);
    const unsigned long long hi2 = __shfl_down_sync(0xffffffffu, hi, off);
    const unsigned long long c2 = __shfl_down_sync(0xffffffffu, c_acc, off);
    const unsigned long long nl = lo + lo2;
    hi = hi + hi2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
    c_acc += c2;
  }
  if ((threadIdx.x & 31) == 0) {
    add128(&tot[0], &tot[1], lo, hi);
    atomicAdd(&tot[2], c_acc);
  }
}

sj_status check_inputs(sj_handle *h, const void *const *ptrs, const int64_t *ns, int np) {
  for (int q = 0; q < np; ++q)
    if (ns[q] > 0 && (!ptrs[q] || where(ptrs[q], handle_device(h)) < 0)) return SJ_ERR_INVALID_ARG;
  return SJ_OK;
}

// Keys of A -> codes 0..K-1 (first appearance); B's keys -> A's code or -1.
void encode_keys(const std::vector<int64_t> &a, const std::vector<int64_t> &b,
                 std::vector<int32_t> &ca, std::vector<int32_t> &cb, int &K) {
  std::unordered_map<int64_t, int32_t> m;
  m.reserve(a.size() * 2 + 1);
  ca.resize(a.size());
  for (size_t i = 0; i < a.size(); ++i) ca[i] = m.emplace(a[i], (int32_t)m.size()).first->second;
  K = (int)m.size();
  cb.resize(b.size());
  for (size_t j = 0; j < b.size(); ++j) {
    auto it = m.find(b[j]);
    cb[j] = it == m.end() ? -1 : it->second;
  }
}

}  // namespace
}  // namespace sj

using namespace sj;

extern "C" sj_status sj_block(sj_handle *h, const int64_t *ka, int64_t nA, const int64_t *kb,
                              int64_t nB, int32_t n_attr, int32_t min_match, sj_pair *out,
                              int64_t capacity, int64_t *n_out, sj_stats *st) {
  if (!h || nA < 0 || nB < 0 || n_attr < 1 || n_attr > 64 || min_match < 1 ||
      min_match > n_attr || !n_out || capacity < 0 || (capacity > 0 && !out))
    return SJ_ERR_INVALID_ARG;
  if (nA >= (1ll << 31) || nB >= (1ll << 31)) return SJ_ERR_UNSUPPORTED;
  const int dev = handle_device(h);
  cudaStream_t stm = static_cast<cudaStream_t>(handle_stream(h));
  RL_CUDA(cudaSetDevice(dev));
  const void *ptrs[2] = {ka, kb};
  const int64_t ns[2] = {nA, nB};
  if (check_inputs(h, ptrs, ns, 2) != SJ_OK) return SJ_ERR_INVALID_ARG;
  if (st) std::memset(st, 0, sizeof *st);
  std::vector<int64_t> ha, hb;
  sj_status s = to_host(ka, nA * n_attr, dev, stm, ha);
  if (s == SJ_OK) s = to_host(kb, nB * n_attr, dev, stm, hb);
  if (s != SJ_OK) return s;
  // One block per attribute: B's distinct values, then one column for A's
  // values that B lacks (no B row has it, so they never match).
  std::vector<int32_t> ca((size_t)nA * n_attr), cb((size_t)nB * n_attr);
  int64_t d = 0;
  for (int a = 0; a < n_attr; ++a) {
    std::unordered_map<int64_t, int32_t> m;
    m.reserve((size_t)nB * 2 + 1);
    for (int64_t j = 0; j < nB; ++j) {
      const int32_t code = m.emplace(hb[(size_t)j * n_attr + a], (int32_t)m.size()).first->second;
      cb[(size_t)j * n_attr + a] = (int32_t)(d + code);
    }
    const int64_t K = (int64_t)m.size();
    for (int64_t i = 0; i < nA; ++i) {
      auto it = m.find(ha[(size_t)i * n_attr + a]);
      ca[(size_t)i * n_attr + a] = (int32_t)(d + (it == m.end() ? K : it->second));
    }
    d += K + 1;
  }
  sj_handle *ax = nullptr;
  // one-hot rows are sparse: score only the blocks with a common nonzero
  s = aux_handle(h, std::max<int64_t>(d, 1), SJ_BF16, &ax, SJ_FLAG_BLOCK_SPARSE);
  if (s != SJ_OK) return s;
  DevBuf xa, xb, dca, dcb;
  RL_CUDA(xa.alloc((size_t)nA * d * 4));
  RL_CUDA(xb.alloc((size_t)nB * d * 4));
  RL_CUDA(cudaMemsetAsync(xa.p, 0, (size_t)nA * d * 4, stm));
  RL_CUDA(cudaMemsetAsync(xb.p, 0, (size_t)nB * d * 4, stm));
  s = to_device(ca, dca, stm);
  if (s == SJ_OK) s = to_device(cb, dcb, stm);
  if (s != SJ_OK) return s;
  const float scale = (float)(1.0 / std::sqrt((double)n_attr));
  const int sm = handle_sm_count(h);
  if (nA > 0) {
    onehot_scatter_kernel<<<grid_for(nA * n_attr, 256, sm), 256, 0, stm>>>(
        dca.as<int32_t>(), nA * n_attr, n_attr, d, scale, xa.as<float>());
    RL_CUDA(cudaGetLastError());
  }
  if (nB > 0) {
    onehot_scatter_kernel<<<grid_for(nB * n_attr, 256, sm), 256, 0, stm>>>(
        dcb.as<int32_t>(), nB * n_attr, n_attr, d, scale, xb.as<float>());
    RL_CUDA(cudaGetLastError());
  }
  const double tau = ((double)min_match - 0.5) / (double)n_attr;
  // sj_threshold returns after the stream drained its work: the one-hot
  // buffers may be freed afterwards
  s = sj_threshold(ax, xa.as<float>(), nA, xb.as<float>(), nB, tau, out, capacity, n_out, st);
  if (st) st->n_launches += 2;
  return s;
}

extern "C" sj_status sj_join_groupby_sum(sj_handle *h, const int64_t *a_id, const int32_t *a_val,
                                         int64_t nA, const int64_t *b_id, const int64_t *b_group,
                                         int64_t nB, sj_group *out, int64_t capacity,
                                         int64_t *n_groups) {
  if (!h || nA < 0 || nB < 0 || !n_groups || capacity < 0 || (capacity > 0 && !out))
    return SJ_ERR_INVALID_ARG;
  if (nA >= (1ll << 31) || nB >= (1ll << 31)) return SJ_ERR_UNSUPPORTED;
  const int dev = handle_device(h);
  cudaStream_t stm = static_cast<cudaStream_t>(handle_stream(h));
  RL_CUDA(cudaSetDevice(dev));
  const void *ptrs[4] = {a_id, a_val, b_id, b_group};
  const int64_t ns[4] = {nA, nA, nB, nB};
  if (check_inputs(h, ptrs, ns, 4) != SJ_OK || where(n_groups, dev) < 0) return SJ_ERR_INVALID_ARG;
  std::vector<int64_t> ha, hb, hg;
  std::vector<int32_t> hv;
  sj_status s = to_host(a_id, nA, dev, stm, ha);
  if (s == SJ_OK) s = to_host(b_id, nB, dev, stm, hb);
  if (s == SJ_OK) s = to_host(b_group, nB, dev, stm, hg);
  if (s == SJ_OK) s = to_host(a_val, nA, dev, stm, hv);
  if (s != SJ_OK) return s;
  std::vector<int32_t> ca, cb;
  int K = 0;
  encode_keys(ha, hb, ca, cb, K);
  // groups of the B rows that join, ordered by value
  std::vector<int64_t> gv;
  for (int64_t j = 0; j < nB; ++j)
    if (cb[j] >= 0) gv.push_back(hg[j]);
  std::sort(gv.begin(), gv.end());
  gv.erase(std::unique(gv.begin(), gv.end()), gv.end());
  const int64_t G = (int64_t)gv.size();
  int64_t need = G;
  s = store(n_groups, &need, 8, dev, stm);
  if (s != SJ_OK) return s;
  if (G > capacity) return SJ_ERR_CAPACITY;
  if (G == 0) return SJ_OK;
  std::vector<int32_t> gb((size_t)nB, 0);
  for (int64_t j = 0; j < nB; ++j)
    if (cb[j] >= 0) gb[j] = (int32_t)(std::lower_bound(gv.begin(), gv.end(), hg[j]) - gv.begin());
  DevBuf dca, dva, dcb, dgb, keyacc, grpacc;
  s = to_device(ca, dca, stm);
  if (s == SJ_OK) s = to_device(hv, dva, stm);
  if (s == SJ_OK) s = to_device(cb, dcb, stm);
  if (s == SJ_OK) s = to_device(gb, dgb, stm);
  if (s != SJ_OK) return s;
  RL_CUDA(keyacc.alloc((size_t)K * 16));
  RL_CUDA(grpacc.alloc((size_t)G * 24));
  RL_CUDA(cudaMemsetAsync(keyacc.p, 0, (size_t)K * 16, stm));
  RL_CUDA(cudaMemsetAsync(grpacc.p, 0, (size_t)G * 24, stm));
  unsigned long long *ksum = keyacc.as<unsigned long long>(), *kcnt = ksum + K;
  unsigned long long *glo = grpacc.as<unsigned long long>(), *ghi = glo + G, *gcnt = ghi + G;
  const int sm = handle_sm_count(h);
  if (nA > 0) {
    key_agg_kernel<<<grid_for(nA, 256, sm), 256, 0, stm>>>(dca.as<int32_t>(), dva.as<int32_t>(),
                                                          nA, K, ksum, kcnt);
    RL_CUDA(cudaGetLastError());
  }
  group_agg_kernel<<<grid_for(nB, 256, sm), 256, 0, stm>>>(dcb.as<int32_t>(), dgb.as<int32_t>(),
                                                          nB, (int)G, ksum, kcnt, glo, ghi, gcnt);
  RL_CUDA(cudaGetLastError());
  std::vector<unsigned long long> res((size_t)G * 3);
  RL_CUDA(cudaMemcpyAsync(res.data(), grpacc.p, (size_t)G * 24, cudaMemcpyDeviceToHost, stm));
  RL_CUDA(cudaStreamSynchronize(stm));
  std::vector<sj_group> groups((size_t)G);
  for (int64_t g = 0; g < G; ++g) {
    groups[g].group = gv[g];
    groups[g].sum_lo = res[g];
    groups[g].sum_hi = (int64_t)res[G + g];
    groups[g].count = (int64_t)res[2 * G + g];
  }
  return store(out, groups.data(), (size_t)G * sizeof(sj_group), dev, stm);
}

extern "C" sj_status sj_join_sum_product(sj_handle *h, const int64_t *a_id, const int32_t *a_val,
                                         int64_t nA, const int64_t *b_id, const int32_t *b_val,
                                         int64_t nB, sj_group *out) {
  if (!h || nA < 0 || nB < 0 || !out) return SJ_ERR_INVALID_ARG;
  if (nA >= (1ll << 31) || nB >= (1ll << 31)) return SJ_ERR_UNSUPPORTED;
  const int dev = handle_device(h);
  cudaStream_t stm = static_cast<cudaStream_t>(handle_stream(h));
  RL_CUDA(cudaSetDevice(dev));
  const void *ptrs[4] = {a_id, a_val, b_id, b_val};
  const int64_t ns[4] = {nA, nA, nB, nB};
  if (check_inputs(h, ptrs, ns, 4) != SJ_OK || where(out, dev) < 0) return SJ_ERR_INVALID_ARG;
  std::vector<int64_t> ha, hb;
  std::vector<int32_t> hva, hvb;
  sj_status s = to_host(a_id, nA, dev, stm, ha);
  if (s == SJ_OK) s = to_host(b_id, nB, dev, stm, hb);
  if (s == SJ_OK) s = to_host(a_val, nA, dev, stm, hva);
  if (s == SJ_OK) s = to_host(b_val, nB, dev, stm, hvb);
  if (s != SJ_OK) return s;
  std::vector<int32_t> ca, cb;
  int K = 0;
  encode_keys(ha, hb, ca, cb, K);
  sj_group r{};
  if (nA > 0 && nB > 0) {
    DevBuf dca, dva, dcb, dvb, keyacc, tot;
    s = to_device(ca, dca, stm);
    if (s == SJ_OK) s = to_device(hva, dva, stm);
    if (s == SJ_OK) s = to_device(cb, dcb, stm);
    if (s == SJ_OK) s = to_device(hvb, dvb, stm);
    if (s != SJ_OK) return s;
    RL_CUDA(keyacc.alloc((size_t)K * 16));
    RL_CUDA(tot.alloc(24));
    RL_CUDA(cudaMemsetAsync(keyacc.p, 0, (size_t)K * 16, stm));
    RL_CUDA(cudaMemsetAsync(tot.p, 0, 24, stm));
    unsigned long long *ksum = keyacc.as<unsigned long long>(), *kcnt = ksum + K;
    const int sm = handle_sm_count(h);
    key_agg_kernel<<<grid_for(nA, 256, sm), 256, 0, stm>>>(dca.as<int32_t>(), dva.as<int32_t>(),
                                                          nA, K, ksum, kcnt);
    RL_CUDA(cudaGetLastError());
    dot_agg_kernel<<<grid_for(nB, 256, sm), 256, 0, stm>>>(dcb.as<int32_t>(), dvb.as<int32_t>(),
                                                          nB, ksum, kcnt,
                                                          tot.as<unsigned long long>());
    RL_CUDA(cudaGetLastError());
    unsigned long long t3[3];
    RL_CUDA(cudaMemcpyAsync(t3, tot.p, 24, cudaMemcpyDeviceToHost, stm));
    RL_CUDA(cudaStreamSynchronize(stm));
    r.sum_lo = t3[0];
    r.sum_hi = (int64_t)t3[1];
    r.count = (int64_t)t3[2];
  }
  return store(out, &r, sizeof r, dev, stm);
}
