// srs_reduce.cu -- the statistic and the top-k of the semicoherent search.
//
// Sec. III.C of arXiv:2609.12476: the segment powers are summed with equal
// weights into n_sigma = (sum_i P_i - 2 N) / (2 sqrt(N)) (Eqs. weights,
// semicoherent_statistic), and the largest cells are kept.  The mixed form's
// k_mixed leaves one running sum of (P - 2) / 2 per work item (a chunk of a
// template's segments); k_reduce_mixed_top32 sums a template's items in
// order, writes the n_sigma map and selects the top k <= 32 on the way;
// k_reduce_mixed + k_topk_tile + k_keys_to_cands do the same for larger k.
// The plain FP64 form finishes its sums with k_finish_plain.
#include <cuda_runtime.h>
#include <cstdint>

#include "srs_internal.h"
#include "srs_kernels.h"
#include "srs_device.cuh"

namespace srs {

// ---------------------------------------------------------------------------
// Statistic and top-k keys
// ---------------------------------------------------------------------------
// make_key / key_value: srs_device.cuh

// Sum over items q0..q1-1 of partial[q][b], in item order (so the result does
// not depend on scheduling), with Neumaier's compensated FP32 summation: the
// error is a few units in the last place of the sum whatever the number of
// items.  GB300's FP64 pipe retires about two operations per clock per SM,
// which made a per-item FP64 add and conversion the bound of this pass; the
// compensated sum runs on the FP32 pipe.  Loads are issued eight at a time.
__device__ __forceinline__ double sum_items(const float* __restrict__ partial, int q0, int q1, int n_bins, int b) {
  float s = 0.f, c = 0.f;
  const float* p = partial + (long long)q0 * n_bins + b;
  int q = q0;
  for (; q + 8 <= q1; q += 8, p += 8ll * n_bins) {
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = p[(long long)u * n_bins];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float t = s + x[u];
      c += fabsf(s) >= fabsf(x[u]) ? (s - t) + x[u] : (x[u] - t) + s;
      s = t;
    }
  }
  for (; q < q1; ++q, p += n_bins) {
    const float x = *p;
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  return (double)s + (double)c;
}

// Mixed form: n_sigma[m][b] = (sum over the template's items of Z) / sqrt(nseg_m).
// One thread per (template, bin).
__global__ void k_reduce_mixed(const float* __restrict__ partial, const int* __restrict__ item_off,
                               const int* __restrict__ nseg, int n_templates, int n_bins, float* __restrict__ map,
                               unsigned long long* __restrict__ keys) {
  const long long total = (long long)n_templates * n_bins;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(f / n_bins);
    const int b = (int)(f - (long long)m * n_bins);
    const double z = sum_items(partial, item_off[m], item_off[m + 1], n_bins, b);
    const float v = (float)(z / sqrt((double)nseg[m]));
    if (map) map[f] = v;
    keys[f] = make_key(v, (uint32_t)f);
  }
}

// Warp-level top-32 lists: one key per lane, sorted descending across the
// lanes (lane 0 holds the largest); missing keys are 0.
__device__ __forceinline__ unsigned long long warp_sort32_desc(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, stride);
      const bool keep_max = ((lane & stride) == 0) == ((lane & size) == 0);
      v = keep_max ? (v > o ? v : o) : (v < o ? v : o);
    }
  }
  return v;
}
// The 32 largest of two descending lists: max against the other list
// reversed gives a bitonic sequence holding them, which a half-cleaner sorts.
__device__ __forceinline__ unsigned long long warp_merge32_desc(unsigned long long a, unsigned long long b) {
  const int lane = threadIdx.x & 31;
  const unsigned long long br = __shfl_sync(0xffffffffu, b, 31 - lane);
  unsigned long long v = a > br ? a : br;
#pragma unroll
  for (int stride = 16; stride > 0; stride >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, stride);
    v = ((lane & stride) == 0) ? (v > o ? v : o) : (v < o ? v : o);
  }
  return v;
}

// Mixed form with k <= 32: k_reduce_mixed's cells, and the top k on the way.
// Each warp keeps the top 32 keys of the cells it has reduced; each block
// merges its warps' lists into scratch; the last block to finish (a ticket
// taken after a fence; no block waits for another) merges the blocks' lists
// and writes the candidates.
__global__ void __launch_bounds__(256)
k_reduce_mixed_top32(const float* __restrict__ partial, const int* __restrict__ item_off,
                     const int* __restrict__ nseg, int n_templates, int n_bins, float* __restrict__ map, int k,
                     unsigned long long* __restrict__ scratch, int* __restrict__ ticket,
                     srs_candidate* __restrict__ cands) {
  __shared__ unsigned long long s_top[8][32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long total = (long long)n_templates * n_bins;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long top = 0ull;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
    const long long f = base + threadIdx.x;
    unsigned long long key = 0ull;
    if (f < total) {
      const int m = (int)(f / n_bins);
      const int b = (int)(f - (long long)m * n_bins);
      const double z = sum_items(partial, item_off[m], item_off[m + 1], n_bins, b);
      const float v = (float)(z / sqrt((double)nseg[m]));
      if (map) map[f] = v;
      key = make_key(v, (uint32_t)f);
    }
    top = warp_merge32_desc(top, warp_sort32_desc(key));
  }
  s_top[warp][lane] = top;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) top = warp_merge32_desc(top, s_top[w][lane]);
    scratch[(long long)blockIdx.x * 32 + lane] = top;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: merge every block's list (each already sorted)
  top = 0ull;
  for (int blk = warp; blk < (int)gridDim.x; blk += (int)(blockDim.x >> 5))
    top = warp_merge32_desc(top, __ldcg(&scratch[(long long)blk * 32 + lane]));
  s_top[warp][lane] = top;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) top = warp_merge32_desc(top, s_top[w][lane]);
    if (lane < k) {
      const uint32_t flat = ~(uint32_t)(top & 0xffffffffull);
      srs_candidate c;
      c.value = key_value(top);
      c.template_idx = (int32_t)(flat / (uint32_t)n_bins);
      c.bin = (int32_t)(flat % (uint32_t)n_bins);
      cands[lane] = c;
    }
    if (lane == 0) *ticket = 0;
  }
}

// Plain form: n_sigma = (S - 2 N) / (2 sqrt(N)) in FP64.
__global__ void k_finish_plain(const double* __restrict__ S, const int* __restrict__ nseg, int n_templates,
                               int n_bins, float* __restrict__ map, unsigned long long* __restrict__ keys) {
  const long long total = (long long)n_templates * n_bins;
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
       f += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(f / n_bins);
    const double N = (double)nseg[m];
    const float v = (float)((S[f] - 2.0 * N) / (2.0 * sqrt(N)));
    if (map) map[f] = v;
    keys[f] = make_key(v, (uint32_t)f);
  }
}

// Top-k of each tile of `tile` keys (a power of two, >= 2k): bitonic sort
// (descending) in shared memory, first k written to out[blockIdx.x * k ...].
// Missing keys are 0, which sorts below every real key.
__global__ void __launch_bounds__(512)
k_topk_tile(const unsigned long long* __restrict__ in, long long n, int k, int tile,
            unsigned long long* __restrict__ out) {
  extern __shared__ unsigned long long s[];
  const long long base = (long long)blockIdx.x * tile;
  for (int t = threadIdx.x; t < tile; t += blockDim.x) {
    const long long g = base + t;
    s[t] = g < n ? in[g] : 0ull;
  }
  __syncthreads();
  for (int size = 2; size <= tile; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < tile / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool desc = ((lo & size) == 0);
        const unsigned long long x = s[lo], y = s[hi];
        if ((x < y) == desc) { s[lo] = y; s[hi] = x; }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) out[(long long)blockIdx.x * k + t] = s[t];
}

__global__ void k_keys_to_cands(const unsigned long long* __restrict__ keys, int k, int n_bins,
                                srs_candidate* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k) return;
  const unsigned long long key = keys[t];
  const uint32_t flat = ~(uint32_t)(key & 0xffffffffull);
  srs_candidate c;
  c.value = key_value(key);
  c.template_idx = (int32_t)(flat / (uint32_t)n_bins);
  c.bin = (int32_t)(flat % (uint32_t)n_bins);
  out[t] = c;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_reduce_mixed(const float* partial, const int* item_off, const int* nseg, int n_templates,
                                int n_bins, float* map, unsigned long long* keys, int n_sm, cudaStream_t st) {
  long long total = (long long)n_templates * n_bins;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  k_reduce_mixed<<<(unsigned)blocks, 256, 0, st>>>(partial, item_off, nseg, n_templates, n_bins, map, keys);
  return cudaGetLastError();
}

cudaError_t launch_reduce_mixed_top32(const float* partial, const int* item_off, const int* nseg, int n_templates,
                                      int n_bins, float* map, int k, unsigned long long* scratch, int* ticket,
                                      srs_candidate* cands, int n_sm, cudaStream_t st) {
  if (k < 1 || k > 32) return cudaErrorInvalidValue;
  long long total = (long long)n_templates * n_bins;
  long long blocks = (total + 255) / 256;
  // kTop32BlocksPerSm = 8 blocks of 256 per SM fill it: the pass streams the
  // partial sums from HBM, and the loads in flight (eight per thread) bound it;
  // the scratch holds 32 keys per block
  if (blocks > (long long)n_sm * kTop32BlocksPerSm) blocks = (long long)n_sm * kTop32BlocksPerSm;
  k_reduce_mixed_top32<<<(unsigned)blocks, 256, 0, st>>>(partial, item_off, nseg, n_templates, n_bins, map, k,
                                                          scratch, ticket, cands);
  return cudaGetLastError();
}

cudaError_t launch_finish_plain(const double* S, const int* nseg, int n_templates, int n_bins, float* map,
                                unsigned long long* keys, int n_sm, cudaStream_t st) {
  long long total = (long long)n_templates * n_bins;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)n_sm * 16) blocks = (long long)n_sm * 16;
  k_finish_plain<<<(unsigned)blocks, 256, 0, st>>>(S, nseg, n_templates, n_bins, map, keys);
  return cudaGetLastError();
}

static int pow2_at_least(long long v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Tile of the next top-k level for `cur` keys: a power of two >= 2k, at most
// 1024 keys (4096 when 2k > 1024).
static int topk_tile(long long cur, int k) {
  const int kp = pow2_at_least(2 * (long long)k);
  int tile = pow2_at_least(cur);
  if (tile < kp) tile = kp;
  const int cap = kp > 1024 ? kTopkTile : 1024;
  if (tile > cap) tile = cap;
  return tile;
}

// Keys each of the two scratch buffers of launch_topk must hold (the first
// level writes the most).
long long topk_scratch_keys(long long n, int k) {
  const int tile = topk_tile(n, k);
  return ((n + tile - 1) / tile) * (long long)k;
}

// Reduce n keys to the top k (k <= 1024) through tiles; result in whichever
// of buf_a / buf_b (each topk_scratch_keys(n, k) keys) the last level wrote,
// returned in *result.
cudaError_t launch_topk(const unsigned long long* keys, long long n, int k, unsigned long long* buf_a,
                        unsigned long long* buf_b, const unsigned long long** result, int* launches,
                        cudaStream_t st) {
  const unsigned long long* src = keys;
  unsigned long long* dst = buf_a;
  long long cur = n;
  // a tile's keys (kTopkTile x 8 B = 32 KB of dynamic shared memory) fit the
  // default per-block limit, so no attribute is set
  static_assert(kTopkTile * 8 <= 48 * 1024, "top-k tile beyond the default dynamic shared memory");
  for (;;) {
    const int tile = topk_tile(cur, k);
    const long long tiles = (cur + tile - 1) / tile;
    const int threads = tile / 2 < 512 ? tile / 2 : 512;
    k_topk_tile<<<(unsigned)tiles, threads, (size_t)tile * 8, st>>>(src, cur, k, tile, dst);
    ++*launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cur = tiles * k;
    src = dst;
    if (tiles == 1) break;
    dst = (dst == buf_a) ? buf_b : buf_a;
  }
  *result = src;
  return cudaSuccess;
}

cudaError_t launch_keys_to_cands(const unsigned long long* keys, int k, int n_bins, srs_candidate* out,
                                 cudaStream_t st) {
  k_keys_to_cands<<<(k + 255) / 256, 256, 0, st>>>(keys, k, n_bins, out);
  return cudaGetLastError();
}

}  // namespace srs
