// srs_score_tc.cu -- the proposal network over every cell of a coarse map, on
// the fifth-generation tensor cores.
//
// The network's first layer applied to all cells of an n_sigma map is a 2-D
// convolution: z1[m][b][j] = sum over the 9 x 33 patch around (m, b) of
// W1[j][r*33 + c] asinh(map[m + r - 4][b + c - 16]), i.e. a GEMM with M = the
// cells, K = 297 (padded to 304) and N = 64 hidden units.  Each CTA takes
// tiles of 128 consecutive bins of one template row: it stages the tile's
// 9 x 160 window of features (FP16), expands it into the 128 x 304 A operand
// in shared memory (im2col), and one thread issues 19 tcgen05.mma (kind::f16,
// M = 128, N = 64, K = 16) that accumulate z1 in FP32 in tensor memory.  The
// epilogue reads each cell's 64 sums back with tcgen05.ld (one TMEM lane per
// cell), adds b1, applies the ReLU and the output layer (w2, b2) and writes
// the logit.  W1 (FP16, the B operand) stays in shared memory for all of a
// CTA's tiles.  FP16 features and weights, FP32 accumulation: the precision
// the proposal specifies (FP16 weights with FP32 accumulation).
//
// Operand layout (PTX ISA, tcgen05 shared-memory matrix descriptors, no
// swizzling, K-major): 8 x 16-byte core matrices; a row's K elements k..k+7
// form one 16-byte line; core matrices adjacent in K are 128 bytes apart
// (leading byte offset), groups of 8 rows are 38 x 128 bytes apart (stride
// byte offset).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "srs_internal.h"
#include "srs_learn.h"

namespace srs {
namespace {

constexpr int kTcM = 128;                       // cells per tile (TMEM lanes)
constexpr int kTcN = kHidden;                   // 64 hidden units (TMEM columns)
constexpr int kTcK = 304;                       // 297 inputs padded to whole K = 16 steps
constexpr int kTcKSteps = kTcK / 16;            // 19 MMAs per tile
constexpr int kKCores = kTcK / 8;               // 38 core matrices along K
constexpr int kCoreBytes = 128;                 // 8 rows x 16 bytes
constexpr int kLbo = kCoreBytes;                // next core matrix along K
constexpr int kSbo = kKCores * kCoreBytes;      // next group of 8 rows: 4864 bytes
constexpr int kABytes = (kTcM / 8) * kSbo;      // 77 824
constexpr int kBBytes = (kTcN / 8) * kSbo;      // 38 912
constexpr int kWinCols = kTcM + kPatchBins - 1; // 160 bins of window per tile
constexpr int kWinBytes = kPatchTemplates * kWinCols * 2;
constexpr int kTmemCols = 64;                   // FP32 accumulator: 64 columns x 128 lanes
static_assert(kTcN == 64 && kTcK >= kPatchSize && kTcK % 16 == 0, "tile shape");
static_assert(kABytes % 1024 == 0 && kBBytes % 1024 == 0, "operand alignment");

// Instruction descriptor of kind::f16 (PTX ISA, tcgen05 instruction
// descriptor): D format F32 (bits 4-5 = 1), A and B F16 (bits 7-9, 10-12 = 0),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), the fixed
// version 1 (bit 46), base offset 0, no swizzling (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((kLbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((kSbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) of a K-major operand in the core-matrix layout.
__device__ __forceinline__ uint32_t core_offset(int row, int k) {
  return (uint32_t)((row >> 3) * kSbo + (k >> 3) * kCoreBytes + (row & 7) * 16 + (k & 7) * 2);
}

// Wait for phase `parity` of the mbarrier, giving up after ~2^31 cycles (about a second).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

}  // namespace

// One CTA of 128 threads (one warpgroup: warp w reads TMEM lanes 32w..32w+31)
// per SM, persistent over the tiles.
__global__ void __launch_bounds__(kTcM, 1)
k_score_tc(const float* __restrict__ map, int n_templates, int n_bins, const __half* __restrict__ W1h,
           const float* __restrict__ b1, const __half* __restrict__ w2h, const float* __restrict__ b2p,
           float* __restrict__ scores, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + kABytes;
  __half* win = reinterpret_cast<__half*>(smem + kABytes + kBBytes);
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  __shared__ float s_b1[kHidden], s_w2[kHidden];
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t bar = smem_u32(&s_bar);

  // tensor memory for the accumulator (warp 0 allocates and frees it)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  // B operand: W1 [64][297] FP16, zero-padded to K = 304
  for (int idx = tid; idx < kTcN * kTcK; idx += blockDim.x) {
    const int j = idx / kTcK, k = idx - j * kTcK;
    const __half v = k < kPatchSize ? W1h[j * kPatchSize + k] : __float2half(0.f);
    *reinterpret_cast<__half*>(sB + core_offset(j, k)) = v;
  }
  if (tid < kHidden) {
    s_b1[tid] = b1[tid];
    s_w2[tid] = __half2float(w2h[tid]);
  }
  const float b2 = *b2p;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);

  const int tiles_per_row = (n_bins + kTcM - 1) / kTcM;
  const long long tiles = (long long)n_templates * tiles_per_row;
  uint32_t parity = 0;
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int m = (int)(t / tiles_per_row);
    const int b0 = (int)(t - (long long)m * tiles_per_row) * kTcM;
    // window of features: templates m-4..m+4, bins b0-16 .. b0+143, zero outside the map
    for (int idx = tid; idx < kPatchTemplates * kWinCols; idx += blockDim.x) {
      const int r = idx / kWinCols, c = idx - r * kWinCols;
      const int mm = m + r - kPatchTemplates / 2, bb = b0 + c - kPatchBins / 2;
      float v = 0.f;
      if (mm >= 0 && mm < n_templates && bb >= 0 && bb < n_bins) v = asinhf(map[(long long)mm * n_bins + bb]);
      win[idx] = __float2half_rn(v);
    }
    __syncthreads();
    // A operand: row tid = the patch of cell (m, b0 + tid), k = r * 33 + c
    {
      int r = 0, c = 0;
      for (int k8 = 0; k8 < kKCores; ++k8) {
        __align__(16) __half v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const bool in = r < kPatchTemplates;
          v[e] = in ? win[r * kWinCols + tid + c] : __float2half(0.f);
          if (++c == kPatchBins) { c = 0; ++r; }
        }
        *reinterpret_cast<uint4*>(sA + core_offset(tid, k8 * 8)) = *reinterpret_cast<const uint4*>(v);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      for (int ks = 0; ks < kTcKSteps; ++ks) {
        const uint64_t ad = smem_desc(a_base + (uint32_t)(ks * 2 * kLbo));
        const uint64_t bd = smem_desc(b_base + (uint32_t)(ks * 2 * kLbo));
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(ks) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    // every thread waits for the accumulator (bounded: on a timeout the flag
    // is set and the CTA stops after freeing its tensor memory)
    if (!mbar_wait_bounded(bar, parity)) {
      s_abort = 1;
      if (atomicExch(err, 1) == 0) err[1] = (int)t;
    }
    parity ^= 1u;
    __syncthreads();
    if (s_abort) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: this thread's cell is TMEM lane tid
    float acc = b2;
#pragma unroll
    for (int q = 0; q < kTcN / 16; ++q) {
      float z[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 16), z);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int u = 0; u < 16; ++u) acc = fmaf(s_w2[q * 16 + u], fmaxf(z[u] + s_b1[q * 16 + u], 0.f), acc);
    }
    const int b = b0 + tid;
    if (b < n_bins) scores[(long long)m * n_bins + b] = acc;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // after a timeout, one more bounded wait for the MMAs in flight before the
  // tensor memory is freed
  if (s_abort && tid == 0) mbar_wait_bounded(bar, parity ^ 1u);
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

size_t score_tc_smem_bytes() { return (size_t)kABytes + kBBytes + kWinBytes; }

cudaError_t launch_score_tc(const float* map, int n_templates, int n_bins, const __half* W1h, const float* b1,
                            const __half* w2h, const float* b2, float* scores, int* err, int n_sm,
                            cudaStream_t st) {
  const size_t smem = score_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_score_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)n_templates * ((n_bins + kTcM - 1) / kTcM);
  const int grid = (int)(tiles < n_sm ? tiles : n_sm);
  if (grid <= 0) return cudaSuccess;
  k_score_tc<<<grid, kTcM, smem, st>>>(map, n_templates, n_bins, W1h, b1, w2h, b2, scores, err);
  return cudaGetLastError();
}

}  // namespace srs
