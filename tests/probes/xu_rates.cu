// xu_rates.cu -- throughput of the special-function (XU / MUFU) operations the
// mixed spreader issues per sample: sqrt.approx, ex2.approx, sin.approx and
// cos.approx (via __sincosf), plus FP32 FMA for scale.  Each thread runs four
// independent chains of ITERS operations; the result is operations per clock
// per SM at the clock the device reports.  Prints one JSON object.
// Every thread writes one float to out[global thread index] (in bounds).
#include <cstdio>
#include <cuda_runtime.h>

constexpr int ITERS = 4096;

__device__ __forceinline__ float ex2a(float x) { float y; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sqa(float x) { float y; asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

template <int OP>
__global__ void k_rate(float* out, float seed) {
  float a = seed + threadIdx.x * 1e-3f, b = a + 0.1f, c = a + 0.2f, d = a + 0.3f;
  for (int i = 0; i < ITERS; ++i) {
    if (OP == 0) { a = sqa(a) + 0.5f; b = sqa(b) + 0.5f; c = sqa(c) + 0.5f; d = sqa(d) + 0.5f; }
    if (OP == 1) { a = ex2a(a) * 0.5f; b = ex2a(b) * 0.5f; c = ex2a(c) * 0.5f; d = ex2a(d) * 0.5f; }
    if (OP == 2) {
      float s, co;
      __sincosf(a, &s, &co); a = s + co; __sincosf(b, &s, &co); b = s + co;
      __sincosf(c, &s, &co); c = s + co; __sincosf(d, &s, &co); d = s + co;
    }
    if (OP == 3) { a = fmaf(a, 0.999f, 0.5f); b = fmaf(b, 0.998f, 0.25f); c = fmaf(c, 0.997f, 0.5f); d = fmaf(d, 0.996f, 0.25f); }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a + b + c + d;
}

template <int OP>
double rate(float* out, int blocks, int threads, int n_sm, double clk_hz, int ops_per_iter) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_rate<OP><<<blocks, threads>>>(out, 1.0f);
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) k_rate<OP><<<blocks, threads>>>(out, 1.0f);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double ops = 5.0 * blocks * threads * (double)ITERS * ops_per_iter;
  return ops / (ms * 1e-3) / (n_sm * clk_hz);
}

int main() {
  int dev = 0, n_sm = 0, clk_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int threads = 256, blocks = n_sm * 8;
  float* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) return 1;
  const double clk = clk_khz * 1e3;
  const double r_sqrt = rate<0>(out, blocks, threads, n_sm, clk, 4);
  const double r_ex2 = rate<1>(out, blocks, threads, n_sm, clk, 4);
  const double r_sincos = rate<2>(out, blocks, threads, n_sm, clk, 8);  // sin and cos each count
  const double r_fma = rate<3>(out, blocks, threads, n_sm, clk, 4);
  const cudaError_t e = cudaGetLastError();
  cudaFree(out);
  std::printf("{\"sm_count\": %d, \"clock_mhz\": %.0f, \"sqrt_per_clk_sm\": %.2f, \"ex2_per_clk_sm\": %.2f, "
              "\"sincos_per_clk_sm\": %.2f, \"ffma_per_clk_sm\": %.2f, \"error\": \"%s\"}\n",
              n_sm, clk / 1e6, r_sqrt, r_ex2, r_sincos, r_fma, cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
