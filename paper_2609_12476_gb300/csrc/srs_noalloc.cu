// srs_noalloc.cu -- segment spectra without allocating device memory.
//
// Some callers cannot let a library call cudaMalloc or cudaFree.  A detector
// pipeline that hands all of a GPU's memory to its own allocator at start-up
// (a framework's caching allocator, a fixed arena) has nothing left for the
// library to grab, and a low-latency path cannot afford the device-wide
// synchronisation that cudaFree implies or the stall of a fresh allocation in
// the middle of a stream of segments.  srs_segment_spectra_static() serves
// them: it runs the same mixed-precision spreading / FFT / deconvolution
// kernel as srs_segment_spectra(), but every piece of scratch that kernel
// needs (its tables, work queue, error flag and, for float64 strain, the
// float32 copy of the samples) lives in the fixed array below, which is part
// of the library image and is held by every GPU that loads the library until
// the process exits.  The caller owns the strain and the output.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "srs_internal.h"
#include "srs_kernels.h"

namespace {

using namespace srs;

// Maximum scratch of one srs_segment_spectra_static() call.
constexpr size_t kStaticScratchBytes = (size_t)SRS_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per device (host code
// may not use the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {nullptr};

srs_status scratch_for_device(int dev, void** out, std::string& msg) {
  if (dev < 0 || dev >= kMaxDevices) {
    msg = "device ordinal out of range for the static scratch table";
    return SRS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      msg = std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e);
      return SRS_ERR_CUDA;
    }
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return SRS_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// True when p is device (or managed) memory of device `dev`: the scratch, the
// SM count and the launch all belong to the current device.
bool is_device_pointer_on(const void* p, int dev) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeManaged) return true;
  return attr.type == cudaMemoryTypeDevice && attr.device == dev;
}

void put_msg(char* buf, size_t len, const std::string& m) {
  if (buf && len > 0) {
    std::snprintf(buf, len, "%s", m.c_str());
  }
}

srs_status run(void* stream_v, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
               int32_t n_templates, int32_t seg_begin, int32_t seg_end, const srs_params* params, double* F,
               std::string& msg) {
  cudaStream_t st = static_cast<cudaStream_t>(stream_v);
  if (!strain || !F || !params || !mc) { msg = "strain, mc, params and F are required"; return SRS_ERR_ARG; }
  if (dtype != SRS_F32 && dtype != SRS_F64) { msg = "dtype must be SRS_F32 or SRS_F64"; return SRS_ERR_ARG; }
  if (params->precision != SRS_MIXED) { msg = "the static-scratch call runs the mixed form only"; return SRS_ERR_ARG; }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); msg = "cudaGetDevice failed"; return SRS_ERR_CUDA; }
  if (!is_device_pointer_on(strain, dev) || !is_device_pointer_on(F, dev)) {
    msg = "strain and F must be device pointers on the current device";
    return SRS_ERR_ARG;
  }
  Plan pl;
  srs_status s = make_plan(*params, mc, n_templates, n_samples, true, seg_begin, seg_end, pl, msg);
  if (s != SRS_OK) return s;

  // Layout of the scratch for this call.
  const size_t n_items = pl.items.size();
  // float64 strain: only the requested segments are converted to float32
  const int64_t samples = (int64_t)(seg_end - seg_begin) * pl.n_s;
  size_t off = 0;
  const size_t o_flags = off; off = align256(off + 64 + 64);          // queue, error flag
  const size_t o_betas = off; off = align256(off + (size_t)n_templates * sizeof(double));
  const size_t o_items = off; off = align256(off + n_items * sizeof(Item));
  const size_t o_corr = off; off = align256(off + (size_t)pl.n_bins * sizeof(float));
  const size_t o_tw = off; off = align256(off + (size_t)pl.n_fine * 2 * sizeof(float));
  const size_t o_x32 = off;
  if (dtype == SRS_F64) off = align256(off + (size_t)samples * sizeof(float));
  if (off > kStaticScratchBytes) {
    char b[256];
    std::snprintf(b, sizeof b, "this request needs %zu bytes of static scratch; the maximum is %zu bytes",
                  off, kStaticScratchBytes);
    msg = b;
    return SRS_ERR_ARG;
  }
  void* base_v = nullptr;
  s = scratch_for_device(dev, &base_v, msg);
  if (s != SRS_OK) return s;
  unsigned char* base = static_cast<unsigned char*>(base_v);
  int* queue = reinterpret_cast<int*>(base + o_flags);
  int* err = reinterpret_cast<int*>(base + o_flags + 64);
  double* d_betas = reinterpret_cast<double*>(base + o_betas);
  Item* d_items = reinterpret_cast<Item*>(base + o_items);
  float* d_corr = reinterpret_cast<float*>(base + o_corr);
  float* d_tw = reinterpret_cast<float*>(base + o_tw);
  float* d_x32 = reinterpret_cast<float*>(base + o_x32);

  const std::vector<float> corr = mixed_corr(pl);
  std::vector<float> tw(2 * (size_t)pl.n_fine);
  for (int m = 0; m < pl.n_fine; ++m) { tw[2 * m] = (float)pl.tw_re[m]; tw[2 * m + 1] = (float)pl.tw_im[m]; }

  auto ck = [&](cudaError_t e, const char* where) {
    if (e == cudaSuccess) return true;
    cudaGetLastError();
    msg = std::string(where) + ": " + cudaGetErrorString(e);
    return false;
  };
  // The array keeps the previous call's contents: the queue and error flag
  // must start at zero.
  if (!ck(cudaMemsetAsync(base + o_flags, 0, 128, st), "clear queue / error flag")) return SRS_ERR_CUDA;
  if (!ck(cudaMemcpyAsync(d_betas, pl.beta.data(), (size_t)n_templates * sizeof(double), cudaMemcpyHostToDevice, st), "copy betas") ||
      !ck(cudaMemcpyAsync(d_items, pl.items.data(), n_items * sizeof(Item), cudaMemcpyHostToDevice, st), "copy items") ||
      !ck(cudaMemcpyAsync(d_corr, corr.data(), corr.size() * sizeof(float), cudaMemcpyHostToDevice, st), "copy corr") ||
      !ck(cudaMemcpyAsync(d_tw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice, st), "copy twiddles"))
    return SRS_ERR_CUDA;
  int n_sm = 0;
  if (!ck(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev), "SM count")) return SRS_ERR_CUDA;
  const float* x32 = nullptr;
  // the same staging rule as srs_segment_spectra (SRS_NO_TMA=1: no TMA)
  int use_tma = (pl.n_s % 4) == 0 && !tma_disabled();
  if (dtype == SRS_F64) {
    const int64_t first = (int64_t)seg_begin * pl.n_s;
    if (!ck(launch_to_f32(static_cast<const double*>(strain) + first, d_x32, samples, n_sm, st), "k_to_f32"))
      return SRS_ERR_CUDA;
    // the kernel reads segment i at x32 + i n_s, so the base sits seg_begin
    // segments before the copy (integer arithmetic: no access lands there)
    x32 = reinterpret_cast<const float*>(reinterpret_cast<uintptr_t>(d_x32) - (uintptr_t)first * sizeof(float));
  } else {
    x32 = static_cast<const float*>(strain);
    if (((uintptr_t)x32 % 16) != 0) use_tma = 0;
  }

  MixedArgs a;
  std::memset(&a, 0, sizeof a);
  a.n_s = (int)pl.n_s;
  a.n_fine = pl.n_fine;
  a.n_bins = pl.n_bins;
  a.half_bins = pl.half_bins;
  a.run = pl.run;
  a.span = pl.span;
  a.n_anchor = pl.n_anchor;
  a.threads = pl.threads;
  a.n_pass = (int)pl.radices.size();
  a.ns4 = (int)((pl.n_s + 3) & ~3LL);
  a.nb4 = (pl.n_bins + 3) & ~3;
  a.chunk = pl.chunk;
  a.use_tma = use_tma;
  a.seg_begin = seg_begin;
  a.seg_range = seg_end - seg_begin;
  a.aa.fs = pl.fs;
  a.aa.t_coh = pl.t_coh;
  a.aa.f_c = pl.f_c;
  a.aa.n_s = pl.n_s;
  a.aa.span = pl.span;
  a.aa.n_anchor = pl.n_anchor;
  a.aa.local = 0;
  a.fft_fixed = (pl.n_fine == 1200 && pl.radices == std::vector<int32_t>{4, 4, 3, 5, 5}) ? 1200 : 0;
  a.kc = (float)pl.k_c;
  a.kc_int = (pl.k_c >= 1.0 && pl.k_c < 1073741824.0 && pl.k_c == std::floor(pl.k_c)) ? (int)pl.k_c : 0;
  a.inv_ns = (float)(1.0 / (double)pl.n_s);
  a.es_beta_log2e = mixed_es_e(pl);
  a.two_over_w = (float)(2.0 / pl.w);
  mixed_fixed_point(pl, a);
  a.corr = d_corr;
  a.tw = d_tw;
  for (size_t k = 0; k < pl.radices.size() && k < 16; ++k) a.radices[k] = (int8_t)pl.radices[k];

  if (!ck(launch_mixed(true, pl.w, x32, d_items, (int)n_items, d_betas, queue, a, nullptr,
                       reinterpret_cast<double2*>(F), err, n_sm, 0, st), "k_mixed"))
    return SRS_ERR_CUDA;
  int flag[5] = {0, 0, 0, 0, 0};
  if (!ck(cudaMemcpyAsync(flag, err, sizeof flag, cudaMemcpyDeviceToHost, st), "read error flag") ||
      !ck(cudaStreamSynchronize(st), "k_mixed"))
    return SRS_ERR_CUDA;
  if (flag[0]) {
    char buf[240];
    err_flag_message(flag, buf, sizeof buf);
    msg = buf;
    return SRS_ERR_TIMEOUT;
  }
  return SRS_OK;
}

}  // namespace

extern "C" srs_status srs_segment_spectra_static(void* cuda_stream, const void* strain, int64_t n_samples,
                                                 int32_t dtype, const double* mc, int32_t n_templates,
                                                 int32_t seg_begin, int32_t seg_end, const srs_params* params,
                                                 double* F, char* err_msg, size_t err_len) {
  std::string msg;
  srs_status s;
  try {
    s = run(cuda_stream, strain, n_samples, dtype, mc, n_templates, seg_begin, seg_end, params, F, msg);
  } catch (...) {
    s = SRS_ERR_OOM;
    msg = "host error while planning";
  }
  put_msg(err_msg, err_len, s == SRS_OK ? std::string() : msg);
  return s;
}
