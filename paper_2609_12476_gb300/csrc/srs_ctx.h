// srs_ctx.h -- the context object behind srs_ctx* and the helpers every C ABI
// source of libsrs uses (internal).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "srs_internal.h"

namespace srs {

// A device buffer that only grows.
// Largest single device allocation the library makes (SIZE_MAX unless
// SRS_ALLOC_LIMIT_BYTES is set in the environment, read once per process): a
// larger request fails as out of memory without calling cudaMalloc, which
// lets tests drive the out-of-memory path without exhausting a GPU.
size_t alloc_limit();

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p) return cudaSuccess;
    if (bytes > alloc_limit()) return cudaErrorMemoryAllocation;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t b = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) cap = b;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

}  // namespace srs

struct srs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_sm = 0;
  std::string err;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  // last plan whose tables are on the device (key: call kind, sizes, params, templates)
  bool have_plan = false;
  std::vector<unsigned char> plan_key;
  srs::Plan plan;
  // the search's device sequence as a CUDA graph, and what it was captured for
  bool use_graphs = true;
  // refinement of a fine-template subset: run the layout the tuner picks for
  // whole banks of this shape (128 threads, global sample loads) instead of
  // tuning every one-off subset
  bool subset_layout = false;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  int graph_launches = 0;
  int ctas_per_sm = 0;      // 0: as many as fit
  // autotuned (segments per item, CTAs per SM) of the mixed spreader per shape
  struct Tuned {
    std::vector<unsigned char> key;
    int chunk, ctas, threads, global_x;
    double ms;
  };
  std::vector<Tuned> tuned;
  int* hflag = nullptr;     // pinned copies of the device error flag: [0] synchronous calls,
                            // [8 (1 + k)] the k-th srs_search_async since the last srs_sync
  // stream-ordered searches (srs_search_async) since the last srs_sync: per call
  // the events around the whole sequence (0, 1) and around the transform kernel (2, 3)
  static constexpr int kAsyncSlots = 256;
  cudaEvent_t aev[kAsyncSlots][4] = {};
  int async_n = 0;
  srs_status async_status = SRS_OK;   // a failure found when the slots ran out and were synced
  std::string async_err;
  srs_report async_rep = {};          // sizes of the last asynchronous call
  // cuFFT plan of the unfused comparison path (handle valid when fft_plan_ok)
  int fft_plan = 0;
  bool fft_plan_ok = false;
  int fft_n = 0;
  long long fft_batch = 0;
  // asynchronous searches from host strain: two device staging buffers filled
  // on a copy stream, so that the next call's upload overlaps this call's search
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t stage_ready[2] = {nullptr, nullptr}, stage_free[2] = {nullptr, nullptr};
  // events around a whole proposal search (it runs searches that use the others)
  cudaEvent_t pev[2] = {nullptr, nullptr};
  // the captured graph (kept for its event-record nodes, re-pointed per launch)
  cudaGraph_t graph = nullptr;
  cudaGraphNode_t graph_ev_node[2] = {nullptr, nullptr};
  srs::DevBuf items, order, grid, anchors, partial, betas, nseg, item_off, corr, tw, keys, topk_a, topk_b, cands, queue, strain,
      strain32, errflag, map, S, F, psi, th, im, ii;
  // two-stage search: power cube chunk, stack-slide tracks and running sums
  srs::DevBuf strain_stage0, strain_stage1;
  srs::DevBuf cube, slide_cell, slide_coef, slide_w2, slide_seff, slide_len, slide_beta0, slide_frac, slide_Z, slide_map,
      white_s, white_sums, white_musig;
  bool have_slide = false;
  bool slide_open = false;                // running sums started (SRS_SLIDE_FIRST) and not yet finished
  std::vector<unsigned char> slide_key;   // what slide_cell / slide_len were computed for
  std::vector<cudaEvent_t> slide_ev;      // per chunk: cube start, slide start, slide end
  std::vector<int> slide_len_host;        // track length per row (copy of slide_len)
  std::vector<double> slide_frac_host;    // t0 fraction per row
  long long slide_reads_total = -1;       // cube powers a whole search over these tracks sums
  // learned proposal
  srs::DevBuf xb, yb, z1, logits, dz, lossv, grad, wts, adam_m, adam_v, w1h, w2h, idx, patches, cells_m, cells_b,
      sp_items, sp_bins, sp_partial, sp_cells, sp_out, sp_betas, cmap, ccands, inj;
  std::vector<srs::DevBuf*> all_buffers() {
    return {&items, &order, &grid, &anchors, &partial, &betas, &nseg, &item_off, &corr, &tw, &keys, &topk_a, &topk_b, &cands,
            &queue, &strain, &strain32, &errflag, &map, &S, &F, &psi, &th, &im, &ii, &xb, &yb, &z1, &logits, &dz,
            &lossv, &grad, &wts, &adam_m, &adam_v, &w1h, &w2h, &idx, &patches, &cells_m, &cells_b, &sp_items,
            &sp_bins, &sp_partial, &sp_cells, &sp_out, &sp_betas, &cmap, &ccands, &inj, &cube, &slide_cell,
            &slide_coef, &slide_w2, &slide_seff, &slide_len, &slide_beta0, &slide_frac, &slide_Z, &slide_map,
            &strain_stage0, &strain_stage1, &white_s, &white_sums, &white_musig};
  }
};

namespace srs {

inline srs_status set_err(srs_ctx* c, srs_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

inline srs_status cuda_err(srs_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a non-sticky error so the context stays usable
  return set_err(c, e == cudaErrorMemoryAllocation ? SRS_ERR_OOM : SRS_ERR_CUDA, m);
}

// Milliseconds between two recorded events; 0 (and the runtime's error state
// cleared) when they cannot be compared.
inline float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.f;
  }
  return ms;
}

// Search entry used by the proposal pipeline (srs_capi.cpp).
srs_status search_impl(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                       int32_t n_templates, const srs_params* params, float* stat_map, srs_candidate* cands,
                       int32_t* n_cands, srs_report* report, bool async_mode = false);
// Wait for the stream and settle every srs_search_async since the last sync.
srs_status sync_impl(srs_ctx* ctx, srs_report* report);
srs_status strain_f32(srs_ctx* ctx, const void* dstrain, int32_t dtype, int64_t samples, int64_t n_s,
                      const float** out, int* use_tma);
// Strain on the device (the caller's pointer, or a staged copy of `samples` host samples).
srs_status stage_strain(srs_ctx* ctx, const void* strain, int64_t samples, int32_t dtype, int on_device,
                        const void** dev);
// Argument checks every strain-taking entry point shares.
srs_status check_common(srs_ctx* ctx, const void* strain, int32_t dtype, const srs_params* params);
// The local resampling bank (Sec. III.B): n_beta values uniform over [beta_min, beta_max].
std::vector<double> bank_betas(const srs_bank& bank);
srs_status check_bank(srs_ctx* ctx, const srs_bank* bank);
// Power cube of segments [seg_begin, seg_end), every bank entry, from FP32
// device strain (mixed form, per-segment templates), into the device cube
// [n_beta][n_bins][seg_end - seg_begin].  Queued on the context's stream
// without a sync; the caller clears and checks the error flag.
srs_status cube_device(srs_ctx* ctx, const float* s32, int64_t n_samples, const std::vector<double>& bank,
                       int32_t seg_begin, int32_t seg_end, const srs_params* params, float* dcube, int* launches,
                       const Plan** plan_out);
// Clear / read the device error flag of the mixed spreader.
srs_status clear_err_flag(srs_ctx* ctx);
srs_status read_err_flag(srs_ctx* ctx);

}  // namespace srs

#define SRS_CK(call, where)                                  \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return srs::cuda_err(ctx, e_, where); \
  } while (0)
