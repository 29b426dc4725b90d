// srs_capi.cpp -- the extern "C" entry points of libsrs (include/srs.h).
//
// Owns the per-context device workspace and stream, turns a host plan
// (srs_plan.cpp) into kernel launches (srs_kernels.cu), and copies results to
// the caller's buffers.  No exception crosses the ABI.
#include <cuda_runtime.h>
#include <cufft.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "srs_ctx.h"
#include "srs_internal.h"
#include "srs_kernels.h"

using namespace srs;

namespace srs {

// Strain on the device: the caller's pointer, or a copy of the first
// `samples` samples of the caller's host array.
srs_status stage_strain(srs_ctx* ctx, const void* strain, int64_t samples, int32_t dtype, int on_device,
                        const void** dev) {
  if (on_device) {
    *dev = strain;
    return SRS_OK;
  }
  size_t bytes = (size_t)samples * (dtype == SRS_F64 ? 8 : 4);
  SRS_CK(ctx->strain.ensure(bytes), "alloc strain");
  SRS_CK(cudaMemcpyAsync(ctx->strain.p, strain, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy strain");
  *dev = ctx->strain.p;
  return SRS_OK;
}

srs_status check_common(srs_ctx* ctx, const void* strain, int32_t dtype, const srs_params* params) {
  if (!ctx) return SRS_ERR_ARG;
  {
    // an error left by an earlier unchecked runtime call must not be blamed on this call
    const cudaError_t stale = cudaGetLastError();
    if (stale != cudaSuccess) std::fprintf(stderr, "srs: cleared stale CUDA error: %s\n", cudaGetErrorString(stale));
  }
  if (!strain) return set_err(ctx, SRS_ERR_ARG, "strain is NULL");
  if (!params) return set_err(ctx, SRS_ERR_ARG, "params is NULL");
  if (dtype != SRS_F32 && dtype != SRS_F64) return set_err(ctx, SRS_ERR_ARG, "dtype must be SRS_F32 or SRS_F64");
  if (params->io_on_device != 0 && params->io_on_device != 1) return set_err(ctx, SRS_ERR_ARG, "io_on_device must be 0 or 1");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "cudaSetDevice");
  return SRS_OK;
}

}  // namespace srs

namespace {

void fill_radices(const Plan& pl, int8_t* r) {
  for (int k = 0; k < 16; ++k) r[k] = 0;
  for (size_t k = 0; k < pl.radices.size() && k < 16; ++k) r[k] = (int8_t)pl.radices[k];
}

MixedArgs mixed_args(const Plan& pl, const srs_ctx* ctx, int seg_begin, int seg_range) {
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
  a.seg_begin = seg_begin;
  a.seg_range = seg_range;
  a.ns4 = (int)((pl.n_s + 3) & ~3LL);
  a.nb4 = (pl.n_bins + 3) & ~3;
  a.chunk = pl.chunk;
  a.use_tma = 0;
  a.aa.fs = pl.fs;
  a.aa.t_coh = pl.t_coh;
  a.aa.f_c = pl.f_c;
  a.aa.n_s = pl.n_s;
  a.aa.span = pl.span;
  a.aa.n_anchor = pl.n_anchor;
  a.aa.local = pl.local ? 1 : 0;
  a.fft_fixed = (pl.n_fine == 1200 && pl.radices == std::vector<int32_t>{4, 4, 3, 5, 5}) ? 1200 : 0;
  a.kc = (float)pl.k_c;
  a.kc_int = (pl.k_c >= 1.0 && pl.k_c < 1073741824.0 && pl.k_c == std::floor(pl.k_c)) ? (int)pl.k_c : 0;
  a.inv_ns = (float)(1.0 / (double)pl.n_s);
  a.es_beta_log2e = mixed_es_e(pl);
  a.two_over_w = (float)(2.0 / pl.w);
  mixed_fixed_point(pl, a);
  a.corr = ctx->corr.as<float>();
  a.tw = ctx->tw.as<float>();
  a.order = pl.order.empty() ? nullptr : ctx->order.as<int>();
  fill_radices(pl, a.radices);
  return a;
}

PlainArgs plain_args(const Plan& pl, const srs_ctx* ctx, int seg_begin, int seg_range) {
  PlainArgs p;
  std::memset(&p, 0, sizeof p);
  p.fs = pl.fs;
  p.t_coh = pl.t_coh;
  p.f_c = pl.f_c;
  p.beta_es = pl.beta_es;
  p.n_s = (int)pl.n_s;
  p.n_fine = pl.n_fine;
  p.n_bins = pl.n_bins;
  p.half_bins = pl.half_bins;
  p.w = pl.w;
  p.n_pass = (int)pl.radices.size();
  p.seg_begin = seg_begin;
  p.seg_range = seg_range;
  p.corr = ctx->corr.as<double>();
  p.tw = ctx->tw.as<double>();
  fill_radices(pl, p.radices);
  return p;
}

AnchorArgs anchor_args(const Plan& pl) {
  AnchorArgs aa;
  aa.local = pl.local ? 1 : 0;
  aa.fs = pl.fs;
  aa.t_coh = pl.t_coh;
  aa.f_c = pl.f_c;
  aa.n_s = pl.n_s;
  aa.span = pl.span;
  aa.n_anchor = pl.n_anchor;
  return aa;
}

// Upload the tables of a plan (deconvolution, twiddles, templates).
srs_status upload_tables(srs_ctx* ctx, const Plan& pl) {
  const bool mixed = pl.precision == SRS_MIXED;
  if (mixed) {
    const std::vector<float> corr = mixed_corr(pl);
    std::vector<float> tw(2 * pl.n_fine);
    for (int m = 0; m < pl.n_fine; ++m) { tw[2 * m] = (float)pl.tw_re[m]; tw[2 * m + 1] = (float)pl.tw_im[m]; }
    SRS_CK(ctx->corr.ensure(corr.size() * 4), "alloc corr");
    SRS_CK(ctx->tw.ensure(tw.size() * 4), "alloc tw");
    SRS_CK(cudaMemcpyAsync(ctx->corr.p, corr.data(), corr.size() * 4, cudaMemcpyHostToDevice, ctx->stream), "copy corr");
    SRS_CK(cudaMemcpyAsync(ctx->tw.p, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice, ctx->stream), "copy tw");
    SRS_CK(cudaStreamSynchronize(ctx->stream), "sync tables");
  } else {
    std::vector<double> tw(2 * pl.n_fine);
    for (int m = 0; m < pl.n_fine; ++m) { tw[2 * m] = pl.tw_re[m]; tw[2 * m + 1] = pl.tw_im[m]; }
    SRS_CK(ctx->corr.ensure(pl.corr.size() * 8), "alloc corr");
    SRS_CK(ctx->tw.ensure(tw.size() * 8), "alloc tw");
    SRS_CK(cudaMemcpyAsync(ctx->corr.p, pl.corr.data(), pl.corr.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "copy corr");
    SRS_CK(cudaMemcpyAsync(ctx->tw.p, tw.data(), tw.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "copy tw");
    SRS_CK(cudaStreamSynchronize(ctx->stream), "sync tables");
  }
  SRS_CK(ctx->betas.ensure(pl.beta.size() * 8), "alloc betas");
  SRS_CK(ctx->nseg.ensure(pl.nseg.size() * 4), "alloc nseg");
  SRS_CK(cudaMemcpyAsync(ctx->betas.p, pl.beta.data(), pl.beta.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "copy betas");
  SRS_CK(cudaMemcpyAsync(ctx->nseg.p, pl.nseg.data(), pl.nseg.size() * 4, cudaMemcpyHostToDevice, ctx->stream), "copy nseg");
  if (mixed && !pl.items.empty()) {
    SRS_CK(ctx->items.ensure(pl.items.size() * sizeof(Item)), "alloc items");
    SRS_CK(ctx->item_off.ensure(pl.item_off.size() * 4), "alloc item_off");
    SRS_CK(cudaMemcpyAsync(ctx->items.p, pl.items.data(), pl.items.size() * sizeof(Item), cudaMemcpyHostToDevice, ctx->stream), "copy items");
    SRS_CK(cudaMemcpyAsync(ctx->item_off.p, pl.item_off.data(), pl.item_off.size() * 4, cudaMemcpyHostToDevice, ctx->stream), "copy item_off");
  }
  SRS_CK(cudaStreamSynchronize(ctx->stream), "sync tables");
  return SRS_OK;
}

std::vector<unsigned char> make_key(int kind, const srs_params* p, int64_t n_samples, int32_t dtype, const double* mc,
                                    int32_t n_templates, int32_t a, int32_t b) {
  std::vector<unsigned char> k;
  auto put = [&](const void* d, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(d);
    k.insert(k.end(), c, c + n);
  };
  put(&kind, sizeof kind);
  put(p, sizeof *p);
  put(&n_samples, sizeof n_samples);
  put(&dtype, sizeof dtype);
  put(&a, sizeof a);
  put(&b, sizeof b);
  put(&n_templates, sizeof n_templates);
  if (mc && n_templates > 0) put(mc, sizeof(double) * (size_t)n_templates);
  return k;
}

// The search's small device words share one buffer (one memset per search):
// [0] work-queue counter, [4] top-k ticket, [16..20] error flag and where.
constexpr size_t kQueueBytes = 128;
int* search_errflag(srs_ctx* ctx) { return ctx->queue.as<int>() + 16; }

// Pinned error-flag copies: slot 0 for synchronous calls, one slot of eight
// ints per asynchronous call since the last srs_sync.
constexpr size_t kHostFlagBytes = (size_t)8 * (1 + srs_ctx::kAsyncSlots) * sizeof(int);

// An event around the transform kernel: inside a stream capture it must become
// an event-record node (external), outside one it is an ordinary record.
cudaError_t record_kernel_event(cudaEvent_t ev, cudaStream_t st, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st);
}

// Drop the captured search graph (an in-flight launch finishes on its own).
void destroy_graph(srs_ctx* ctx) {
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->graph_exec = nullptr;
  ctx->graph = nullptr;
  ctx->graph_ev_node[0] = ctx->graph_ev_node[1] = nullptr;
  ctx->graph_key.clear();
}

// The captured graph's event-record nodes for the context's transform-kernel
// events (ev2, ev3), so that each launch can point them at its own events.
void find_event_nodes(srs_ctx* ctx) {
  ctx->graph_ev_node[0] = ctx->graph_ev_node[1] = nullptr;
  size_t n = 0;
  if (cudaGraphGetNodes(ctx->graph, nullptr, &n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return;
  }
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(ctx->graph, nodes.data(), &n) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev = nullptr;
    if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
    if (ev == ctx->ev2) ctx->graph_ev_node[0] = nd;
    if (ev == ctx->ev3) ctx->graph_ev_node[1] = nd;
  }
  cudaGetLastError();
}

// Plan for this call, reusing the context's last plan (and its device tables)
// when the call kind, sizes, parameters and templates are the same.
srs_status get_plan(srs_ctx* ctx, int kind, const srs_params* params, const double* mc, int32_t n_templates,
                    int64_t n_samples, int32_t dtype, bool spectra_mode, int32_t a, int32_t b, const Plan** out,
                    const double* betas_in = nullptr, bool local = false) {
  srs_params key_p = *params;
  key_p.io_on_device = 0;
  std::vector<unsigned char> key = make_key(kind, &key_p, n_samples, dtype, betas_in ? betas_in : mc, n_templates, a, b);
  if (ctx->have_plan && key == ctx->plan_key) {
    *out = &ctx->plan;
    return SRS_OK;
  }
  ctx->have_plan = false;
  // a new plan means new tables: a captured graph may point at the old ones
  destroy_graph(ctx);
  std::string msg;
  srs_status s = make_plan(*params, mc, n_templates, n_samples, spectra_mode, a, b, ctx->plan, msg, betas_in, local);
  if (s != SRS_OK) return set_err(ctx, s, msg);
  s = upload_tables(ctx, ctx->plan);
  if (s != SRS_OK) return s;
  ctx->plan_key.swap(key);
  ctx->have_plan = true;
  *out = &ctx->plan;
  return SRS_OK;
}

}  // namespace

namespace srs {

size_t alloc_limit() {
  static const size_t limit = [] {
    const char* v = std::getenv("SRS_ALLOC_LIMIT_BYTES");
    if (!v || !*v) return (size_t)-1;
    char* end = nullptr;
    const unsigned long long b = std::strtoull(v, &end, 10);
    return (end && *end == '\0' && b > 0) ? (size_t)b : (size_t)-1;
  }();
  return limit;
}

// The mixed form reads FP32 samples: convert FP64 strain once per call, and
// use FP32 strain in place when TMA can read it (16-byte aligned, n_s % 4 == 0).
bool tma_disabled() {
  const char* no_tma = std::getenv("SRS_NO_TMA");
  return no_tma && no_tma[0] == '1';
}

void err_flag_message(const int* f, char* buf, size_t n) {
  if (f[0] == 2)
    std::snprintf(buf, n, "the spreader's cell walk reached its bound with samples unused (a time map that steps "
                  "back): item %d segment %d sample %d block %d", f[1], f[2], f[3], f[4]);
  else
    std::snprintf(buf, n, "a device wait gave up (TMA copy did not complete in time): item %d segment %d parity %d "
                  "block %d", f[1], f[2], f[3], f[4]);
}

srs_status strain_f32(srs_ctx* ctx, const void* dstrain, int32_t dtype, int64_t samples, int64_t n_s,
                      const float** out, int* use_tma) {
  // SRS_NO_TMA=1 in the environment selects plain shared-memory staging.
  const bool tma_ok_len = (n_s % 4) == 0 && !tma_disabled();
  if (dtype == SRS_F64) {
    SRS_CK(ctx->strain32.ensure((size_t)samples * 4), "alloc strain32");
    SRS_CK(launch_to_f32(static_cast<const double*>(dstrain), ctx->strain32.as<float>(), samples, ctx->n_sm,
                         ctx->stream), "k_to_f32");
    *out = ctx->strain32.as<float>();
    *use_tma = tma_ok_len ? 1 : 0;
    return SRS_OK;
  }
  const bool aligned = ((uintptr_t)dstrain % 16) == 0;
  *out = static_cast<const float*>(dstrain);
  *use_tma = (tma_ok_len && aligned) ? 1 : 0;
  return SRS_OK;
}

}  // namespace srs

namespace {

// Autotuner of the mixed spreader: segments per work item, threads per CTA
// (256, or 128 where the anchor expansion stays accurate over the longer warp
// span), TMA staging or direct global reads of the samples, and resident CTAs
// per SM.  Each candidate runs the spreader over the items of the first
// templates (at most kTuneSpectra spectra; all of a smaller search), timed
// with CUDA events, and is scored by spectra per second; the choice is kept
// per shape (segment length, band, fine grid, kernel width, templates,
// spectra).  Large searches skip the small chunks and the smallest CTA caps.
constexpr long long kTuneSpectra = 150000;

// One-segment items queued last by the tuned search: about two per resident
// CTA of the largest configuration, so that the last wave is fine-grained.
int32_t tail_singles(const srs_ctx* ctx) { return 2 * 8 * ctx->n_sm; }

srs_status upload_items(srs_ctx* ctx, Plan& pl) {
  if (!pl.order.empty()) {
    SRS_CK(ctx->order.ensure(pl.order.size() * 4), "alloc order");
    SRS_CK(cudaMemcpyAsync(ctx->order.p, pl.order.data(), pl.order.size() * 4, cudaMemcpyHostToDevice, ctx->stream),
           "copy order");
  }
  SRS_CK(ctx->items.ensure(pl.items.size() * sizeof(Item)), "alloc items");
  SRS_CK(ctx->item_off.ensure(pl.item_off.size() * 4), "alloc item_off");
  SRS_CK(ctx->partial.ensure(pl.items.size() * (size_t)pl.n_bins * 4), "alloc partial");
  SRS_CK(cudaMemcpyAsync(ctx->items.p, pl.items.data(), pl.items.size() * sizeof(Item), cudaMemcpyHostToDevice, ctx->stream), "copy items");
  SRS_CK(cudaMemcpyAsync(ctx->item_off.p, pl.item_off.data(), pl.item_off.size() * 4, cudaMemcpyHostToDevice, ctx->stream), "copy item_off");
  return SRS_OK;
}

srs_status autotune_mixed(srs_ctx* ctx, Plan& pl, const float* s32, int use_tma, int* ctas_out) {
  std::vector<unsigned char> key;
  auto put = [&](const void* d, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(d);
    key.insert(key.end(), c, c + n);
  };
  put(&pl.n_s, sizeof pl.n_s);
  put(&pl.n_bins, sizeof pl.n_bins);
  put(&pl.n_fine, sizeof pl.n_fine);
  put(&pl.w, sizeof pl.w);
  put(&pl.n_templates, sizeof pl.n_templates);
  put(&pl.n_spectra, sizeof pl.n_spectra);
  key.push_back((unsigned char)use_tma);
  key.push_back((unsigned char)pl.allow_128);
  key.push_back((unsigned char)pl.lanes128);
  // SRS_MIXED_LAYOUT=<threads>:<tma|global>[:<chunk>:<ctas>] restricts the
  // search to one layout (used to check every layout against the same
  // reference, and to profile one fixed configuration).
  int only_threads = 0, only_gx = -1, only_chunk = 0, only_ctas = -1;
  if (const char* lay = std::getenv("SRS_MIXED_LAYOUT")) {
    const std::string l(lay);
    key.insert(key.end(), l.begin(), l.end());
    if (l.rfind("128", 0) == 0) only_threads = 128;
    if (l.rfind("256", 0) == 0) only_threads = 256;
    if (l.find(":global") != std::string::npos) only_gx = 1;
    if (l.find(":tma") != std::string::npos) only_gx = 0;
    int t = 0, c = 0, k = -1;
    char st[16] = {0};
    if (std::sscanf(lay, "%d:%15[a-z]:%d:%d", &t, st, &c, &k) == 4 && c >= 1 && c <= 16 && k >= 0) {
      only_chunk = c;
      only_ctas = k;
    }
  }
  for (const auto& t : ctx->tuned)
    if (t.key == key) {
      set_cta(pl, t.threads);
      pl.global_x = t.global_x != 0;
      if (!pl.tuned_items || t.chunk != pl.chunk) {
        make_items(pl, t.chunk, false, 0, 0, tail_singles(ctx));
        { srs_status us = upload_items(ctx, pl); if (us != SRS_OK) return us; }
        pl.tuned_items = true;
      }
      *ctas_out = t.ctas;
      return SRS_OK;
    }
  // templates [0, n_tune) carry at least kTuneSpectra spectra (or all of them)
  int32_t n_tune = 0;
  long long tune_spectra = 0;
  while (n_tune < pl.n_templates && tune_spectra < kTuneSpectra) tune_spectra += pl.nseg[n_tune++];
  const bool large = pl.n_spectra > kTuneSpectra;
  struct Choice { int chunk, ctas, threads, global_x; };
  Choice best_c{pl.chunk, 0, kSpreadThreads, 0};
  double best = 1e30;  // ms per spectrum
  for (int threads : {256, 128}) {
    if (threads == 128 && !pl.allow_128) continue;
    if (only_threads && threads != only_threads) continue;
    set_cta(pl, threads);
    for (int gx : {0, 1}) {
      if (gx == 0 && !use_tma) continue;
      if (only_gx >= 0 && gx != only_gx) continue;
      for (int ch : {1, 2, 4, 8, 16}) {
        if (large && ch < 4 && only_chunk == 0) continue;
        if (only_chunk && ch != only_chunk) continue;
        make_items(pl, ch, false, 0, 0);   // no tail while timing a prefix of the items
        srs_status us = upload_items(ctx, pl);
        if (us != SRS_OK) return us;
        MixedArgs a = mixed_args(pl, ctx, 0, 0);
        a.use_tma = gx ? 0 : 1;
        const int n_items = pl.item_off[n_tune];
        const int cands_256[] = {0, 3, 2}, cands_128[] = {0, 7, 6, 5, 4};
        const int* ctl = threads == 256 ? cands_256 : cands_128;
        const int n_ct = large ? (threads == 256 ? 2 : 3) : (threads == 256 ? 3 : 5);
        for (int ci = 0; ci < (only_ctas >= 0 ? 1 : n_ct); ++ci) {
          const int ct = only_ctas >= 0 ? only_ctas : ctl[ci];
          float best_ms = 1e30f;
          for (int rep = 0; rep < 3; ++rep) {
            SRS_CK(cudaMemsetAsync(ctx->queue.p, 0, kQueueBytes, ctx->stream), "memset queue");
            SRS_CK(cudaEventRecord(ctx->ev2, ctx->stream), "event");
            SRS_CK(launch_mixed(false, pl.w, s32, ctx->items.as<Item>(), n_items, ctx->betas.as<double>(),
                                ctx->queue.as<int>(), a, ctx->partial.as<float>(), nullptr, search_errflag(ctx),
                                ctx->n_sm, ct, ctx->stream), "k_mixed (tuning)");
            SRS_CK(cudaEventRecord(ctx->ev3, ctx->stream), "event");
            SRS_CK(cudaEventSynchronize(ctx->ev3), "tuning");
            const float ms = elapsed_ms(ctx->ev2, ctx->ev3);
            best_ms = std::min(best_ms, ms);
            if (ms > 20.f) break;  // long launches: one timing is enough
          }
          const double per = best_ms / (double)tune_spectra;
          if (per < best) { best = per; best_c = {ch, ct, threads, gx}; }
        }
      }
    }
  }
  set_cta(pl, best_c.threads);
  pl.global_x = best_c.global_x != 0;
  make_items(pl, best_c.chunk, false, 0, 0, tail_singles(ctx));
  pl.tuned_items = true;
  { srs_status us = upload_items(ctx, pl); if (us != SRS_OK) return us; }
  SRS_CK(cudaStreamSynchronize(ctx->stream), "tuning");
  ctx->tuned.push_back({key, best_c.chunk, best_c.ctas, best_c.threads, best_c.global_x, best});
  *ctas_out = best_c.ctas;
  return SRS_OK;
}

srs_status check_err_flag(srs_ctx* ctx) {
  int flag[5] = {0, 0, 0, 0, 0};
  SRS_CK(cudaMemcpy(flag, ctx->errflag.p, sizeof flag, cudaMemcpyDeviceToHost), "read error flag");
  if (flag[0]) {
    char buf[240];
    err_flag_message(flag, buf, sizeof buf);
    return set_err(ctx, SRS_ERR_TIMEOUT, buf);
  }
  return SRS_OK;
}

}  // namespace

srs_status srs::search_impl(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                            int32_t n_templates, const srs_params* params, float* stat_map, srs_candidate* cands,
                            int32_t* n_cands, srs_report* report, bool async_mode) {
  srs_status s = check_common(ctx, strain, dtype, params);
  if (s != SRS_OK) return s;
  if (!cands || !n_cands) return set_err(ctx, SRS_ERR_ARG, "cands and n_cands are required");

  // events of this call: the context's own, or the next asynchronous slot
  int slot = -1;
  cudaEvent_t e0 = ctx->ev0, e1 = ctx->ev1, e2 = ctx->ev2, e3 = ctx->ev3;
  if (async_mode) {
    if (ctx->async_n == srs_ctx::kAsyncSlots) {
      // every slot is in use: settle them (a failure is kept for the next srs_sync)
      const srs_status ss = sync_impl(ctx, nullptr);
      if (ss != SRS_OK && ctx->async_status == SRS_OK) {
        ctx->async_status = ss;
        ctx->async_err = ctx->err;
      }
    }
    slot = ctx->async_n;
    for (int q = 0; q < 4; ++q)
      if (!ctx->aev[slot][q]) SRS_CK(cudaEventCreate(&ctx->aev[slot][q]), "event");
    e0 = ctx->aev[slot][0];
    e1 = ctx->aev[slot][1];
    e2 = ctx->aev[slot][2];
    e3 = ctx->aev[slot][3];
  }
  const Plan* plp = nullptr;
  s = get_plan(ctx, 1, params, mc, n_templates, n_samples, dtype, false, 0, 0, &plp);
  if (s != SRS_OK) return s;
  Plan& pl = ctx->plan;
  const bool mixed = pl.precision == SRS_MIXED;
  const bool f64 = dtype == SRS_F64;
  const int on_dev = params->io_on_device;
  int32_t max_seg = *std::max_element(pl.nseg.begin(), pl.nseg.end());
  const void* dstrain = nullptr;
  if (async_mode && !on_dev) {
    // Host strain, asynchronous: upload into one of two staging buffers on the
    // copy stream (after the search that last used that buffer has copied it
    // out), then copy it on the search stream into the context's strain
    // buffer, the one a captured graph reads.
    const size_t bytes = (size_t)max_seg * pl.n_s * (f64 ? 8 : 4);
    if (!ctx->copy_stream) SRS_CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int b = 0; b < 2; ++b) {
      if (!ctx->stage_ready[b]) SRS_CK(cudaEventCreateWithFlags(&ctx->stage_ready[b], cudaEventDisableTiming), "event");
      if (!ctx->stage_free[b]) SRS_CK(cudaEventCreateWithFlags(&ctx->stage_free[b], cudaEventDisableTiming), "event");
    }
    const int b = slot & 1;
    DevBuf& stage = b ? ctx->strain_stage1 : ctx->strain_stage0;
    if (stage.cap < bytes) {
      // a new buffer: nothing may still read the old one
      SRS_CK(cudaStreamSynchronize(ctx->stream), "staging");
      SRS_CK(stage.ensure(bytes), "alloc staging");
    }
    SRS_CK(ctx->strain.ensure(bytes), "alloc strain");
    SRS_CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->stage_free[b], 0), "staging");
    SRS_CK(cudaMemcpyAsync(stage.p, strain, bytes, cudaMemcpyHostToDevice, ctx->copy_stream), "copy strain");
    SRS_CK(cudaEventRecord(ctx->stage_ready[b], ctx->copy_stream), "event");
    SRS_CK(cudaStreamWaitEvent(ctx->stream, ctx->stage_ready[b], 0), "staging");
    SRS_CK(cudaMemcpyAsync(ctx->strain.p, stage.p, bytes, cudaMemcpyDeviceToDevice, ctx->stream), "stage strain");
    SRS_CK(cudaEventRecord(ctx->stage_free[b], ctx->stream), "event");
    dstrain = ctx->strain.p;
  } else {
    s = stage_strain(ctx, strain, (int64_t)max_seg * pl.n_s, dtype, on_dev, &dstrain);
    if (s != SRS_OK) return s;
  }

  const long long n_map = (long long)n_templates * pl.n_bins;
  const int k = (int)std::min<long long>(pl.top_k, n_map);
  float* dmap = nullptr;
  if (stat_map) {
    if (on_dev) {
      dmap = stat_map;
    } else {
      SRS_CK(ctx->map.ensure(n_map * 4), "alloc map");
      dmap = ctx->map.as<float>();
    }
  }
  SRS_CK(ctx->keys.ensure(n_map * 8), "alloc keys");
  // k <= 32 (mixed form): the reduction selects the top k itself
  const bool top32 = mixed && k <= 32;
  const long long scratch = std::max(topk_scratch_keys(n_map, k), (long long)kTop32BlocksPerSm * ctx->n_sm * 32);
  SRS_CK(ctx->topk_a.ensure(scratch * 8), "alloc topk");
  SRS_CK(ctx->topk_b.ensure(scratch * 8), "alloc topk");
  srs_candidate* dc = on_dev ? cands : nullptr;
  if (!on_dev) {
    SRS_CK(ctx->cands.ensure((size_t)k * sizeof(srs_candidate)), "alloc cands");
    dc = ctx->cands.as<srs_candidate>();
  }
  int launches = 0;
  long long n_items = (long long)pl.items.size();
  if (mixed) {
    SRS_CK(ctx->partial.ensure(n_items * pl.n_bins * 4), "alloc partial");
    SRS_CK(ctx->queue.ensure(kQueueBytes), "alloc queue");
  } else {
    SRS_CK(ctx->S.ensure(n_map * 8), "alloc S");
  }

  // FP32 strain buffer before any capture (the conversion itself is part of the sequence)
  const float* s32 = nullptr;
  int use_tma = 0;
  if (mixed) {
    const bool tma_len = (pl.n_s % 4) == 0 && !tma_disabled();
    if (f64) {
      SRS_CK(ctx->strain32.ensure((size_t)max_seg * pl.n_s * 4), "alloc strain32");
      s32 = ctx->strain32.as<float>();
      use_tma = tma_len ? 1 : 0;
    } else {
      s32 = static_cast<const float*>(dstrain);
      use_tma = (tma_len && ((uintptr_t)dstrain % 16) == 0) ? 1 : 0;
    }
  }
  if (mixed && params->chunk == 0) {
    // the tuner needs the FP32 strain and the tables on the device
    if (f64) SRS_CK(launch_to_f32(static_cast<const double*>(dstrain), ctx->strain32.as<float>(),
                                  (int64_t)max_seg * pl.n_s, ctx->n_sm, ctx->stream), "k_to_f32 (before tuning)");
    int ct = 0;
    s = autotune_mixed(ctx, pl, s32, use_tma, &ct);
    if (s != SRS_OK) return s;
    ctx->ctas_per_sm = ct;
    n_items = (long long)pl.items.size();
    SRS_CK(ctx->partial.ensure(n_items * pl.n_bins * 4), "alloc partial");
    if (pl.global_x) use_tma = 0;
  } else {
    ctx->ctas_per_sm = 0;
    if (mixed && ctx->subset_layout && pl.allow_128) {
      // a refinement's template subset: 128 threads and global sample loads,
      // the tuner's choice for whole banks of the paper's search shape
      if (pl.threads != 128 || !pl.global_x) {
        set_cta(pl, 128);
        pl.global_x = true;
        make_items(pl, pl.chunk, false, 0, 0, tail_singles(ctx));
        s = upload_items(ctx, pl);
        if (s != SRS_OK) return s;
        n_items = (long long)pl.items.size();
        SRS_CK(ctx->partial.ensure(n_items * pl.n_bins * 4), "alloc partial");
      }
      use_tma = 0;
    } else if (mixed && (pl.threads != kSpreadThreads || pl.global_x)) {
      // an explicit chunk runs the default layout: 256 threads, TMA staging
      // where possible (items rebuilt: their anchor rows follow the layout)
      set_cta(pl, kSpreadThreads);
      pl.global_x = false;
      make_items(pl, pl.chunk, false, 0, 0, 0);
      s = upload_items(ctx, pl);
      if (s != SRS_OK) return s;
      n_items = (long long)pl.items.size();
      SRS_CK(ctx->partial.ensure(n_items * pl.n_bins * 4), "alloc partial");
    }
  }
  // The device part of a search: one stream-ordered sequence, replayed from a
  // CUDA graph when the plan and the buffers are the same as last time.
  // events around the transform kernel inside the sequence (a captured graph
  // holds the context's own pair and is re-pointed per launch)
  cudaEvent_t k_ev2 = e2, k_ev3 = e3;
  bool capturing = false;
  auto enqueue = [&]() -> srs_status {
    launches = 0;
    if (mixed) {
      MixedArgs a = mixed_args(pl, ctx, 0, 0);
      a.use_tma = use_tma;
      if (f64) {
        SRS_CK(launch_to_f32(static_cast<const double*>(dstrain), ctx->strain32.as<float>(), (int64_t)max_seg * pl.n_s,
                             ctx->n_sm, ctx->stream), "k_to_f32");
        ++launches;
      }
      // one memset clears the work queue, the top-k ticket and the error flag
      SRS_CK(cudaMemsetAsync(ctx->queue.p, 0, kQueueBytes, ctx->stream), "memset queue");
      SRS_CK(record_kernel_event(k_ev2, ctx->stream, capturing), "event");
      SRS_CK(launch_mixed(false, pl.w, s32, ctx->items.as<Item>(), (int)n_items, ctx->betas.as<double>(),
                          ctx->queue.as<int>(), a, ctx->partial.as<float>(), nullptr, search_errflag(ctx),
                          ctx->n_sm, ctx->ctas_per_sm, ctx->stream), "k_mixed");
      SRS_CK(record_kernel_event(k_ev3, ctx->stream, capturing), "event");
      ++launches;
      if (top32) {
        SRS_CK(launch_reduce_mixed_top32(ctx->partial.as<float>(), ctx->item_off.as<int>(), ctx->nseg.as<int>(),
                                         n_templates, pl.n_bins, dmap, k, ctx->topk_a.as<unsigned long long>(),
                                         ctx->queue.as<int>() + 4, dc, ctx->n_sm, ctx->stream),
               "k_reduce_mixed_top32");
        ++launches;
        return SRS_OK;
      }
      SRS_CK(launch_reduce_mixed(ctx->partial.as<float>(), ctx->item_off.as<int>(), ctx->nseg.as<int>(), n_templates,
                                 pl.n_bins, dmap, ctx->keys.as<unsigned long long>(), ctx->n_sm, ctx->stream),
             "k_reduce_mixed");
      ++launches;
    } else {
      PlainArgs p = plain_args(pl, ctx, 0, 0);
      SRS_CK(cudaMemsetAsync(ctx->S.p, 0, n_map * 8, ctx->stream), "memset S");
      SRS_CK(record_kernel_event(k_ev2, ctx->stream, capturing), "event");
      SRS_CK(launch_plain(f64, false, dstrain, ctx->betas.as<double>(), ctx->nseg.as<int>(), p, max_seg, n_templates,
                          ctx->S.as<double>(), nullptr, ctx->stream), "k_plain");
      SRS_CK(record_kernel_event(k_ev3, ctx->stream, capturing), "event");
      ++launches;
      SRS_CK(launch_finish_plain(ctx->S.as<double>(), ctx->nseg.as<int>(), n_templates, pl.n_bins, dmap,
                                 ctx->keys.as<unsigned long long>(), ctx->n_sm, ctx->stream), "k_finish_plain");
      ++launches;
    }
    const unsigned long long* top = nullptr;
    SRS_CK(launch_topk(ctx->keys.as<unsigned long long>(), n_map, k, ctx->topk_a.as<unsigned long long>(),
                       ctx->topk_b.as<unsigned long long>(), &top, &launches, ctx->stream), "k_topk_tile");
    SRS_CK(launch_keys_to_cands(top, k, pl.n_bins, dc, ctx->stream), "k_keys_to_cands");
    ++launches;
    return SRS_OK;
  };
  std::vector<unsigned char> gkey = ctx->plan_key;
  for (const void* ptr : {dstrain, (const void*)s32, (const void*)dmap, (const void*)dc, (const void*)ctx->partial.p,
                          (const void*)ctx->keys.p, (const void*)ctx->strain32.p, (const void*)ctx->items.p,
                          (const void*)ctx->betas.p, (const void*)ctx->nseg.p, (const void*)ctx->item_off.p,
                          (const void*)ctx->corr.p, (const void*)ctx->tw.p, (const void*)ctx->queue.p,
                          (const void*)ctx->topk_a.p, (const void*)ctx->topk_b.p,
                          (const void*)(pl.order.empty() ? nullptr : ctx->order.p),
                          (const void*)ctx->S.p})
    gkey.insert(gkey.end(), (const unsigned char*)&ptr, (const unsigned char*)&ptr + sizeof ptr);
  gkey.push_back((unsigned char)ctx->ctas_per_sm);
  gkey.push_back((unsigned char)(pl.threads >> 4));
  gkey.push_back((unsigned char)use_tma);
  SRS_CK(cudaEventRecord(e0, ctx->stream), "event");
  bool ran = false;
  if (ctx->use_graphs) {
    if (!(ctx->graph_exec && gkey == ctx->graph_key)) {
      destroy_graph(ctx);
      cudaGraph_t g = nullptr;
      k_ev2 = ctx->ev2;
      k_ev3 = ctx->ev3;
      const cudaError_t be = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
      if (be == cudaSuccess) {
        capturing = true;
        const srs_status es = enqueue();
        capturing = false;
        const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
        cudaError_t ie = cudaErrorUnknown;
        if (es == SRS_OK && ce == cudaSuccess && g) ie = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
        if (ie == cudaSuccess) {
          ctx->graph_key = gkey;
          ctx->graph_launches = launches;
          ctx->graph = g;
          g = nullptr;
          find_event_nodes(ctx);
        } else {
          std::fprintf(stderr, "srs: graph capture not used (enqueue %d: %s; end %s; instantiate %s)\n", (int)es,
                       ctx->err.c_str(), cudaGetErrorString(ce), cudaGetErrorString(ie));
          ctx->graph_exec = nullptr;
        }
        if (g) cudaGraphDestroy(g);
      } else {
        std::fprintf(stderr, "srs: begin capture failed: %s\n", cudaGetErrorString(be));
      }
      cudaGetLastError();
      k_ev2 = e2;
      k_ev3 = e3;
    }
    if (ctx->graph_exec) {
      if (ctx->graph_ev_node[0] && ctx->graph_ev_node[1]) {
        SRS_CK(cudaGraphExecEventRecordNodeSetEvent(ctx->graph_exec, ctx->graph_ev_node[0], e2), "graph event");
        SRS_CK(cudaGraphExecEventRecordNodeSetEvent(ctx->graph_exec, ctx->graph_ev_node[1], e3), "graph event");
      } else if (async_mode) {
        // no re-pointable timing nodes: time this call's transform kernel without the graph
        destroy_graph(ctx);
      }
    }
    if (ctx->graph_exec) {
      SRS_CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream), "graph launch");
      launches = ctx->graph_launches;
      ran = true;
    }
  }
  if (!ran) {
    s = enqueue();
    if (s != SRS_OK) return s;
  }
  SRS_CK(cudaEventRecord(e1, ctx->stream), "event");
  // the device error flag, to this call's pinned slot (read at return, or at srs_sync)
  if (mixed)
    SRS_CK(cudaMemcpyAsync(ctx->hflag + (async_mode ? 8 * (1 + slot) : 0), search_errflag(ctx), 5 * sizeof(int),
                           cudaMemcpyDeviceToHost, ctx->stream), "read error flag");
  if (async_mode) {
    if (!on_dev) {
      // host results: written when the stream reaches them (pinned buffers overlap)
      SRS_CK(cudaMemcpyAsync(cands, dc, (size_t)k * sizeof(srs_candidate), cudaMemcpyDeviceToHost, ctx->stream),
             "copy cands");
      if (stat_map)
        SRS_CK(cudaMemcpyAsync(stat_map, dmap, n_map * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy map");
    }
    ctx->async_n = slot + 1;
    srs_report& r = ctx->async_rep;
    std::memset(&r, 0, sizeof r);
    r.n_spectra = pl.n_spectra;
    r.w = pl.w;
    r.n_fine = pl.n_fine;
    r.sigma = pl.sigma;
    r.beta_es = pl.beta_es;
    r.chunk = mixed ? pl.chunk : 1;
    r.n_items = mixed ? (int32_t)n_items : (int32_t)pl.n_spectra;
    r.kernel_launches = launches;
    r.cta_threads = mixed ? pl.threads : 256;
    r.staging = (mixed && use_tma) ? 1 : 0;
    r.ctas_per_sm = mixed ? ctx->ctas_per_sm : 0;
    *n_cands = k;
    return SRS_OK;
  }
  if (!on_dev) {
    SRS_CK(cudaMemcpyAsync(cands, dc, (size_t)k * sizeof(srs_candidate), cudaMemcpyDeviceToHost, ctx->stream), "copy cands");
    if (stat_map) SRS_CK(cudaMemcpyAsync(stat_map, dmap, n_map * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy map");
  }
  SRS_CK(cudaStreamSynchronize(ctx->stream), "search");
  if (mixed && ctx->hflag[0]) {
    char b[240];
    err_flag_message(ctx->hflag, b, sizeof b);
    return set_err(ctx, SRS_ERR_TIMEOUT, b);
  }
  *n_cands = k;
  if (report) {
    const float ms = elapsed_ms(e0, e1);
    report->device_ms = ms;
    report->n_spectra = pl.n_spectra;
    report->spectra_per_s = ms > 0 ? pl.n_spectra / (ms * 1e-3) : 0.0;
    report->w = pl.w;
    report->n_fine = pl.n_fine;
    report->sigma = pl.sigma;
    report->beta_es = pl.beta_es;
    report->chunk = mixed ? pl.chunk : 1;
    report->cta_threads = mixed ? pl.threads : 256;
    report->staging = (mixed && use_tma) ? 1 : 0;
    report->ctas_per_sm = mixed ? ctx->ctas_per_sm : 0;
    report->n_items = mixed ? (int32_t)n_items : (int32_t)pl.n_spectra;
    report->kernel_launches = launches;
    report->spread_ms = elapsed_ms(e2, e3);
  }
  return SRS_OK;
}

srs_status srs::sync_impl(srs_ctx* ctx, srs_report* report) {
  SRS_CK(cudaStreamSynchronize(ctx->stream), "sync");
  srs_status st = ctx->async_status;
  std::string msg = ctx->async_err;
  double dev = 0.0, spr = 0.0;
  const int n = ctx->async_n;
  for (int k = 0; k < n; ++k) {
    int* f = ctx->hflag + 8 * (1 + k);
    if (f[0] && st == SRS_OK) {
      char d[240], b[280];
      err_flag_message(f, d, sizeof d);
      std::snprintf(b, sizeof b, "asynchronous search %d: %s", k, d);
      st = SRS_ERR_TIMEOUT;
      msg = b;
    }
    f[0] = 0;
    dev += elapsed_ms(ctx->aev[k][0], ctx->aev[k][1]);
    spr += elapsed_ms(ctx->aev[k][2], ctx->aev[k][3]);
  }
  if (report) {
    *report = ctx->async_rep;
    if (n > 0) {
      report->device_ms = dev / n;
      report->spread_ms = spr / n;
      report->spectra_per_s = report->device_ms > 0 ? report->n_spectra / (report->device_ms * 1e-3) : 0.0;
    }
  }
  ctx->async_n = 0;
  ctx->async_status = SRS_OK;
  ctx->async_err.clear();
  if (st != SRS_OK) return set_err(ctx, st, msg);
  return SRS_OK;
}

namespace {

// cuFFT, loaded when the comparison path first runs (the rest of the library
// does not depend on it).
struct CufftApi {
  bool tried = false, ok = false;
  decltype(&cufftPlanMany) plan_many = nullptr;
  decltype(&cufftSetStream) set_stream = nullptr;
  decltype(&cufftExecC2C) exec_c2c = nullptr;
  decltype(&cufftDestroy) destroy = nullptr;
};
CufftApi& cufft_api() {
  static CufftApi api;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!api.tried) {
    api.tried = true;
    std::vector<std::string> names = {"libcufft.so.12", "libcufft.so"};
    if (const char* home = std::getenv("CUDA_HOME")) names.push_back(std::string(home) + "/lib64/libcufft.so.12");
    names.push_back("/usr/local/cuda/lib64/libcufft.so.12");
    void* h = nullptr;
    for (const std::string& n : names)
      if (!h) h = dlopen(n.c_str(), RTLD_NOW | RTLD_LOCAL);
    if (h) {
      api.plan_many = reinterpret_cast<decltype(&cufftPlanMany)>(dlsym(h, "cufftPlanMany"));
      api.set_stream = reinterpret_cast<decltype(&cufftSetStream)>(dlsym(h, "cufftSetStream"));
      api.exec_c2c = reinterpret_cast<decltype(&cufftExecC2C)>(dlsym(h, "cufftExecC2C"));
      api.destroy = reinterpret_cast<decltype(&cufftDestroy)>(dlsym(h, "cufftDestroy"));
      api.ok = api.plan_many && api.set_stream && api.exec_c2c && api.destroy;
    }
  }
  return api;
}

srs_status spectra_impl(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                        int32_t n_templates, int32_t seg_begin, int32_t seg_end, const srs_params* params,
                        double* F, srs_report* report, bool via_cufft = false) {
  srs_status s = check_common(ctx, strain, dtype, params);
  if (s != SRS_OK) return s;
  if (!F) return set_err(ctx, SRS_ERR_ARG, "F is NULL");
  const Plan* plp = nullptr;
  s = get_plan(ctx, 2, params, mc, n_templates, n_samples, dtype, true, seg_begin, seg_end, &plp);
  if (s != SRS_OK) return s;
  const Plan& pl = *plp;
  const bool mixed = pl.precision == SRS_MIXED;
  if (via_cufft && !mixed) return set_err(ctx, SRS_ERR_ARG, "the cuFFT comparison runs the mixed form only");
  if (via_cufft && !cufft_api().ok) return set_err(ctx, SRS_ERR_UNSUPPORTED, "libcufft could not be loaded");
  const bool f64 = dtype == SRS_F64;
  const int on_dev = params->io_on_device;
  const void* dstrain = nullptr;
  s = stage_strain(ctx, strain, (int64_t)seg_end * pl.n_s, dtype, on_dev, &dstrain);
  if (s != SRS_OK) return s;
  const int range = seg_end - seg_begin;
  const size_t fbytes = (size_t)n_templates * range * pl.n_bins * 16;
  double2* dF = reinterpret_cast<double2*>(F);
  if (!on_dev) {
    SRS_CK(ctx->F.ensure(fbytes), "alloc F");
    dF = ctx->F.as<double2>();
  }
  int launches = 0, staged = 0;
  SRS_CK(cudaEventRecord(ctx->ev0, ctx->stream), "event");
  if (mixed) {
    const long long n_items = (long long)pl.items.size();
    SRS_CK(ctx->queue.ensure(64), "alloc queue");
    SRS_CK(ctx->errflag.ensure(64), "alloc error flag");
    MixedArgs a = mixed_args(pl, ctx, seg_begin, range);
    const float* s32 = nullptr;
    s = strain_f32(ctx, dstrain, dtype, (int64_t)seg_end * pl.n_s, pl.n_s, &s32, &a.use_tma);
    if (s != SRS_OK) return s;
    staged = a.use_tma;
    if (f64) ++launches;
    const long long n_spec = (long long)n_templates * range;
    if (via_cufft) {
      SRS_CK(ctx->grid.ensure((size_t)n_spec * pl.n_fine * sizeof(float2)), "alloc grid");
      a.grid_out = ctx->grid.as<float2>();
    }
    SRS_CK(cudaMemsetAsync(ctx->queue.p, 0, 64, ctx->stream), "memset queue");
    SRS_CK(cudaMemsetAsync(ctx->errflag.p, 0, 64, ctx->stream), "memset error flag");
    SRS_CK(launch_mixed(true, pl.w, s32, ctx->items.as<Item>(), (int)n_items, ctx->betas.as<double>(),
                        ctx->queue.as<int>(), a, nullptr, dF, ctx->errflag.as<int>(), ctx->n_sm, 0, ctx->stream),
           "k_mixed");
    launches += 1;
    if (via_cufft) {
      // unfused comparison: batched single-precision C2C transforms of the
      // spread grids in HBM, then deconvolution and band selection
      CufftApi& api = cufft_api();
      SRS_CK(cudaEventRecord(ctx->ev2, ctx->stream), "event");
      if (!ctx->fft_plan_ok || ctx->fft_n != pl.n_fine || ctx->fft_batch != n_spec) {
        if (ctx->fft_plan_ok) api.destroy(ctx->fft_plan);
        ctx->fft_plan_ok = false;
        int n = pl.n_fine;
        cufftHandle h;
        if (api.plan_many(&h, 1, &n, nullptr, 1, n, nullptr, 1, n, CUFFT_C2C, (int)n_spec) != CUFFT_SUCCESS)
          return set_err(ctx, SRS_ERR_CUDA, "cufftPlanMany failed");
        ctx->fft_plan = h;
        ctx->fft_plan_ok = true;
        ctx->fft_n = pl.n_fine;
        ctx->fft_batch = n_spec;
      }
      if (api.set_stream(ctx->fft_plan, ctx->stream) != CUFFT_SUCCESS ||
          api.exec_c2c(ctx->fft_plan, reinterpret_cast<cufftComplex*>(ctx->grid.p),
                       reinterpret_cast<cufftComplex*>(ctx->grid.p), CUFFT_FORWARD) != CUFFT_SUCCESS)
        return set_err(ctx, SRS_ERR_CUDA, "cufftExecC2C failed");
      SRS_CK(cudaEventRecord(ctx->ev3, ctx->stream), "event");
      SRS_CK(launch_grid_deconv(ctx->grid.as<float2>(), n_spec, pl.n_fine, pl.n_bins, pl.half_bins,
                                ctx->corr.as<float>(), dF, ctx->n_sm, ctx->stream), "k_grid_deconv");
      launches += 2;
    }
  } else {
    PlainArgs p = plain_args(pl, ctx, seg_begin, range);
    SRS_CK(launch_plain(f64, true, dstrain, ctx->betas.as<double>(), ctx->nseg.as<int>(), p, range, n_templates,
                        nullptr, dF, ctx->stream), "k_plain");
    launches += 1;
  }
  SRS_CK(cudaEventRecord(ctx->ev1, ctx->stream), "event");
  if (!on_dev) SRS_CK(cudaMemcpyAsync(F, dF, fbytes, cudaMemcpyDeviceToHost, ctx->stream), "copy F");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "spectra");
  if (mixed) {
    s = check_err_flag(ctx);
    if (s != SRS_OK) return s;
  }
  if (report) {
    const float ms = elapsed_ms(ctx->ev0, ctx->ev1);
    std::memset(report, 0, sizeof *report);
    report->device_ms = ms;
    report->n_spectra = pl.n_spectra;
    report->spectra_per_s = ms > 0 ? pl.n_spectra / (ms * 1e-3) : 0.0;
    report->w = pl.w;
    report->n_fine = pl.n_fine;
    report->sigma = pl.sigma;
    report->beta_es = pl.beta_es;
    report->chunk = pl.chunk;
    report->n_items = (int32_t)pl.items.size();
    report->cta_threads = mixed ? pl.threads : 256;
    report->staging = staged;
    report->kernel_launches = launches;
    if (via_cufft) {
      report->spread_ms = elapsed_ms(ctx->ev0, ctx->ev2);
      report->fft_ms = elapsed_ms(ctx->ev2, ctx->ev3);
    }
  }
  return SRS_OK;
}

srs_status time_map_impl(srs_ctx* ctx, const double* mc, int32_t n_templates, const int32_t* item_m,
                         const int32_t* item_i, int32_t n_items, const srs_params* params, int64_t n_samples,
                         double* psi_out, double* theta_out) {
  if (!ctx) return SRS_ERR_ARG;
  if (!params || !item_m || !item_i || !psi_out || !theta_out || n_items <= 0)
    return set_err(ctx, SRS_ERR_ARG, "time_map: NULL argument or no items");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "cudaSetDevice");
  int32_t max_i = 0;
  for (int32_t k = 0; k < n_items; ++k) {
    if (item_m[k] < 0 || item_m[k] >= n_templates || item_i[k] < 0) return set_err(ctx, SRS_ERR_ARG, "time_map: item out of range");
    max_i = std::max(max_i, item_i[k]);
  }
  Plan pl;
  std::string msg;
  srs_status s = make_plan(*params, mc, n_templates, n_samples, true, 0, 1, pl, msg);
  if (s != SRS_OK) return set_err(ctx, s, msg);
  if (max_i >= pl.n_seg_total) return set_err(ctx, SRS_ERR_ARG, "time_map: segment beyond the strain");
  for (int32_t k = 0; k < n_items; ++k) {
    // Sec. II: every sample of the segment must precede coalescence
    double t_last = ((double)(item_i[k] + 1) * (double)pl.n_s - 1.0) / pl.fs;
    if (!(1.0 - 8.0 / 3.0 * pl.beta[item_m[k]] * t_last > 0.0))
      return set_err(ctx, SRS_ERR_DOMAIN, "time_map: a segment reaches coalescence (1 - 8/3 beta t <= 0)");
  }
  ctx->have_plan = false;
  s = upload_tables(ctx, pl);
  if (s != SRS_OK) return s;
  const size_t out_bytes = (size_t)n_items * pl.n_s * 8;
  SRS_CK(ctx->psi.ensure(out_bytes), "alloc psi");
  SRS_CK(ctx->th.ensure(out_bytes), "alloc th");
  if (pl.precision == SRS_MIXED) {
    std::vector<Item> its(n_items);
    for (int32_t k = 0; k < n_items; ++k) its[k] = Item{item_m[k], item_i[k], item_i[k] + 1, k};
    SRS_CK(ctx->items.ensure(its.size() * sizeof(Item)), "alloc items");
    SRS_CK(cudaMemcpyAsync(ctx->items.p, its.data(), its.size() * sizeof(Item), cudaMemcpyHostToDevice, ctx->stream), "copy items");
    SRS_CK(ctx->anchors.ensure((size_t)n_items * pl.n_anchor * sizeof(Anchor)), "alloc anchors");
    SRS_CK(launch_anchors(ctx->items.as<Item>(), n_items, ctx->betas.as<double>(), anchor_args(pl),
                          ctx->anchors.as<Anchor>(), (long long)n_items * pl.n_anchor, ctx->n_sm, ctx->stream), "k_anchors");
    MixedArgs a = mixed_args(pl, ctx, 0, 0);
    SRS_CK(launch_time_map_mixed(ctx->anchors.as<Anchor>(), n_items, a, ctx->psi.as<double>(), ctx->th.as<double>(),
                                 ctx->stream), "k_time_map_mixed");
  } else {
    SRS_CK(ctx->im.ensure((size_t)n_items * 4), "alloc im");
    SRS_CK(ctx->ii.ensure((size_t)n_items * 4), "alloc ii");
    SRS_CK(cudaMemcpyAsync(ctx->im.p, item_m, (size_t)n_items * 4, cudaMemcpyHostToDevice, ctx->stream), "copy im");
    SRS_CK(cudaMemcpyAsync(ctx->ii.p, item_i, (size_t)n_items * 4, cudaMemcpyHostToDevice, ctx->stream), "copy ii");
    PlainArgs p = plain_args(pl, ctx, 0, 0);
    SRS_CK(launch_time_map_plain(ctx->im.as<int>(), ctx->ii.as<int>(), n_items, ctx->betas.as<double>(), p,
                                 ctx->psi.as<double>(), ctx->th.as<double>(), ctx->stream), "k_time_map_plain");
  }
  SRS_CK(cudaMemcpyAsync(psi_out, ctx->psi.p, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy psi");
  SRS_CK(cudaMemcpyAsync(theta_out, ctx->th.p, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy th");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "time_map");
  return SRS_OK;
}

}  // namespace

namespace srs {

std::vector<double> bank_betas(const srs_bank& bank) {
  std::vector<double> b((size_t)bank.n_beta);
  const double step = bank.n_beta > 1 ? (bank.beta_max - bank.beta_min) / (bank.n_beta - 1) : 0.0;
  for (int32_t k = 0; k < bank.n_beta; ++k) b[(size_t)k] = bank.beta_min + k * step;
  return b;
}

srs_status check_bank(srs_ctx* ctx, const srs_bank* bank) {
  if (!bank) return set_err(ctx, SRS_ERR_ARG, "bank is NULL");
  if (bank->n_beta < 1 || bank->n_beta > 65536) return set_err(ctx, SRS_ERR_ARG, "bank size must be in [1, 65536]");
  if (!(bank->beta_min > 0) || !std::isfinite(bank->beta_max) || !(bank->beta_max >= bank->beta_min))
    return set_err(ctx, SRS_ERR_ARG, "bank needs 0 < beta_min <= beta_max");
  if (bank->n_beta > 1 && !(bank->beta_max > bank->beta_min))
    return set_err(ctx, SRS_ERR_ARG, "a bank of several entries needs beta_max > beta_min");
  return SRS_OK;
}

srs_status clear_err_flag(srs_ctx* ctx) {
  SRS_CK(ctx->errflag.ensure(64), "alloc error flag");
  SRS_CK(cudaMemsetAsync(ctx->errflag.p, 0, 64, ctx->stream), "memset error flag");
  return SRS_OK;
}

srs_status read_err_flag(srs_ctx* ctx) { return check_err_flag(ctx); }

}  // namespace srs

namespace {

// Power-cube work items: [seg_begin, seg_end) of every bank entry in chunks,
// queued segment-major (all bank entries of one segment chunk, then the next)
// so that the bank's CTAs share each chunk's samples in L2 and fill the
// cube's segment-innermost rows in order.
srs_status cube_items(srs_ctx* ctx, Plan& pl, int32_t chunk, int32_t seg_begin, int32_t seg_end) {
  make_items(pl, chunk, true, seg_begin, seg_end);
  pl.order.clear();
  int32_t most = 0;
  for (int32_t m = 0; m < pl.n_templates; ++m) most = std::max(most, pl.item_off[m + 1] - pl.item_off[m]);
  for (int32_t c = 0; c < most; ++c)
    for (int32_t m = 0; m < pl.n_templates; ++m)
      if (pl.item_off[m] + c < pl.item_off[m + 1]) pl.order.push_back(pl.item_off[m] + c);
  SRS_CK(ctx->items.ensure(pl.items.size() * sizeof(Item)), "alloc items");
  SRS_CK(ctx->order.ensure(pl.order.size() * 4), "alloc order");
  SRS_CK(cudaMemcpyAsync(ctx->items.p, pl.items.data(), pl.items.size() * sizeof(Item), cudaMemcpyHostToDevice,
                         ctx->stream), "copy items");
  SRS_CK(cudaMemcpyAsync(ctx->order.p, pl.order.data(), pl.order.size() * 4, cudaMemcpyHostToDevice, ctx->stream),
         "copy order");
  // the host vectors may change on the next plan: finish the copies now
  SRS_CK(cudaStreamSynchronize(ctx->stream), "copy items");
  return SRS_OK;
}

// Layout tuner of the power cube, like the search's (CTA size, staging,
// segments per item, resident CTAs per SM), timed on the first queue
// positions (at most kTuneSpectra / 2 spectra) and kept per shape.
srs_status tune_cube(srs_ctx* ctx, Plan& pl, const float* x, int use_tma, float* dcube, int32_t seg_begin,
                     int32_t seg_end) {
  std::vector<unsigned char> key = {'c', 'u', 'b', 'e'};
  auto put = [&](const void* d, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(d);
    key.insert(key.end(), c, c + n);
  };
  const int32_t range = seg_end - seg_begin;
  put(&pl.n_s, sizeof pl.n_s);
  put(&pl.n_bins, sizeof pl.n_bins);
  put(&pl.n_fine, sizeof pl.n_fine);
  put(&pl.w, sizeof pl.w);
  put(&pl.n_templates, sizeof pl.n_templates);
  put(&range, sizeof range);
  key.push_back((unsigned char)use_tma);
  key.push_back((unsigned char)pl.allow_128);
  key.push_back((unsigned char)pl.lanes128);
  const char* lay = std::getenv("SRS_MIXED_LAYOUT");
  int only_threads = 0, only_gx = -1;
  if (lay) {
    const std::string l(lay);
    key.insert(key.end(), l.begin(), l.end());
    if (l.rfind("128", 0) == 0) only_threads = 128;
    if (l.rfind("256", 0) == 0) only_threads = 256;
    if (l.find(":global") != std::string::npos) only_gx = 1;
    if (l.find(":tma") != std::string::npos) only_gx = 0;
  }
  for (const auto& t : ctx->tuned)
    if (t.key == key) {
      set_cta(pl, t.threads);
      pl.global_x = t.global_x != 0;
      pl.ctas = t.ctas;
      srs_status s = cube_items(ctx, pl, t.chunk, seg_begin, seg_end);
      if (s == SRS_OK) pl.tuned_items = true;
      return s;
    }
  const long long total = (long long)pl.n_templates * range;
  const long long tune_cap = kTuneSpectra / 2;
  struct Choice { int chunk, ctas, threads, global_x; };
  Choice best_c{4, 0, kSpreadThreads, use_tma ? 0 : 1};
  double best = 1e30;
  for (int threads : {256, 128}) {
    if (threads == 128 && !pl.allow_128) continue;
    if (only_threads && threads != only_threads) continue;
    set_cta(pl, threads);
    for (int gx : {0, 1}) {
      if (gx == 0 && !use_tma) continue;
      if (only_gx >= 0 && gx != only_gx) continue;
      for (int ch : {2, 4, 8, 16}) {
        if (ch > range && ch != 2) continue;
        srs_status s = cube_items(ctx, pl, ch, seg_begin, seg_end);
        if (s != SRS_OK) return s;
        // the first queue positions, up to tune_cap spectra
        int n_pos = 0;
        long long spectra = 0;
        while (n_pos < (int)pl.order.size() && spectra < tune_cap) {
          const Item& it = pl.items[(size_t)pl.order[(size_t)n_pos++]];
          spectra += it.i1 - it.i0;
        }
        MixedArgs a = mixed_args(pl, ctx, seg_begin, range);
        a.use_tma = gx ? 0 : 1;
        a.cube_out = dcube;
        const int c256[] = {0, 3}, c128[] = {0, 7, 6};
        const int* ctl = threads == 256 ? c256 : c128;
        const int n_ct = threads == 256 ? 2 : 3;
        for (int ci = 0; ci < n_ct; ++ci) {
          float best_ms = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {
            SRS_CK(cudaMemsetAsync(ctx->queue.p, 0, 64, ctx->stream), "memset queue");
            SRS_CK(cudaEventRecord(ctx->ev2, ctx->stream), "event");
            SRS_CK(launch_mixed(true, pl.w, x, ctx->items.as<Item>(), n_pos, ctx->betas.as<double>(),
                                ctx->queue.as<int>(), a, nullptr, nullptr, ctx->errflag.as<int>(), ctx->n_sm,
                                ctl[ci], ctx->stream), "k_mixed (cube tuning)");
            SRS_CK(cudaEventRecord(ctx->ev3, ctx->stream), "event");
            SRS_CK(cudaEventSynchronize(ctx->ev3), "tuning");
            best_ms = std::min(best_ms, elapsed_ms(ctx->ev2, ctx->ev3));
          }
          const double per = best_ms / (double)std::max<long long>(1, std::min(spectra, total));
          if (per < best) { best = per; best_c = {ch, ctl[ci], threads, gx}; }
        }
      }
    }
  }
  set_cta(pl, best_c.threads);
  pl.global_x = best_c.global_x != 0;
  pl.ctas = best_c.ctas;
  srs_status s = cube_items(ctx, pl, best_c.chunk, seg_begin, seg_end);
  if (s != SRS_OK) return s;
  pl.tuned_items = true;
  ctx->tuned.push_back({key, best_c.chunk, best_c.ctas, best_c.threads, best_c.global_x, best});
  return SRS_OK;
}

}  // namespace

namespace srs {

srs_status cube_device(srs_ctx* ctx, const float* s32, int64_t n_samples, const std::vector<double>& bank,
                       int32_t seg_begin, int32_t seg_end, const srs_params* params, float* dcube, int* launches,
                       const Plan** plan_out) {
  const Plan* plp = nullptr;
  srs_status s = get_plan(ctx, 3, params, nullptr, (int32_t)bank.size(), n_samples, SRS_F32, true, seg_begin, seg_end,
                          &plp, bank.data(), true);
  if (s != SRS_OK) return s;
  Plan& pl = ctx->plan;
  if (plan_out) *plan_out = plp;
  if (pl.precision != SRS_MIXED) return set_err(ctx, SRS_ERR_UNSUPPORTED, "the power cube runs the mixed form only");
  const float* x = nullptr;
  int use_tma = 0;
  s = strain_f32(ctx, s32, SRS_F32, (int64_t)seg_end * pl.n_s, pl.n_s, &x, &use_tma);
  if (s != SRS_OK) return s;
  SRS_CK(ctx->queue.ensure(64), "alloc queue");
  if (!pl.tuned_items) {
    s = tune_cube(ctx, pl, x, use_tma, dcube, seg_begin, seg_end);
    if (s != SRS_OK) return s;
  }
  MixedArgs a = mixed_args(pl, ctx, seg_begin, seg_end - seg_begin);
  a.use_tma = (use_tma && !pl.global_x) ? 1 : 0;
  a.cube_out = dcube;
  SRS_CK(cudaMemsetAsync(ctx->queue.p, 0, 64, ctx->stream), "memset queue");
  SRS_CK(launch_mixed(true, pl.w, x, ctx->items.as<Item>(), (int)pl.items.size(), ctx->betas.as<double>(),
                      ctx->queue.as<int>(), a, nullptr, nullptr, ctx->errflag.as<int>(), ctx->n_sm, pl.ctas,
                      ctx->stream), "k_mixed (power cube)");
  if (launches) ++*launches;
  return SRS_OK;
}

}  // namespace srs

extern "C" {

srs_status srs_create(srs_ctx** out, int device, void* cuda_stream) {
  if (!out) return SRS_ERR_ARG;
  *out = nullptr;
  srs_ctx* c = new (std::nothrow) srs_ctx();
  if (!c) return SRS_ERR_OOM;
  int n_dev = 0;
  if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
    cudaGetLastError();
    delete c;
    return device < 0 ? SRS_ERR_ARG : SRS_ERR_CUDA;
  }
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return SRS_ERR_CUDA;
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return SRS_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreate(&c->ev2) != cudaSuccess || cudaEventCreate(&c->ev3) != cudaSuccess ||
      cudaMallocHost(&c->hflag, kHostFlagBytes) != cudaSuccess) {
    cudaGetLastError();
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return SRS_ERR_CUDA;
  }
  std::memset(c->hflag, 0, kHostFlagBytes);
  // SRS_NO_GRAPHS=1: launch the search's kernels directly, not from a captured
  // graph (profilers replay a direct launch with all of its launch attributes)
  if (const char* ng = std::getenv("SRS_NO_GRAPHS")) c->use_graphs = !(ng[0] == '1');
  *out = c;
  return SRS_OK;
}

void srs_destroy(srs_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  for (auto& slot : c->aev)
    for (cudaEvent_t& e : slot)
      if (e) cudaEventDestroy(e);
  for (cudaEvent_t& e : c->pev)
    if (e) cudaEventDestroy(e);
  if (c->fft_plan_ok) cufft_api().destroy(c->fft_plan);
  for (cudaEvent_t e : c->slide_ev)
    if (e) cudaEventDestroy(e);
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
  }
  for (int b = 0; b < 2; ++b) {
    if (c->stage_ready[b]) cudaEventDestroy(c->stage_ready[b]);
    if (c->stage_free[b]) cudaEventDestroy(c->stage_free[b]);
  }
  if (c->hflag) cudaFreeHost(c->hflag);
  for (DevBuf* b : c->all_buffers()) b->release();
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev2) cudaEventDestroy(c->ev2);
  if (c->ev3) cudaEventDestroy(c->ev3);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* srs_last_error(const srs_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

srs_status srs_plan(const srs_params* params, const double* mc, int32_t n_templates, int64_t n_samples,
                    srs_plan_info* info, double* beta_out, int32_t* nseg_out) {
  if (!params) return SRS_ERR_ARG;
  try {
    Plan pl;
    std::string msg;
    srs_status s = make_plan(*params, mc, n_templates, n_samples, false, 0, 0, pl, msg);
    if (s != SRS_OK) return s;
    fill_info(pl, info);
    for (int32_t m = 0; m < n_templates; ++m) {
      if (beta_out) beta_out[m] = pl.beta[m];
      if (nseg_out) nseg_out[m] = pl.nseg[m];
    }
    return SRS_OK;
  } catch (...) {
    return SRS_ERR_OOM;
  }
}

srs_status srs_search(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                      int32_t n_templates, const srs_params* params, float* stat_map, srs_candidate* cands,
                      int32_t* n_cands, srs_report* report) {
  try {
    return search_impl(ctx, strain, n_samples, dtype, mc, n_templates, params, stat_map, cands, n_cands, report);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_power_cube(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const srs_bank* bank,
                          int32_t seg_begin, int32_t seg_end, const srs_params* params, float* cube,
                          srs_report* report) {
  try {
    srs_status s = check_common(ctx, strain, dtype, params);
    if (s != SRS_OK) return s;
    s = check_bank(ctx, bank);
    if (s != SRS_OK) return s;
    if (!cube) return set_err(ctx, SRS_ERR_ARG, "cube is NULL");
    if (params->precision != SRS_MIXED) return set_err(ctx, SRS_ERR_UNSUPPORTED, "the power cube runs the mixed form only");
    const int64_t n_s = (int64_t)std::llround(params->t_coh * params->fs);
    if (n_s < 1 || seg_begin < 0 || seg_end <= seg_begin || (int64_t)seg_end * n_s > n_samples)
      return set_err(ctx, SRS_ERR_ARG, "need 0 <= seg_begin < seg_end <= segments in the strain");
    const std::vector<double> bb = bank_betas(*bank);
    const int on_dev = params->io_on_device;
    const void* dstrain = nullptr;
    s = stage_strain(ctx, strain, (int64_t)seg_end * n_s, dtype, on_dev, &dstrain);
    if (s != SRS_OK) return s;
    SRS_CK(cudaEventRecord(ctx->ev0, ctx->stream), "event");
    const float* s32 = nullptr;
    int tma = 0, launches = 0;
    s = strain_f32(ctx, dstrain, dtype, (int64_t)seg_end * n_s, n_s, &s32, &tma);
    if (s != SRS_OK) return s;
    if (dtype == SRS_F64) ++launches;
    s = clear_err_flag(ctx);
    if (s != SRS_OK) return s;
    const int64_t n_bins = std::llround((params->f_hi - params->f_lo) * params->t_coh);
    const size_t bytes = (size_t)bank->n_beta * (size_t)std::max<int64_t>(n_bins, 1) * (size_t)(seg_end - seg_begin) * 4;
    float* dcube = cube;
    if (!on_dev) {
      SRS_CK(ctx->cube.ensure(bytes), "alloc cube");
      dcube = ctx->cube.as<float>();
    }
    SRS_CK(cudaEventRecord(ctx->ev2, ctx->stream), "event");
    const Plan* pl = nullptr;
    s = cube_device(ctx, s32, n_samples, bb, seg_begin, seg_end, params, dcube, &launches, &pl);
    if (s != SRS_OK) return s;
    SRS_CK(cudaEventRecord(ctx->ev1, ctx->stream), "event");
    if (!on_dev) SRS_CK(cudaMemcpyAsync(cube, dcube, bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy cube");
    SRS_CK(cudaStreamSynchronize(ctx->stream), "power cube");
    s = check_err_flag(ctx);
    if (s != SRS_OK) return s;
    if (report) {
      std::memset(report, 0, sizeof *report);
      report->device_ms = elapsed_ms(ctx->ev0, ctx->ev1);
      report->spread_ms = elapsed_ms(ctx->ev2, ctx->ev1);
      report->n_spectra = (int64_t)bank->n_beta * (seg_end - seg_begin);
      report->spectra_per_s = report->device_ms > 0 ? report->n_spectra / (report->device_ms * 1e-3) : 0.0;
      report->w = pl->w;
      report->n_fine = pl->n_fine;
      report->sigma = pl->sigma;
      report->beta_es = pl->beta_es;
      report->chunk = pl->chunk;
      report->n_items = (int32_t)pl->items.size();
      report->cta_threads = pl->threads;
      report->staging = tma;
      report->kernel_launches = launches;
    }
    return SRS_OK;
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_selftest_wait(srs_ctx* ctx) {
  if (!ctx) return SRS_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "cudaSetDevice");
  srs_status s = clear_err_flag(ctx);
  if (s != SRS_OK) return s;
  SRS_CK(launch_wait_selftest(ctx->errflag.as<int>(), ctx->stream), "k_wait_selftest");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "self-test");
  return check_err_flag(ctx);
}

srs_status srs_segment_spectra_cufft(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                                     const double* mc, int32_t n_templates, int32_t seg_begin, int32_t seg_end,
                                     const srs_params* params, double* F, srs_report* report) {
  try {
    return spectra_impl(ctx, strain, n_samples, dtype, mc, n_templates, seg_begin, seg_end, params, F, report, true);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_search_async(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                            int32_t n_templates, const srs_params* params, float* stat_map, srs_candidate* cands,
                            int32_t* n_cands) {
  try {
    return search_impl(ctx, strain, n_samples, dtype, mc, n_templates, params, stat_map, cands, n_cands, nullptr,
                       true);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_sync(srs_ctx* ctx, srs_report* report) {
  if (!ctx) return SRS_ERR_ARG;
  try {
    return sync_impl(ctx, report);
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_segment_spectra(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                               const double* mc, int32_t n_templates, int32_t seg_begin, int32_t seg_end,
                               const srs_params* params, double* F, srs_report* report) {
  try {
    return spectra_impl(ctx, strain, n_samples, dtype, mc, n_templates, seg_begin, seg_end, params, F, report);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_time_map(srs_ctx* ctx, const double* mc, int32_t n_templates, const int32_t* item_m,
                        const int32_t* item_i, int32_t n_items, const srs_params* params, int64_t n_samples,
                        double* psi_out, double* theta_out) {
  try {
    return time_map_impl(ctx, mc, n_templates, item_m, item_i, n_items, params, n_samples, psi_out, theta_out);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

}  // extern "C"
