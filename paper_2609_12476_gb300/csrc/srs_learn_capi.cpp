// srs_learn_capi.cpp -- C ABI of the learned proposal (include/srs.h): training
// data synthesis, the MLP (forward, gradient, Adam training), scoring of a
// coarse map, direct refinement of fine cells, and the proposal search that
// chains them.  Host orchestration only; every step runs in srs_learn.cu /
// srs_kernels.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "srs_ctx.h"
#include "srs_internal.h"
#include "srs_kernels.h"
#include "srs_learn.h"

using namespace srs;

namespace {

constexpr double kTwoPi = 6.28318530717958647692;

// splitmix64 (Steele, Lea & Flood 2014): the minibatch order of training.
uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void shuffle(std::vector<int32_t>& v, uint64_t& state) {
  for (size_t i = v.size(); i > 1; --i) {
    const size_t j = (size_t)(splitmix64(state) % i);
    std::swap(v[i - 1], v[j]);
  }
}

srs_status begin(srs_ctx* ctx) {
  if (!ctx) return SRS_ERR_ARG;
  cudaGetLastError();  // an earlier unchecked call's error is not this call's
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "cudaSetDevice");
  return SRS_OK;
}

// FP32 master parameters on the device and their FP16 copies (W1, w2).
srs_status upload_params(srs_ctx* ctx, const float* params) {
  SRS_CK(ctx->wts.ensure((size_t)kParams * 4), "alloc params");
  SRS_CK(ctx->w1h.ensure((size_t)kHidden * kPatchSize * 2), "alloc W1 fp16");
  SRS_CK(ctx->w2h.ensure((size_t)kHidden * 2), "alloc w2 fp16");
  SRS_CK(cudaMemcpyAsync(ctx->wts.p, params, (size_t)kParams * 4, cudaMemcpyHostToDevice, ctx->stream), "copy params");
  SRS_CK(launch_weights_to_half(ctx->wts.as<float>(), ctx->w1h.as<__half>(), ctx->w2h.as<__half>(), ctx->stream),
         "k_weights_to_half");
  return SRS_OK;
}

const float* b1_ptr(srs_ctx* ctx) { return ctx->wts.as<float>() + kHidden * kPatchSize; }
const float* b2_ptr(srs_ctx* ctx) { return ctx->wts.as<float>() + kParams - 1; }

// Device copy of a host array, or the device pointer itself.
template <typename T>
srs_status to_device(srs_ctx* ctx, DevBuf& buf, const T* src, size_t count, int on_device, const T** out) {
  if (on_device) {
    *out = src;
    return SRS_OK;
  }
  SRS_CK(buf.ensure(count * sizeof(T)), "alloc staging");
  SRS_CK(cudaMemcpyAsync(buf.p, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream), "copy staging");
  *out = buf.as<T>();
  return SRS_OK;
}

srs_status forward(srs_ctx* ctx, const float* X, int32_t n, float* logits, float* Z1) {
  SRS_CK(launch_mlp_forward(X, n, ctx->w1h.as<__half>(), b1_ptr(ctx), ctx->w2h.as<__half>(), b2_ptr(ctx), logits, Z1,
                            ctx->n_sm, ctx->stream), "k_mlp_forward");
  return SRS_OK;
}

// Every cell's logit on the tensor cores: the first layer as an implicit-GEMM
// convolution over the map (k_score_tc), FP16 features and weights, FP32 sums.
srs_status score_map_impl(srs_ctx* ctx, const float* map, int32_t n_templates, int32_t n_bins, float* scores) {
  srs_status s = clear_err_flag(ctx);
  if (s != SRS_OK) return s;
  SRS_CK(launch_score_tc(map, n_templates, n_bins, ctx->w1h.as<__half>(), b1_ptr(ctx), ctx->w2h.as<__half>(),
                         b2_ptr(ctx), scores, ctx->errflag.as<int>(), ctx->n_sm, ctx->stream),
         "k_score_tc");
  int flag[2] = {0, 0};
  SRS_CK(cudaMemcpyAsync(flag, ctx->errflag.p, sizeof flag, cudaMemcpyDeviceToHost, ctx->stream), "read error flag");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "k_score_tc");
  if (flag[0]) {
    char b[128];
    std::snprintf(b, sizeof b, "score_map: a wait for the tensor cores gave up (tile %d)", flag[1]);
    return set_err(ctx, SRS_ERR_TIMEOUT, b);
  }
  return SRS_OK;
}

srs_status refine_impl(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                       int32_t n_templates, const srs_params* params, const int32_t* cell_m, const int32_t* cell_b,
                       int32_t n_cells, float* nsigma, srs_report* report, int64_t* seg_bins_out,
                       int32_t* templates_out, const Plan* planned = nullptr) {
  if (!params || !mc || !nsigma || (n_cells > 0 && (!cell_m || !cell_b)) || n_cells < 0)
    return set_err(ctx, SRS_ERR_ARG, "refine: NULL argument");
  if (dtype != SRS_F32 && dtype != SRS_F64) return set_err(ctx, SRS_ERR_ARG, "dtype must be SRS_F32 or SRS_F64");
  srs_params pc = *params;
  pc.precision = SRS_MIXED;
  if (pc.eps < kMixedMinEps) pc.eps = kMixedMinEps;   // direct sums: eps only sizes a NUFFT not used here
  pc.chunk = kSparseChunk;
  Plan own;
  if (!planned) {
    std::string msg;
    srs_status s0 = make_plan(pc, mc, n_templates, n_samples, false, 0, 0, own, msg);
    if (s0 != SRS_OK) return set_err(ctx, s0, msg);
  }
  const Plan& pl = planned ? *planned : own;
  srs_status s = SRS_OK;
  for (int32_t c = 0; c < n_cells; ++c)
    if (cell_m[c] < 0 || cell_m[c] >= n_templates || cell_b[c] < 0 || cell_b[c] >= pl.n_bins)
      return set_err(ctx, SRS_ERR_ARG, "refine: cell outside the map");
  if (n_cells == 0) return SRS_OK;

  // Templates with many requested bins are cheaper through the NUFFT (all
  // bins of a spectrum at once) than through direct sums (one pass over the
  // samples per bin): take those through the mixed search on that template
  // subset and read the requested cells off its map.
  {
    std::vector<int32_t> per_t(n_templates, 0);
    std::vector<long long> ks(n_cells);
    for (int32_t c = 0; c < n_cells; ++c) ks[c] = (long long)cell_m[c] * pl.n_bins + cell_b[c];
    std::vector<long long> u(ks);
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    for (long long key : u) ++per_t[(int32_t)(key / pl.n_bins)];
    std::vector<int32_t> dense;
    for (int32_t m = 0; m < n_templates; ++m)
      if (per_t[m] > kDirectMaxBins) dense.push_back(m);
    if (!dense.empty()) {
      std::vector<int32_t> slot(n_templates, -1);
      std::vector<double> dmc(dense.size());
      for (size_t k = 0; k < dense.size(); ++k) { slot[dense[k]] = (int32_t)k; dmc[k] = mc[dense[k]]; }
      std::vector<int32_t> rest_m, rest_b, rest_idx;
      for (int32_t c = 0; c < n_cells; ++c)
        if (slot[cell_m[c]] < 0) { rest_m.push_back(cell_m[c]); rest_b.push_back(cell_b[c]); rest_idx.push_back(c); }
      // dense templates: mixed search with a device map
      srs_params ps = pc;
      ps.io_on_device = 1;
      ps.top_k = 1;
      ps.chunk = 4;    // no autotuning of a one-off template subset: the full banks' tuned layout
      const void* dstrain_all = strain;
      if (!params->io_on_device) {
        const size_t bytes = (size_t)n_samples * (dtype == SRS_F64 ? 8 : 4);
        SRS_CK(ctx->F.ensure(bytes), "alloc strain");
        SRS_CK(cudaMemcpyAsync(ctx->F.p, strain, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy strain");
        dstrain_all = ctx->F.p;
      }
      SRS_CK(ctx->S.ensure(dense.size() * (size_t)pl.n_bins * 4), "alloc dense map");
      SRS_CK(ctx->ccands.ensure(sizeof(srs_candidate)), "alloc cands");
      int32_t nc = 0;
      srs_report rs;
      std::memset(&rs, 0, sizeof rs);
      // a one-off template subset: launched directly, not captured as a graph
      const bool graphs = ctx->use_graphs;
      ctx->use_graphs = false;
      ctx->subset_layout = true;
      s = search_impl(ctx, dstrain_all, n_samples, dtype, dmc.data(), (int32_t)dense.size(), &ps,
                      ctx->S.as<float>(), ctx->ccands.as<srs_candidate>(), &nc, &rs);
      ctx->subset_layout = false;
      ctx->use_graphs = graphs;
      if (s != SRS_OK) return s;
      std::vector<float> dmap(dense.size() * (size_t)pl.n_bins);
      SRS_CK(cudaMemcpy(dmap.data(), ctx->S.p, dmap.size() * 4, cudaMemcpyDeviceToHost), "copy dense map");
      int64_t sb_rest = 0;
      int32_t t_rest = 0;
      std::vector<float> ns_rest(rest_idx.size());
      if (!rest_idx.empty()) {
        s = refine_impl(ctx, dstrain_all, n_samples, dtype, mc, n_templates, &ps, rest_m.data(), rest_b.data(),
                        (int32_t)rest_idx.size(), ns_rest.data(), nullptr, &sb_rest, &t_rest, &pl);
        if (s != SRS_OK) return s;
      }
      for (int32_t c = 0; c < n_cells; ++c)
        if (slot[cell_m[c]] >= 0) nsigma[c] = dmap[(size_t)slot[cell_m[c]] * pl.n_bins + cell_b[c]];
      for (size_t k = 0; k < rest_idx.size(); ++k) nsigma[rest_idx[k]] = ns_rest[k];
      int64_t dense_segs = 0;
      for (int32_t m : dense) dense_segs += pl.nseg[m];
      if (seg_bins_out) *seg_bins_out = sb_rest + dense_segs * (int64_t)pl.n_bins;
      if (templates_out) *templates_out = t_rest + (int32_t)dense.size();
      if (report) {
        std::memset(report, 0, sizeof *report);
        report->n_spectra = dense_segs;
        report->device_ms = rs.device_ms;
      }
      return SRS_OK;
    }
  }

  // unique (template, bin) pairs, grouped by template, up to kSparseMaxBins per group
  std::vector<long long> keys(n_cells);
  for (int32_t c = 0; c < n_cells; ++c) keys[c] = (long long)cell_m[c] * pl.n_bins + cell_b[c];
  std::vector<long long> uk(keys);
  std::sort(uk.begin(), uk.end());
  uk.erase(std::unique(uk.begin(), uk.end()), uk.end());
  std::vector<int32_t> bins;
  std::vector<SparseItem> items;
  std::vector<int32_t> key_item0(uk.size()), key_nitems(uk.size()), key_slot(uk.size()), key_nseg(uk.size());
  const int chunk = kSparseChunk;
  int32_t n_templ_touched = 0;
  int64_t seg_bins = 0;
  size_t k = 0;
  while (k < uk.size()) {
    const int32_t m = (int32_t)(uk[k] / pl.n_bins);
    size_t e = k;
    while (e < uk.size() && uk[e] / pl.n_bins == m) ++e;
    ++n_templ_touched;
    for (size_t g0 = k; g0 < e; g0 += kSparseMaxBins) {
      const size_t g1 = std::min(e, g0 + kSparseMaxBins);
      const int b0 = (int)bins.size();
      const int item0 = (int)items.size();
      for (size_t u = g0; u < g1; ++u) bins.push_back((int32_t)(uk[u] % pl.n_bins));
      for (int32_t i = 0; i < pl.nseg[m]; i += chunk) {
        SparseItem it;
        std::memset(&it, 0, sizeof it);
        it.m = m;
        it.i0 = i;
        it.i1 = std::min(pl.nseg[m], i + chunk);
        it.b0 = b0;
        it.nb = (int)(g1 - g0);
        items.push_back(it);
      }
      for (size_t u = g0; u < g1; ++u) {
        key_item0[u] = item0;
        key_nitems[u] = (int)items.size() - item0;
        key_slot[u] = (int)(u - g0);
        key_nseg[u] = pl.nseg[m];
      }
      seg_bins += (int64_t)pl.nseg[m] * (int64_t)(g1 - g0);
    }
    k = e;
  }
  std::vector<int32_t> c_item0(n_cells), c_nitems(n_cells), c_slot(n_cells), c_nseg(n_cells);
  for (int32_t c = 0; c < n_cells; ++c) {
    const size_t u = (size_t)(std::lower_bound(uk.begin(), uk.end(), keys[c]) - uk.begin());
    c_item0[c] = key_item0[u];
    c_nitems[c] = key_nitems[u];
    c_slot[c] = key_slot[u];
    c_nseg[c] = key_nseg[u];
  }

  // device staging
  int32_t max_seg = *std::max_element(pl.nseg.begin(), pl.nseg.end());
  const int64_t samples = (int64_t)max_seg * pl.n_s;
  const void* dstrain = strain;
  if (!params->io_on_device) {
    SRS_CK(ctx->strain.ensure((size_t)samples * (dtype == SRS_F64 ? 8 : 4)), "alloc strain");
    SRS_CK(cudaMemcpyAsync(ctx->strain.p, strain, (size_t)samples * (dtype == SRS_F64 ? 8 : 4),
                           cudaMemcpyHostToDevice, ctx->stream), "copy strain");
    dstrain = ctx->strain.p;
  }
  const float* s32 = nullptr;
  int use_tma = 0;
  s = strain_f32(ctx, dstrain, dtype, samples, pl.n_s, &s32, &use_tma);
  if (s != SRS_OK) return s;
  SRS_CK(ctx->sp_betas.ensure(pl.beta.size() * 8), "alloc betas");
  SRS_CK(ctx->sp_items.ensure(items.size() * sizeof(SparseItem)), "alloc items");
  SRS_CK(ctx->sp_bins.ensure(bins.size() * 4), "alloc bins");
  SRS_CK(ctx->sp_partial.ensure(items.size() * kSparseMaxBins * 4), "alloc partial");
  SRS_CK(ctx->sp_cells.ensure((size_t)n_cells * 16), "alloc cells");
  SRS_CK(ctx->sp_out.ensure((size_t)n_cells * 4), "alloc out");
  SRS_CK(cudaMemcpyAsync(ctx->sp_betas.p, pl.beta.data(), pl.beta.size() * 8, cudaMemcpyHostToDevice, ctx->stream),
         "copy betas");
  SRS_CK(cudaMemcpyAsync(ctx->sp_items.p, items.data(), items.size() * sizeof(SparseItem), cudaMemcpyHostToDevice,
                         ctx->stream), "copy items");
  SRS_CK(cudaMemcpyAsync(ctx->sp_bins.p, bins.data(), bins.size() * 4, cudaMemcpyHostToDevice, ctx->stream), "copy bins");
  int32_t* dc = ctx->sp_cells.as<int32_t>();
  SRS_CK(cudaMemcpyAsync(dc, c_item0.data(), (size_t)n_cells * 4, cudaMemcpyHostToDevice, ctx->stream), "copy cells");
  SRS_CK(cudaMemcpyAsync(dc + n_cells, c_nitems.data(), (size_t)n_cells * 4, cudaMemcpyHostToDevice, ctx->stream), "copy cells");
  SRS_CK(cudaMemcpyAsync(dc + 2 * (size_t)n_cells, c_slot.data(), (size_t)n_cells * 4, cudaMemcpyHostToDevice, ctx->stream), "copy cells");
  SRS_CK(cudaMemcpyAsync(dc + 3 * (size_t)n_cells, c_nseg.data(), (size_t)n_cells * 4, cudaMemcpyHostToDevice, ctx->stream), "copy cells");
  SparseArgs a;
  std::memset(&a, 0, sizeof a);
  a.n_s = (int)pl.n_s;
  a.span = pl.span;
  a.run = pl.run;
  a.half_bins = pl.half_bins;
  a.kc_int = (pl.k_c >= 1.0 && pl.k_c < 1073741824.0 && pl.k_c == std::floor(pl.k_c)) ? (int)pl.k_c : 0;
  a.kc = (float)pl.k_c;
  a.inv_ns = (float)(1.0 / (double)pl.n_s);
  a.aa.fs = pl.fs;
  a.aa.t_coh = pl.t_coh;
  a.aa.f_c = pl.f_c;
  a.aa.n_s = pl.n_s;
  a.aa.span = pl.span;
  a.aa.n_anchor = pl.n_anchor;
  a.aa.local = 0;
  SRS_CK(cudaEventRecord(ctx->ev0, ctx->stream), "event");
  SRS_CK(launch_sparse_bins(s32, ctx->sp_items.as<SparseItem>(), (int)items.size(), ctx->sp_betas.as<double>(),
                            ctx->sp_bins.as<int>(), a, ctx->sp_partial.as<float>(), ctx->n_sm, ctx->stream),
         "k_sparse_bins");
  SRS_CK(launch_sparse_reduce(ctx->sp_partial.as<float>(), dc, dc + n_cells, dc + 2 * (size_t)n_cells,
                              dc + 3 * (size_t)n_cells, n_cells, ctx->sp_out.as<float>(), ctx->stream),
         "k_sparse_reduce");
  SRS_CK(cudaEventRecord(ctx->ev1, ctx->stream), "event");
  SRS_CK(cudaMemcpyAsync(nsigma, ctx->sp_out.p, (size_t)n_cells * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy n_sigma");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "refine");
  if (report) {
    const float ms = elapsed_ms(ctx->ev0, ctx->ev1);
    std::memset(report, 0, sizeof *report);
    report->device_ms = ms;
    report->spread_ms = ms;
    report->n_spectra = seg_bins;
    report->n_items = (int32_t)items.size();
    report->kernel_launches = 2 + (dtype == SRS_F64 ? 1 : 0);
  }
  if (seg_bins_out) *seg_bins_out = seg_bins;
  if (templates_out) *templates_out = n_templ_touched;
  return SRS_OK;
}

}  // namespace

extern "C" {

srs_status srs_make_strain(srs_ctx* ctx, float* out, int64_t n, double fs, uint64_t seed, int32_t noise,
                           const srs_injection* inj, int32_t n_inj, double f_hi) {
  try {
    srs_status s = begin(ctx);
    if (s != SRS_OK) return s;
    if (!out || n <= 0 || !(fs > 0) || n_inj < 0 || n_inj > 1024 || (n_inj > 0 && !inj))
      return set_err(ctx, SRS_ERR_ARG, "make_strain: bad argument (n > 0, fs > 0, 0 <= n_inj <= 1024)");
    std::vector<InjectionDev> dev(n_inj);
    for (int32_t k = 0; k < n_inj; ++k) {
      if (!(inj[k].mc > 0) || !(inj[k].f0 > 0)) return set_err(ctx, SRS_ERR_ARG, "make_strain: mc and f0 must be positive");
      const double b = chirp_beta(inj[k].mc, inj[k].f0);
      InjectionDev d;
      d.beta = b;
      d.f0 = inj[k].f0;
      d.amp = inj[k].amp;
      d.phi0_cyc = inj[k].phi0 / kTwoPi;
      // Sec. II: time for the 0PN track to go from f0 to f_hi (before coalescence)
      d.t_end = f_hi > inj[k].f0 ? 3.0 / (8.0 * b) * (1.0 - std::pow(inj[k].f0 / f_hi, 8.0 / 3.0)) : 0.0;
      dev[k] = d;
    }
    SRS_CK(ctx->inj.ensure(std::max<size_t>(1, dev.size()) * sizeof(InjectionDev)), "alloc injections");
    if (n_inj > 0)
      SRS_CK(cudaMemcpyAsync(ctx->inj.p, dev.data(), dev.size() * sizeof(InjectionDev), cudaMemcpyHostToDevice,
                             ctx->stream), "copy injections");
    SRS_CK(launch_make_strain(out, n, fs, seed, noise ? 1 : 0, ctx->inj.as<InjectionDev>(), n_inj, ctx->n_sm,
                              ctx->stream), "k_make_strain");
    SRS_CK(cudaStreamSynchronize(ctx->stream), "make_strain");
    return SRS_OK;
  } catch (...) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  }
}

srs_status srs_patches(srs_ctx* ctx, const float* map, int32_t n_templates, int32_t n_bins, const int32_t* cell_m,
                       const int32_t* cell_b, int32_t n_cells, float* out, int32_t io_on_device) {
  srs_status s = begin(ctx);
  if (s != SRS_OK) return s;
  if (!map || !cell_m || !cell_b || !out || n_templates <= 0 || n_bins <= 0 || n_cells <= 0)
    return set_err(ctx, SRS_ERR_ARG, "patches: bad argument");
  const float* dmap;
  const int32_t *dm, *db;
  s = to_device(ctx, ctx->cmap, map, (size_t)n_templates * n_bins, io_on_device, &dmap);
  if (s != SRS_OK) return s;
  s = to_device(ctx, ctx->cells_m, cell_m, (size_t)n_cells, io_on_device, &dm);
  if (s != SRS_OK) return s;
  s = to_device(ctx, ctx->cells_b, cell_b, (size_t)n_cells, io_on_device, &db);
  if (s != SRS_OK) return s;
  float* dout = out;
  if (!io_on_device) {
    SRS_CK(ctx->patches.ensure((size_t)n_cells * kPatchSize * 4), "alloc patches");
    dout = ctx->patches.as<float>();
  }
  SRS_CK(launch_patches(dmap, n_templates, n_bins, dm, db, n_cells, dout, ctx->n_sm, ctx->stream), "k_patches");
  if (!io_on_device)
    SRS_CK(cudaMemcpyAsync(out, dout, (size_t)n_cells * kPatchSize * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy patches");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "patches");
  return SRS_OK;
}

srs_status srs_mlp_forward(srs_ctx* ctx, const float* X, int32_t n, const float* params, float* logits,
                           int32_t io_on_device) {
  srs_status s = begin(ctx);
  if (s != SRS_OK) return s;
  if (!X || !params || !logits || n <= 0) return set_err(ctx, SRS_ERR_ARG, "mlp_forward: bad argument");
  s = upload_params(ctx, params);
  if (s != SRS_OK) return s;
  const float* dX;
  s = to_device(ctx, ctx->xb, X, (size_t)n * kPatchSize, io_on_device, &dX);
  if (s != SRS_OK) return s;
  float* dl = logits;
  if (!io_on_device) {
    SRS_CK(ctx->logits.ensure((size_t)n * 4), "alloc logits");
    dl = ctx->logits.as<float>();
  }
  s = forward(ctx, dX, n, dl, nullptr);
  if (s != SRS_OK) return s;
  if (!io_on_device) SRS_CK(cudaMemcpyAsync(logits, dl, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy logits");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "mlp_forward");
  return SRS_OK;
}

srs_status srs_mlp_grad(srs_ctx* ctx, const float* X, const float* y, int32_t n, const float* params, float* grad,
                        float* loss, int32_t io_on_device) {
  srs_status s = begin(ctx);
  if (s != SRS_OK) return s;
  if (!X || !y || !params || !grad || !loss || n <= 0) return set_err(ctx, SRS_ERR_ARG, "mlp_grad: bad argument");
  s = upload_params(ctx, params);
  if (s != SRS_OK) return s;
  const float *dX, *dy;
  s = to_device(ctx, ctx->xb, X, (size_t)n * kPatchSize, io_on_device, &dX);
  if (s != SRS_OK) return s;
  s = to_device(ctx, ctx->yb, y, (size_t)n, io_on_device, &dy);
  if (s != SRS_OK) return s;
  SRS_CK(ctx->z1.ensure((size_t)n * kHidden * 4), "alloc z1");
  SRS_CK(ctx->logits.ensure((size_t)n * 4), "alloc logits");
  SRS_CK(ctx->dz.ensure((size_t)n * 4), "alloc dz");
  SRS_CK(ctx->lossv.ensure((size_t)n * 4), "alloc loss");
  SRS_CK(ctx->grad.ensure((size_t)kParams * 4), "alloc grad");
  s = forward(ctx, dX, n, ctx->logits.as<float>(), ctx->z1.as<float>());
  if (s != SRS_OK) return s;
  SRS_CK(launch_bce(ctx->logits.as<float>(), dy, n, ctx->dz.as<float>(), ctx->lossv.as<float>(), ctx->stream), "k_bce");
  SRS_CK(launch_mlp_grad(dX, n, ctx->z1.as<float>(), ctx->dz.as<float>(), ctx->w2h.as<__half>(), ctx->grad.as<float>(),
                         ctx->stream), "k_mlp_grad");
  std::vector<float> lv(n);
  SRS_CK(cudaMemcpyAsync(grad, ctx->grad.p, (size_t)kParams * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy grad");
  SRS_CK(cudaMemcpyAsync(lv.data(), ctx->lossv.p, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy loss");
  SRS_CK(cudaStreamSynchronize(ctx->stream), "mlp_grad");
  double acc = 0.0;
  for (float v : lv) acc += v;
  *loss = (float)(acc / n);
  return SRS_OK;
}

srs_status srs_mlp_train(srs_ctx* ctx, const float* X, const float* y, int32_t n, const srs_train_cfg* cfg,
                         float* params, float* loss_per_epoch) {
  try {
    srs_status s = begin(ctx);
    if (s != SRS_OK) return s;
    if (!X || !y || !cfg || !params || n <= 0) return set_err(ctx, SRS_ERR_ARG, "mlp_train: bad argument");
    if (cfg->epochs < 1 || cfg->batch < 1 || cfg->batch > 65536 || !(cfg->lr > 0) || !(cfg->beta1 >= 0 && cfg->beta1 < 1) ||
        !(cfg->beta2 >= 0 && cfg->beta2 < 1) || !(cfg->adam_eps > 0))
      return set_err(ctx, SRS_ERR_ARG, "mlp_train: bad configuration");
    s = upload_params(ctx, params);
    if (s != SRS_OK) return s;
    const int B = std::min(cfg->batch, n);
    SRS_CK(ctx->adam_m.ensure((size_t)kParams * 4), "alloc adam");
    SRS_CK(ctx->adam_v.ensure((size_t)kParams * 4), "alloc adam");
    SRS_CK(cudaMemsetAsync(ctx->adam_m.p, 0, (size_t)kParams * 4, ctx->stream), "zero adam");
    SRS_CK(cudaMemsetAsync(ctx->adam_v.p, 0, (size_t)kParams * 4, ctx->stream), "zero adam");
    SRS_CK(ctx->xb.ensure((size_t)B * kPatchSize * 4), "alloc batch");
    SRS_CK(ctx->yb.ensure((size_t)B * 4), "alloc batch");
    SRS_CK(ctx->z1.ensure((size_t)B * kHidden * 4), "alloc z1");
    SRS_CK(ctx->logits.ensure((size_t)B * 4), "alloc logits");
    SRS_CK(ctx->dz.ensure((size_t)B * 4), "alloc dz");
    SRS_CK(ctx->lossv.ensure((size_t)n * 4), "alloc loss");
    SRS_CK(ctx->grad.ensure((size_t)kParams * 4), "alloc grad");
    SRS_CK(ctx->idx.ensure((size_t)n * 4), "alloc order");
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<float> lv(n);
    uint64_t rng = cfg->seed;
    long long t = 0;
    for (int32_t ep = 0; ep < cfg->epochs; ++ep) {
      shuffle(order, rng);
      SRS_CK(cudaMemcpyAsync(ctx->idx.p, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice, ctx->stream), "copy order");
      SRS_CK(cudaStreamSynchronize(ctx->stream), "copy order");   // `order` is reused next epoch
      for (int32_t b0 = 0; b0 < n; b0 += B) {
        const int nb = std::min(B, n - b0);
        SRS_CK(launch_gather_batch(X, y, ctx->idx.as<int>() + b0, nb, ctx->xb.as<float>(), ctx->yb.as<float>(),
                                   ctx->n_sm, ctx->stream), "k_gather_batch");
        s = forward(ctx, ctx->xb.as<float>(), nb, ctx->logits.as<float>(), ctx->z1.as<float>());
        if (s != SRS_OK) return s;
        SRS_CK(launch_bce(ctx->logits.as<float>(), ctx->yb.as<float>(), nb, ctx->dz.as<float>(),
                          ctx->lossv.as<float>() + b0, ctx->stream), "k_bce");
        SRS_CK(launch_mlp_grad(ctx->xb.as<float>(), nb, ctx->z1.as<float>(), ctx->dz.as<float>(), ctx->w2h.as<__half>(),
                               ctx->grad.as<float>(), ctx->stream), "k_mlp_grad");
        ++t;
        AdamArgs a;
        a.lr = cfg->lr;
        a.b1 = cfg->beta1;
        a.b2 = cfg->beta2;
        a.eps = cfg->adam_eps;
        a.c1 = (float)(1.0 / (1.0 - std::pow((double)cfg->beta1, (double)t)));
        a.c2 = (float)(1.0 / (1.0 - std::pow((double)cfg->beta2, (double)t)));
        SRS_CK(launch_adam(ctx->wts.as<float>(), ctx->grad.as<float>(), ctx->adam_m.as<float>(), ctx->adam_v.as<float>(),
                           a, ctx->w1h.as<__half>(), ctx->w2h.as<__half>(), ctx->stream), "k_adam");
      }
      SRS_CK(cudaMemcpyAsync(lv.data(), ctx->lossv.p, (size_t)n * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy loss");
      SRS_CK(cudaStreamSynchronize(ctx->stream), "train epoch");
      if (loss_per_epoch) {
        double acc = 0.0;
        for (float v : lv) acc += v;
        loss_per_epoch[ep] = (float)(acc / n);
      }
    }
    SRS_CK(cudaMemcpyAsync(params, ctx->wts.p, (size_t)kParams * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy params");
    SRS_CK(cudaStreamSynchronize(ctx->stream), "mlp_train");
    return SRS_OK;
  } catch (...) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  }
}

srs_status srs_score_map(srs_ctx* ctx, const float* map, int32_t n_templates, int32_t n_bins, const float* params,
                         float* scores) {
  srs_status s = begin(ctx);
  if (s != SRS_OK) return s;
  if (!map || !params || !scores || n_templates <= 0 || n_bins <= 0) return set_err(ctx, SRS_ERR_ARG, "score_map: bad argument");
  s = upload_params(ctx, params);
  if (s != SRS_OK) return s;
  s = score_map_impl(ctx, map, n_templates, n_bins, scores);
  if (s != SRS_OK) return s;
  SRS_CK(cudaStreamSynchronize(ctx->stream), "score_map");
  return SRS_OK;
}

srs_status srs_refine(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                      int32_t n_templates, const srs_params* params, const int32_t* cell_m, const int32_t* cell_b,
                      int32_t n_cells, float* nsigma, srs_report* report) {
  try {
    srs_status s = begin(ctx);
    if (s != SRS_OK) return s;
    if (!strain) return set_err(ctx, SRS_ERR_ARG, "refine: strain is NULL");
    return refine_impl(ctx, strain, n_samples, dtype, mc, n_templates, params, cell_m, cell_b, n_cells, nsigma, report,
                       nullptr, nullptr);
  } catch (...) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  }
}

srs_status srs_search_proposed(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                               const double* coarse_mc, int32_t n_coarse, const double* fine_mc, int32_t n_fine,
                               const srs_params* params, const float* mlp_params,
                               const srs_proposal_params* prop, int32_t max_cells, int32_t* cell_m,
                               int32_t* cell_b, float* cell_nsigma, int32_t* n_cells_out, srs_candidate* cands,
                               int32_t* n_cands, srs_proposal_report* report) {
  try {
    if (!prop) return set_err(ctx, SRS_ERR_ARG, "search_proposed: prop is NULL");
    const srs_proposal_params params_prop = *prop;
    const float score_threshold = prop->score_threshold;
    srs_status s = begin(ctx);
    if (s != SRS_OK) return s;
    if (!strain || !params || !coarse_mc || !fine_mc || !mlp_params || n_coarse <= 0 || n_fine <= 0 || !n_cells_out ||
        !cands || !n_cands || max_cells < 0 || (max_cells > 0 && (!cell_m || !cell_b || !cell_nsigma)))
      return set_err(ctx, SRS_ERR_ARG, "search_proposed: bad argument");
    if (dtype != SRS_F32 && dtype != SRS_F64) return set_err(ctx, SRS_ERR_ARG, "dtype must be SRS_F32 or SRS_F64");
    const int n_bins = (int)std::llround((params->f_hi - params->f_lo) * params->t_coh);
    if (n_bins <= 0) return set_err(ctx, SRS_ERR_ARG, "search_proposed: empty band");
    for (cudaEvent_t& e : ctx->pev)
      if (!e) SRS_CK(cudaEventCreate(&e), "event");
    SRS_CK(cudaEventRecord(ctx->pev[0], ctx->stream), "event");
    // 1. strain on the device once, then the coarse search with a device map
    const void* dstrain = strain;
    srs_params pc = *params;
    if (!params->io_on_device) {
      const size_t bytes = (size_t)n_samples * (dtype == SRS_F64 ? 8 : 4);
      SRS_CK(ctx->F.ensure(bytes), "alloc strain");
      SRS_CK(cudaMemcpyAsync(ctx->F.p, strain, bytes, cudaMemcpyHostToDevice, ctx->stream), "copy strain");
      dstrain = ctx->F.p;
    }
    pc.io_on_device = 1;
    SRS_CK(ctx->cmap.ensure((size_t)n_coarse * n_bins * 4), "alloc coarse map");
    SRS_CK(ctx->ccands.ensure((size_t)std::max(1, pc.top_k) * sizeof(srs_candidate)), "alloc coarse cands");
    int32_t nc = 0;
    srs_report rep;
    std::memset(&rep, 0, sizeof rep);
    s = search_impl(ctx, dstrain, n_samples, dtype, coarse_mc, n_coarse, &pc, ctx->cmap.as<float>(),
                    ctx->ccands.as<srs_candidate>(), &nc, &rep);
    if (s != SRS_OK) return s;
    // 2. network scores of every coarse cell
    s = upload_params(ctx, mlp_params);
    if (s != SRS_OK) return s;
    const long long ncells = (long long)n_coarse * n_bins;
    SRS_CK(ctx->sp_out.ensure((size_t)ncells * 4), "alloc scores");
    s = score_map_impl(ctx, ctx->cmap.as<float>(), n_coarse, n_bins, ctx->sp_out.as<float>());
    if (s != SRS_OK) return s;
    std::vector<float> scores(ncells), cmap;
    SRS_CK(cudaMemcpyAsync(scores.data(), ctx->sp_out.p, (size_t)ncells * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy scores");
    if (params_prop.component_top > 0 || params_prop.nms_by_nsigma) {
      cmap.resize(ncells);
      SRS_CK(cudaMemcpyAsync(cmap.data(), ctx->cmap.p, (size_t)ncells * 4, cudaMemcpyDeviceToHost, ctx->stream),
             "copy coarse map");
    }
    SRS_CK(cudaStreamSynchronize(ctx->stream), "score");
    // component rule: of each 8-connected group of above-threshold cells, the
    // component_top cells of highest coarse n_sigma (ties: lower index first)
    std::vector<unsigned char> keep;
    if (params_prop.component_top > 0) {
      keep.assign(ncells, 0);
      std::vector<int32_t> comp_of(ncells, -1), stack, members;
      for (long long c0 = 0; c0 < ncells; ++c0) {
        if (!(scores[c0] > score_threshold) || comp_of[c0] >= 0) continue;
        members.clear();
        stack.assign(1, (int32_t)c0);
        comp_of[c0] = (int32_t)c0;
        while (!stack.empty()) {
          const int32_t c = stack.back();
          stack.pop_back();
          members.push_back(c);
          const int32_t cm = c / n_bins, cb = c % n_bins;
          for (int32_t dm = -1; dm <= 1; ++dm)
            for (int32_t db = -1; db <= 1; ++db) {
              const int32_t m = cm + dm, b = cb + db;
              if (m < 0 || m >= n_coarse || b < 0 || b >= n_bins) continue;
              const int32_t o = m * n_bins + b;
              if (comp_of[o] < 0 && scores[o] > score_threshold) {
                comp_of[o] = (int32_t)c0;
                stack.push_back(o);
              }
            }
        }
        const size_t top = std::min<size_t>(members.size(), (size_t)params_prop.component_top);
        std::partial_sort(members.begin(), members.begin() + top, members.end(), [&](int32_t a, int32_t b) {
          if (cmap[a] != cmap[b]) return cmap[a] > cmap[b];
          return a < b;
        });
        for (size_t u = 0; u < top; ++u) keep[members[u]] = 1;
      }
    }
    // 3. proposed coarse cells -> fine cells (nearest coarse template in log Mc)
    std::vector<int32_t> parent(n_fine);
    {
      std::vector<double> lc(n_coarse);
      bool sorted = true;
      for (int32_t c = 0; c < n_coarse; ++c) {
        lc[c] = std::log(coarse_mc[c]);
        if (c > 0 && !(lc[c] > lc[c - 1])) sorted = false;
      }
      for (int32_t f = 0; f < n_fine; ++f) {
        const double lf = std::log(fine_mc[f]);
        if (sorted) {
          const int32_t hi = (int32_t)(std::lower_bound(lc.begin(), lc.end(), lf) - lc.begin());
          int32_t best = std::min(hi, n_coarse - 1);
          if (hi > 0 && (hi == n_coarse || std::fabs(lf - lc[hi - 1]) <= std::fabs(lf - lc[hi]))) best = hi - 1;
          parent[f] = best;
        } else {
          double bd = 1e300;
          for (int32_t c = 0; c < n_coarse; ++c)
            if (std::fabs(lf - lc[c]) < bd) { bd = std::fabs(lf - lc[c]); parent[f] = c; }
        }
      }
    }
    std::vector<std::vector<int32_t>> children(n_coarse);
    for (int32_t f = 0; f < n_fine; ++f) children[parent[f]].push_back(f);
    std::vector<long long> fk;
    // best score of the coarse cells proposing each fine template (for the budget)
    std::vector<float> tbest(params_prop.template_budget > 0 ? n_fine : 0, -INFINITY);
    int32_t proposed = 0;
    const int32_t rt = std::max(0, params_prop.nms_templates), rb = std::max(0, params_prop.nms_bins);
    const int32_t rows = std::max(0, params_prop.fine_rows);
    for (long long cell = 0; cell < ncells; ++cell) {
      if (!(scores[cell] > score_threshold)) continue;
      if (!keep.empty() && !keep[cell]) continue;
      const int32_t cm = (int32_t)(cell / n_bins), cb = (int32_t)(cell % n_bins);
      if (keep.empty() && (rt > 0 || rb > 0)) {
        // non-maximum suppression: keep a cell only if no cell within
        // (+-rt templates, +-rb bins) has a higher key -- the score, or the
        // coarse n_sigma with nms_by_nsigma (ties: the first in row-major order)
        const std::vector<float>& key = params_prop.nms_by_nsigma ? cmap : scores;
        bool peak = true;
        for (int32_t m = std::max(0, cm - rt); m <= std::min(n_coarse - 1, cm + rt) && peak; ++m)
          for (int32_t b = std::max(0, cb - rb); b <= std::min(n_bins - 1, cb + rb); ++b) {
            const long long o = (long long)m * n_bins + b;
            if (key[o] > key[cell] || (key[o] == key[cell] && o < cell)) { peak = false; break; }
          }
        if (!peak) continue;
      }
      ++proposed;
      for (int32_t c = std::max(0, cm - rows); c <= std::min(n_coarse - 1, cm + rows); ++c)
        for (int32_t f : children[c]) {
          if (!tbest.empty()) tbest[f] = std::max(tbest[f], scores[cell]);
          for (int32_t b = std::max(0, cb - 1); b <= std::min(n_bins - 1, cb + 1); ++b)
            fk.push_back((long long)f * n_bins + b);
        }
    }
    std::sort(fk.begin(), fk.end());
    fk.erase(std::unique(fk.begin(), fk.end()), fk.end());
    if (!tbest.empty()) {
      // template budget: keep the cells of the template_budget fine templates
      // with the highest best proposing score (ties: lower index first)
      std::vector<int32_t> touched;
      for (int32_t f = 0; f < n_fine; ++f)
        if (tbest[f] > -INFINITY) touched.push_back(f);
      if ((int64_t)touched.size() > params_prop.template_budget) {
        std::partial_sort(touched.begin(), touched.begin() + params_prop.template_budget, touched.end(),
                          [&](int32_t a, int32_t b) {
                            if (tbest[a] != tbest[b]) return tbest[a] > tbest[b];
                            return a < b;
                          });
        std::vector<unsigned char> kept(n_fine, 0);
        for (int32_t u = 0; u < params_prop.template_budget; ++u) kept[touched[u]] = 1;
        fk.erase(std::remove_if(fk.begin(), fk.end(), [&](long long v) { return !kept[v / n_bins]; }), fk.end());
      }
    }
    const int32_t nf = (int32_t)fk.size();
    std::vector<int32_t> fm(nf), fb(nf);
    for (int32_t k = 0; k < nf; ++k) { fm[k] = (int32_t)(fk[k] / n_bins); fb[k] = (int32_t)(fk[k] % n_bins); }
    std::vector<float> ns(nf);
    int64_t seg_bins = 0;
    int32_t templ = 0;
    // 4. refinement of the fine cells
    if (nf > 0) {
      s = refine_impl(ctx, dstrain, n_samples, dtype, fine_mc, n_fine, &pc, fm.data(), fb.data(), nf, ns.data(),
                      nullptr, &seg_bins, &templ);
      if (s != SRS_OK) return s;
    }
    SRS_CK(cudaEventRecord(ctx->pev[1], ctx->stream), "event");
    SRS_CK(cudaStreamSynchronize(ctx->stream), "search_proposed");
    for (int32_t k = 0; k < std::min(nf, max_cells); ++k) {
      cell_m[k] = fm[k];
      cell_b[k] = fb[k];
      cell_nsigma[k] = ns[k];
    }
    *n_cells_out = nf;
    // top-k of the evaluated cells: n_sigma desc, template asc, bin asc
    std::vector<int32_t> ord(nf);
    std::iota(ord.begin(), ord.end(), 0);
    const int32_t k = std::min(nf, std::max(0, params->top_k));
    std::partial_sort(ord.begin(), ord.begin() + k, ord.end(), [&](int32_t a, int32_t b) {
      if (ns[a] != ns[b]) return ns[a] > ns[b];
      if (fm[a] != fm[b]) return fm[a] < fm[b];
      return fb[a] < fb[b];
    });
    for (int32_t i = 0; i < k; ++i) {
      cands[i].value = ns[ord[i]];
      cands[i].template_idx = fm[ord[i]];
      cands[i].bin = fb[ord[i]];
    }
    *n_cands = k;
    if (report) {
      const float ms = elapsed_ms(ctx->pev[0], ctx->pev[1]);
      report->device_ms = ms;
      report->coarse_spectra = rep.n_spectra;
      report->proposed_coarse = proposed;
      report->fine_cells = nf;
      report->fine_segment_bins = seg_bins;
      report->fine_templates = templ;
    }
    return SRS_OK;
  } catch (...) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  }
}

}  // extern "C"
