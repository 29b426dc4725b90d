// srs_slide_capi.cpp -- extern "C" entry points of the two-stage search
// (include/srs.h): srs_stack_slide and srs_slide_search.  srs_power_cube,
// stage one alone, sits with the other transform entry points in
// srs_capi.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "srs_ctx.h"
#include "srs_internal.h"
#include "srs_kernels.h"
#include "srs_slide.h"

using namespace srs;

namespace {

srs_status check_slide_params(srs_ctx* ctx, const srs_params* params, int32_t* n_bins) {
  if (!params) return set_err(ctx, SRS_ERR_ARG, "params is NULL");
  if (!(params->t_coh > 0) || !(params->f_hi > params->f_lo)) return set_err(ctx, SRS_ERR_ARG, "need t_coh > 0 and f_hi > f_lo");
  const double nb = (params->f_hi - params->f_lo) * params->t_coh;
  if (std::fabs(nb - std::round(nb)) > 1e-9 * std::max(1.0, nb) || nb < 1 || nb > 1e7)
    return set_err(ctx, SRS_ERR_ARG, "(f_hi - f_lo) * t_coh must be a positive integer");
  if (params->top_k < 1 || params->top_k > 1024) return set_err(ctx, SRS_ERR_ARG, "top_k must be in [1, 1024]");
  if (params->io_on_device != 0 && params->io_on_device != 1) return set_err(ctx, SRS_ERR_ARG, "io_on_device must be 0 or 1");
  *n_bins = (int32_t)std::llround(nb);
  return SRS_OK;
}

srs_status check_grid(srs_ctx* ctx, const srs_slide_grid* g, const srs_params* params) {
  if (!g || !g->mc || !g->c) return set_err(ctx, SRS_ERR_ARG, "grid, grid->mc and grid->c are required");
  if (g->n_rows < 1 || g->n_t0 < 1) return set_err(ctx, SRS_ERR_ARG, "grid needs n_rows >= 1 and n_t0 >= 1");
  if ((long long)g->n_rows * g->n_t0 > 2000000000LL) return set_err(ctx, SRS_ERR_UNSUPPORTED, "stack-slide map too large");
  if (!(g->f0 >= params->f_lo && g->f0 < params->f_hi)) return set_err(ctx, SRS_ERR_ARG, "f0 must lie in [f_lo, f_hi)");
  for (int32_t r = 0; r < g->n_rows; ++r) {
    if (!(g->mc[r] > 0) || !std::isfinite(g->mc[r])) return set_err(ctx, SRS_ERR_ARG, "chirp masses must be positive and finite");
    if (!(g->c[r] >= 0.0 && g->c[r] < 1.0)) return set_err(ctx, SRS_ERR_ARG, "t0 fractions must lie in [0, 1)");
  }
  if (g->weighting != SRS_WEIGHT_EQUAL && g->weighting != SRS_WEIGHT_AMPLITUDE)
    return set_err(ctx, SRS_ERR_ARG, "weighting must be SRS_WEIGHT_EQUAL or SRS_WEIGHT_AMPLITUDE");
  if (g->whiten != 0 && g->whiten != 1) return set_err(ctx, SRS_ERR_ARG, "whiten must be 0 or 1");
  return SRS_OK;
}

srs_status check_cells_and_s_eff(srs_ctx* ctx, const srs_slide_grid* g, const srs_bank* bank, int32_t n_bins) {
  // track cells k n_bins + j are 32-bit on the device
  if ((long long)bank->n_beta * n_bins > 2147483647LL)
    return set_err(ctx, SRS_ERR_UNSUPPORTED, "n_beta * n_bins must stay below 2^31 for the stack-slide's cell table");
  if (!g->s_eff) return SRS_OK;
  const size_t n = (size_t)bank->n_beta * n_bins;
  for (size_t q = 0; q < n; ++q)
    if (!(g->s_eff[q] > 0.0f) || !std::isfinite(g->s_eff[q]))
      return set_err(ctx, SRS_ERR_ARG, "s_eff entries must be positive and finite");
  return SRS_OK;
}

// Tracks of every row (cell and length tables), recomputed only when the
// bank, grid, band or data length change.  *replanned says whether they did.
srs_status plan_tracks(srs_ctx* ctx, const srs_bank* bank, const srs_slide_grid* g, const srs_params* p,
                       int32_t n_bins, int32_t n_total, bool* replanned, const float* s_eff_host) {
  std::vector<unsigned char> key;
  auto put = [&](const void* d, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(d);
    key.insert(key.end(), c, c + n);
  };
  put(&bank->beta_min, sizeof(double));
  put(&bank->beta_max, sizeof(double));
  put(&bank->n_beta, sizeof(int32_t));
  put(&g->f0, sizeof(double));
  put(&g->n_rows, sizeof(int32_t));
  put(&g->n_t0, sizeof(int32_t));
  put(g->mc, sizeof(double) * (size_t)g->n_rows);
  put(g->c, sizeof(double) * (size_t)g->n_rows);
  put(&p->t_coh, sizeof(double));
  put(&p->f_lo, sizeof(double));
  put(&n_bins, sizeof n_bins);
  put(&n_total, sizeof n_total);
  put(&g->weighting, sizeof g->weighting);
  put(&g->whiten, sizeof g->whiten);
  const size_t n_seff = s_eff_host ? (size_t)bank->n_beta * n_bins : 0;
  put(&n_seff, sizeof n_seff);
  if (n_seff) put(s_eff_host, n_seff * sizeof(float));
  *replanned = false;
  if (ctx->have_slide && key == ctx->slide_key) return SRS_OK;
  ctx->have_slide = false;
  *replanned = true;
  if ((long long)g->n_rows * n_total > 2000000000LL) return set_err(ctx, SRS_ERR_UNSUPPORTED, "track table too large");
  std::vector<double> b0((size_t)g->n_rows);
  for (int32_t r = 0; r < g->n_rows; ++r) b0[(size_t)r] = chirp_beta(g->mc[r], g->f0);   // Eq. (beta) at f0
  SRS_CK(ctx->slide_beta0.ensure(b0.size() * 8), "alloc tracks");
  SRS_CK(ctx->slide_frac.ensure(b0.size() * 8), "alloc tracks");
  SRS_CK(ctx->slide_cell.ensure((size_t)g->n_rows * n_total * 4), "alloc tracks");
  SRS_CK(ctx->slide_coef.ensure((size_t)g->n_rows * n_total * 8), "alloc tracks");
  SRS_CK(ctx->slide_w2.ensure((size_t)g->n_rows * (n_total + 1) * 8), "alloc tracks");
  SRS_CK(ctx->slide_len.ensure((size_t)g->n_rows * 4), "alloc tracks");
  if (n_seff) {
    SRS_CK(ctx->slide_seff.ensure(n_seff * 4), "alloc s_eff");
    SRS_CK(cudaMemcpyAsync(ctx->slide_seff.p, s_eff_host, n_seff * 4, cudaMemcpyHostToDevice, ctx->stream), "copy s_eff");
  }
  SRS_CK(cudaMemcpyAsync(ctx->slide_beta0.p, b0.data(), b0.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "copy tracks");
  SRS_CK(cudaMemcpyAsync(ctx->slide_frac.p, g->c, b0.size() * 8, cudaMemcpyHostToDevice, ctx->stream), "copy tracks");
  TrackArgs t;
  t.f0 = g->f0;
  t.f_lo = p->f_lo;
  t.t_coh = p->t_coh;
  t.beta_min = bank->beta_min;
  t.dbeta = bank->n_beta > 1 ? (bank->beta_max - bank->beta_min) / (bank->n_beta - 1) : 0.0;
  t.n_beta = bank->n_beta;
  t.n_bins = n_bins;
  t.n_total = n_total;
  t.weighting = g->weighting;
  t.s_eff = n_seff ? ctx->slide_seff.as<float>() : nullptr;
  t.s_in_weights_only = g->whiten ? 1 : 0;
  SRS_CK(launch_slide_tracks(ctx->slide_beta0.as<double>(), ctx->slide_frac.as<double>(), g->n_rows, t,
                             ctx->slide_cell.as<int>(), ctx->slide_coef.as<float2>(), ctx->slide_len.as<int>(),
                             ctx->slide_w2.as<double>(), ctx->n_sm, ctx->stream),
         "k_slide_tracks");
  ctx->slide_len_host.assign((size_t)g->n_rows, 0);
  SRS_CK(cudaMemcpyAsync(ctx->slide_len_host.data(), ctx->slide_len.p, (size_t)g->n_rows * 4, cudaMemcpyDeviceToHost,
                         ctx->stream), "copy track lengths");
  // the host copies above read caller memory: finish them before returning
  SRS_CK(cudaStreamSynchronize(ctx->stream), "tracks");
  ctx->slide_frac_host.assign(g->c, g->c + g->n_rows);
  ctx->slide_key.swap(key);
  ctx->have_slide = true;
  return SRS_OK;
}

// Cube powers one pass sums: over rows and t0 columns, the track segments
// s < min(len_r, n_total - first) whose segment first + s lies in the chunk.
long long count_reads(const srs_ctx* ctx, int32_t n_t0, int32_t n_total, int32_t seg_begin, int32_t seg_end) {
  long long total = 0;
  for (size_t r = 0; r < ctx->slide_len_host.size(); ++r) {
    const int L = ctx->slide_len_host[r];
    const int e = ctx->slide_frac_host[r] > 0.0 ? 1 : 0;
    for (int32_t n = 0; n < n_t0; ++n) {
      const int first = n + e;
      const int hi = std::min(std::min(L, n_total - first), seg_end - first);
      const int lo = std::max(0, seg_begin - first);
      if (hi > lo) total += hi - lo;
    }
  }
  return total;
}

cudaEvent_t slide_event(srs_ctx* ctx, size_t i) {
  while (ctx->slide_ev.size() <= i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ctx->slide_ev.push_back(e);
  }
  return ctx->slide_ev[i];
}

// Output buffers of a finishing pass (device pointers; host outputs are
// staged in context buffers and copied after the pass).
struct SlideOut {
  float* dmap = nullptr;
  srs_candidate* dc = nullptr;
  int k = 0;
  long long n_map = 0;
};

srs_status prepare_out(srs_ctx* ctx, const srs_slide_grid* g, const srs_params* p, float* nsigma_map,
                       srs_candidate* cands, SlideOut* o) {
  o->n_map = (long long)g->n_rows * g->n_t0;
  o->k = (int)std::min<long long>(p->top_k, o->n_map);
  const int on_dev = p->io_on_device;
  if (nsigma_map) {
    if (on_dev) {
      o->dmap = nsigma_map;
    } else {
      SRS_CK(ctx->slide_map.ensure(o->n_map * 4), "alloc map");
      o->dmap = ctx->slide_map.as<float>();
    }
  }
  SRS_CK(ctx->keys.ensure(o->n_map * 8), "alloc keys");
  const long long scratch = std::max(topk_scratch_keys(o->n_map, o->k), (long long)kTop32BlocksPerSm * ctx->n_sm * 32);
  SRS_CK(ctx->topk_a.ensure(scratch * 8), "alloc topk");
  SRS_CK(ctx->topk_b.ensure(scratch * 8), "alloc topk");
  o->dc = on_dev ? cands : nullptr;
  if (!on_dev) {
    SRS_CK(ctx->cands.ensure((size_t)o->k * sizeof(srs_candidate)), "alloc cands");
    o->dc = ctx->cands.as<srs_candidate>();
  }
  return SRS_OK;
}

// One stack-slide pass over a device cube chunk (with `last`, it also writes
// the map and the top-k keys).
srs_status slide_pass(srs_ctx* ctx, const float* dcube, int32_t seg_begin, int32_t seg_end, int32_t n_total,
                      const srs_slide_grid* g, bool first, bool last, const SlideOut& o, int* launches,
                      bool s_used, long long n_cells) {
  SRS_CK(ctx->slide_Z.ensure((size_t)g->n_rows * g->n_t0 * 4), "alloc running sums");
  SlideArgs a;
  a.n_rows = g->n_rows;
  a.n_t0 = g->n_t0;
  a.n_total = n_total;
  a.seg_begin = seg_begin;
  a.seg_end = seg_end;
  a.ld = seg_end - seg_begin;
  a.first = first ? 1 : 0;
  a.last = last ? 1 : 0;
  a.weighted = (g->weighting != SRS_WEIGHT_EQUAL || s_used) ? 1 : 0;
  // the kernel stages cell * ld + step as 32-bit offsets when they all fit
  a.off32 = n_cells * (long long)a.ld + n_total < 4294967296LL ? 1 : 0;
  SRS_CK(launch_stack_slide(dcube, ctx->slide_cell.as<int>(), ctx->slide_coef.as<float2>(), ctx->slide_len.as<int>(),
                            ctx->slide_w2.as<double>(), ctx->slide_frac.as<double>(), a, ctx->slide_Z.as<float>(),
                            o.dmap, ctx->keys.as<unsigned long long>(), ctx->stream),
         "k_stack_slide");
  ++*launches;
  return SRS_OK;
}

// Top-k of the finished map's keys into the candidates.
srs_status slide_topk(srs_ctx* ctx, const srs_slide_grid* g, const SlideOut& o, int* launches) {
  const unsigned long long* top = nullptr;
  SRS_CK(launch_topk(ctx->keys.as<unsigned long long>(), o.n_map, o.k, ctx->topk_a.as<unsigned long long>(),
                     ctx->topk_b.as<unsigned long long>(), &top, launches, ctx->stream), "k_topk_tile");
  SRS_CK(launch_keys_to_cands(top, o.k, g->n_t0, o.dc, ctx->stream), "k_keys_to_cands");
  ++*launches;
  return SRS_OK;
}

srs_status copy_out(srs_ctx* ctx, const srs_params* p, const SlideOut& o, float* nsigma_map, srs_candidate* cands) {
  if (p->io_on_device) return SRS_OK;
  SRS_CK(cudaMemcpyAsync(cands, o.dc, (size_t)o.k * sizeof(srs_candidate), cudaMemcpyDeviceToHost, ctx->stream),
         "copy cands");
  if (nsigma_map)
    SRS_CK(cudaMemcpyAsync(nsigma_map, o.dmap, o.n_map * 4, cudaMemcpyDeviceToHost, ctx->stream), "copy map");
  return SRS_OK;
}

srs_status stack_slide_impl(srs_ctx* ctx, const float* cube, int32_t seg_begin, int32_t seg_end, int32_t n_total,
                            const srs_bank* bank, const srs_slide_grid* g, const srs_params* p, int32_t flags,
                            float* nsigma_map, srs_candidate* cands, int32_t* n_cands, srs_report* report) {
  if (!ctx) return SRS_ERR_ARG;
  cudaGetLastError();
  int32_t n_bins = 0;
  srs_status s = check_slide_params(ctx, p, &n_bins);
  if (s != SRS_OK) return s;
  if ((s = check_bank(ctx, bank)) != SRS_OK) return s;
  if ((s = check_grid(ctx, g, p)) != SRS_OK) return s;
  if ((s = check_cells_and_s_eff(ctx, g, bank, n_bins)) != SRS_OK) return s;
  if (!cube) return set_err(ctx, SRS_ERR_ARG, "cube is NULL");
  if (flags & ~(SRS_SLIDE_FIRST | SRS_SLIDE_LAST)) return set_err(ctx, SRS_ERR_ARG, "unknown flags");
  const bool first = flags & SRS_SLIDE_FIRST, last = flags & SRS_SLIDE_LAST;
  if (last && (!cands || !n_cands)) return set_err(ctx, SRS_ERR_ARG, "cands and n_cands are required with SRS_SLIDE_LAST");
  if (n_total < 1 || seg_begin < 0 || seg_end <= seg_begin || seg_end > n_total)
    return set_err(ctx, SRS_ERR_ARG, "need 0 <= seg_begin < seg_end <= n_seg_total");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "cudaSetDevice");
  bool replanned = false;
  s = plan_tracks(ctx, bank, g, p, n_bins, n_total, &replanned, g->s_eff);
  if (s != SRS_OK) return s;
  if (!first && (!ctx->slide_open || replanned))
    return set_err(ctx, SRS_ERR_ARG, "a stack-slide chunk without SRS_SLIDE_FIRST must continue an open search of the same templates");
  const size_t cube_bytes = (size_t)bank->n_beta * n_bins * (size_t)(seg_end - seg_begin) * 4;
  const float* dcube = cube;
  if (!p->io_on_device) {
    SRS_CK(ctx->cube.ensure(cube_bytes), "alloc cube");
    SRS_CK(cudaMemcpyAsync(ctx->cube.p, cube, cube_bytes, cudaMemcpyHostToDevice, ctx->stream), "copy cube");
    dcube = ctx->cube.as<float>();
  }
  SlideOut o;
  if (last) {
    s = prepare_out(ctx, g, p, nsigma_map, cands, &o);
    if (s != SRS_OK) return s;
  }
  int launches = 0;
  SRS_CK(cudaEventRecord(ctx->ev0, ctx->stream), "event");
  s = slide_pass(ctx, dcube, seg_begin, seg_end, n_total, g, first, last, o, &launches, g->s_eff != nullptr,
                 (long long)bank->n_beta * n_bins);
  if (s != SRS_OK) return s;
  SRS_CK(cudaEventRecord(ctx->ev2, ctx->stream), "event");
  if (last && (s = slide_topk(ctx, g, o, &launches)) != SRS_OK) return s;
  SRS_CK(cudaEventRecord(ctx->ev1, ctx->stream), "event");
  if (last) {
    s = copy_out(ctx, p, o, nsigma_map, cands);
    if (s != SRS_OK) return s;
  }
  SRS_CK(cudaStreamSynchronize(ctx->stream), "stack-slide");
  ctx->slide_open = !last;
  if (last) *n_cands = o.k;
  if (report) {
    std::memset(report, 0, sizeof *report);
    report->device_ms = elapsed_ms(ctx->ev0, ctx->ev1);
    report->slide_ms = elapsed_ms(ctx->ev0, ctx->ev2);
    report->slide_reads = count_reads(ctx, g->n_t0, n_total, seg_begin, seg_end);
    report->kernel_launches = launches;
  }
  return SRS_OK;
}

srs_status slide_search_impl(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const srs_bank* bank,
                             const srs_slide_grid* g, const srs_params* p, int64_t budget, float* nsigma_map,
                             srs_candidate* cands, int32_t* n_cands, srs_report* report) {
  srs_status s = check_common(ctx, strain, dtype, p);
  if (s != SRS_OK) return s;
  int32_t n_bins = 0;
  if ((s = check_slide_params(ctx, p, &n_bins)) != SRS_OK) return s;
  if ((s = check_bank(ctx, bank)) != SRS_OK) return s;
  if ((s = check_grid(ctx, g, p)) != SRS_OK) return s;
  if ((s = check_cells_and_s_eff(ctx, g, bank, n_bins)) != SRS_OK) return s;
  if (!cands || !n_cands) return set_err(ctx, SRS_ERR_ARG, "cands and n_cands are required");
  if (budget < 0) return set_err(ctx, SRS_ERR_ARG, "cube_budget_bytes must be >= 0");
  if (p->precision != SRS_MIXED) return set_err(ctx, SRS_ERR_UNSUPPORTED, "the power cube runs the mixed form only");
  const double nsd = p->t_coh * p->fs;
  if (!(nsd >= 1) || std::fabs(nsd - std::round(nsd)) > 1e-9 * nsd) return set_err(ctx, SRS_ERR_ARG, "t_coh * fs must be a positive integer");
  const int64_t n_s = std::llround(nsd);
  const int64_t n_total64 = n_samples / n_s;
  if (n_total64 < 1) return set_err(ctx, SRS_ERR_ARG, "strain shorter than one segment");
  if (n_total64 > 10000000) return set_err(ctx, SRS_ERR_UNSUPPORTED, "more than 1e7 segments");
  const int32_t n_total = (int32_t)n_total64;
  const size_t per_seg = (size_t)bank->n_beta * n_bins * 4;
  int32_t chunk = n_total;
  if (budget > 0) chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(n_total, budget / (int64_t)per_seg));
  const int n_chunks = (n_total + chunk - 1) / chunk;
  const std::vector<double> bb = bank_betas(*bank);

  bool replanned = false;
  const bool white = g->whiten != 0;
  // without whitening the tracks are known now; with it, the estimated PSD
  // (amplitude weights) is known after the first chunk
  if (!white || g->s_eff || g->weighting == SRS_WEIGHT_EQUAL) {
    s = plan_tracks(ctx, bank, g, p, n_bins, n_total, &replanned, g->s_eff);
    if (s != SRS_OK) return s;
  }
  SlideOut o;
  s = prepare_out(ctx, g, p, nsigma_map, cands, &o);
  if (s != SRS_OK) return s;
  SRS_CK(ctx->cube.ensure(per_seg * (size_t)chunk), "alloc cube");
  const long long rows = (long long)bank->n_beta * n_bins;
  bool s_used = g->s_eff != nullptr;
  if (white) {
    SRS_CK(ctx->white_s.ensure((size_t)rows * 4), "alloc whitening");
    SRS_CK(ctx->white_sums.ensure((size_t)2 * chunk * 8), "alloc whitening");
    SRS_CK(ctx->white_musig.ensure((size_t)chunk * 8), "alloc whitening");
    if (g->s_eff)
      SRS_CK(cudaMemcpyAsync(ctx->white_s.p, g->s_eff, (size_t)rows * 4, cudaMemcpyHostToDevice, ctx->stream),
             "copy s_eff");
  }
  // every event is created before the first launch
  for (size_t e = 0; e < (size_t)n_chunks * 3; ++e)
    if (!slide_event(ctx, e)) return set_err(ctx, SRS_ERR_CUDA, "cudaEventCreate failed");

  const void* dstrain = nullptr;
  s = stage_strain(ctx, strain, (int64_t)n_total * n_s, dtype, p->io_on_device, &dstrain);
  if (s != SRS_OK) return s;
  SRS_CK(cudaEventRecord(ctx->ev0, ctx->stream), "event");
  int launches = 0, tma = 0;
  const float* s32 = nullptr;
  s = strain_f32(ctx, dstrain, dtype, (int64_t)n_total * n_s, n_s, &s32, &tma);
  if (s != SRS_OK) return s;
  if (dtype == SRS_F64) ++launches;
  if ((s = clear_err_flag(ctx)) != SRS_OK) return s;
  const Plan* pl = nullptr;
  for (int c = 0; c < n_chunks; ++c) {
    const int32_t a = c * chunk, b = std::min(n_total, a + chunk);
    SRS_CK(cudaEventRecord(ctx->slide_ev[3 * c], ctx->stream), "event");
    s = cube_device(ctx, s32, (int64_t)n_total * n_s, bb, a, b, p, ctx->cube.as<float>(), &launches, &pl);
    if (s != SRS_OK) return s;
    if (white) {
      // the PSD from the first chunk (unless given), the moments per chunk
      const bool estimate = !g->s_eff && c == 0;
      SRS_CK(launch_cube_whiten(ctx->cube.as<float>(), rows, b - a, b - a, ctx->white_s.as<float>(), estimate,
                                ctx->white_sums.as<double>(), ctx->white_musig.as<float2>(), nullptr, nullptr,
                                ctx->n_sm, ctx->stream), "k_cube_whiten");
      launches += estimate ? 4 : 3;
      if (c == 0 && !g->s_eff && g->weighting == SRS_WEIGHT_AMPLITUDE) {
        // the estimated PSD enters the amplitude weights: tracks after the first chunk
        std::vector<float> s_host((size_t)rows);
        SRS_CK(cudaMemcpyAsync(s_host.data(), ctx->white_s.p, (size_t)rows * 4, cudaMemcpyDeviceToHost,
                               ctx->stream), "copy PSD estimate");
        SRS_CK(cudaStreamSynchronize(ctx->stream), "PSD estimate");
        s = plan_tracks(ctx, bank, g, p, n_bins, n_total, &replanned, s_host.data());
        if (s != SRS_OK) return s;
        s_used = true;
      }
    }
    SRS_CK(cudaEventRecord(ctx->slide_ev[3 * c + 1], ctx->stream), "event");
    s = slide_pass(ctx, ctx->cube.as<float>(), a, b, n_total, g, c == 0, c == n_chunks - 1, o, &launches, s_used,
                   rows);
    if (s != SRS_OK) return s;
    SRS_CK(cudaEventRecord(ctx->slide_ev[3 * c + 2], ctx->stream), "event");
  }
  s = slide_topk(ctx, g, o, &launches);
  if (s != SRS_OK) return s;
  SRS_CK(cudaEventRecord(ctx->ev1, ctx->stream), "event");
  s = copy_out(ctx, p, o, nsigma_map, cands);
  if (s != SRS_OK) return s;
  SRS_CK(cudaStreamSynchronize(ctx->stream), "slide search");
  ctx->slide_open = false;
  if ((s = read_err_flag(ctx)) != SRS_OK) return s;
  *n_cands = o.k;
  if (report) {
    std::memset(report, 0, sizeof *report);
    report->device_ms = elapsed_ms(ctx->ev0, ctx->ev1);
    for (int c = 0; c < n_chunks; ++c) {
      report->spread_ms += elapsed_ms(ctx->slide_ev[3 * c], ctx->slide_ev[3 * c + 1]);
      report->slide_ms += elapsed_ms(ctx->slide_ev[3 * c + 1], ctx->slide_ev[3 * c + 2]);
    }
    report->n_spectra = (int64_t)bank->n_beta * n_total;
    if (replanned || ctx->slide_reads_total < 0) ctx->slide_reads_total = count_reads(ctx, g->n_t0, n_total, 0, n_total);
    report->slide_reads = ctx->slide_reads_total;
    report->spectra_per_s = report->device_ms > 0 ? report->n_spectra / (report->device_ms * 1e-3) : 0.0;
    report->w = pl->w;
    report->n_fine = pl->n_fine;
    report->sigma = pl->sigma;
    report->beta_es = pl->beta_es;
    report->chunk = chunk;                  // segments per cube chunk
    report->n_items = n_chunks;             // cube chunks
    report->cta_threads = pl->threads;
    report->staging = tma;
    report->kernel_launches = launches;
  }
  return SRS_OK;
}

}  // namespace

extern "C" {

srs_status srs_cube_whiten(srs_ctx* ctx, float* cube, int32_t n_beta, int32_t n_bins, int32_t n_seg, float* s_eff,
                           int32_t estimate, float* mu, float* sigma) {
  if (!ctx) return SRS_ERR_ARG;
  try {
    if (!cube || !s_eff || n_beta < 1 || n_bins < 1 || n_seg < 1 || (estimate != 0 && estimate != 1))
      return set_err(ctx, SRS_ERR_ARG, "need a device cube and s_eff, positive sizes, estimate 0 or 1");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "cudaSetDevice");
    SRS_CK(ctx->white_sums.ensure((size_t)2 * n_seg * 8), "alloc whitening");
    SRS_CK(ctx->white_musig.ensure((size_t)n_seg * 8), "alloc whitening");
    SRS_CK(launch_cube_whiten(cube, (long long)n_beta * n_bins, n_seg, n_seg, s_eff, estimate != 0,
                              ctx->white_sums.as<double>(), ctx->white_musig.as<float2>(), mu, sigma, ctx->n_sm,
                              ctx->stream), "k_cube_whiten");
    SRS_CK(cudaStreamSynchronize(ctx->stream), "whitening");
    return SRS_OK;
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_stack_slide(srs_ctx* ctx, const float* cube, int32_t seg_begin, int32_t seg_end, int32_t n_seg_total,
                           const srs_bank* bank, const srs_slide_grid* grid, const srs_params* params, int32_t flags,
                           float* nsigma_map, srs_candidate* cands, int32_t* n_cands, srs_report* report) {
  try {
    return stack_slide_impl(ctx, cube, seg_begin, seg_end, n_seg_total, bank, grid, params, flags, nsigma_map, cands,
                            n_cands, report);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

srs_status srs_slide_search(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const srs_bank* bank,
                            const srs_slide_grid* grid, const srs_params* params, int64_t cube_budget_bytes,
                            float* nsigma_map, srs_candidate* cands, int32_t* n_cands, srs_report* report) {
  try {
    return slide_search_impl(ctx, strain, n_samples, dtype, bank, grid, params, cube_budget_bytes, nsigma_map, cands,
                             n_cands, report);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, SRS_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(ctx, SRS_ERR_ARG, "unexpected host error");
  }
}

}  // extern "C"
