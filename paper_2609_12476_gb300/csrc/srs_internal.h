// srs_internal.h -- structures shared by the host planner, the C ABI layer and
// the CUDA kernels of libsrs.  Not part of the public ABI (include/srs.h is).
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/srs.h"

namespace srs {

// Threads per CTA of the mixed-precision spreader; each thread owns a run of
// consecutive samples, each warp one FP64 anchor (see Anchor).
constexpr int kSpreadThreads = 256;
constexpr int kSpreadWarps = kSpreadThreads / 32;
// Smallest eps the mixed (FP32) form accepts: its spectra reach about 1.2e-6
// relative L2 error against the exact sum, and the contract is 10 eps.
constexpr double kMixedMinEps = 2e-7;
// Largest kernel width the mixed form is compiled for (eps >= 2e-7 needs <= 8).
constexpr int kMixedMaxW = 8;
// Largest kernel width of the plain FP64 form.
constexpr int kPlainMaxW = 16;

// One work item of the mixed form: segments [i0, i1) of template m; their
// anchors start at row g0 of the anchor table.
struct Item {
  int32_t m, i0, i1, g0;
};

// FP64-derived description of the resampled time over one warp's span of
// samples l = 0 .. span-1 from sample index l_a of a segment (Sec. III.B,
// Eq. new_t expanded around the anchor):
//   delta(l_a + l)/t_coh = psi0 + P1 l + P2 l^2 + P3 l^3 + P4 l^4 + P5 l^5   [periods]
//   f_c * delta(l_a + l)   = th0 + M1 l + k_c (P2 l^2 + ... + P5 l^5)          [cycles]
// psi0, th0: fractions of a period / cycle as 64-bit fixed point, split into
// the high (psi0, th0) and low (psi0lo, th0lo) 32 bits; n1, m1: the linear
// coefficients as 32-bit fixed point (mod 1) with the rounding residual kept
// in p1lo / m1lo (FP32); the quadratic coefficients P2 and k_c P2 as signed
// 64-bit fixed point in 2^-64 periods / cycles per sample^2 (q2, kq2);
// P3..P5 in FP32.
struct Anchor {
  uint32_t psi0, n1, th0, m1;
  long long q2, kq2;
  float p1lo, m1lo, p3, p4;
  float p5;
  uint32_t psi0lo, th0lo, pad;
};
static_assert(sizeof(Anchor) == 64, "anchor layout");

// Everything the kernels need about one call, resolved on the host.
struct Plan {
  // problem
  double fs = 0, t_coh = 0, f_lo = 0, f_hi = 0, f_ref = 0, eps = 0;
  int64_t n_samples = 0, n_s = 0;
  int32_t n_seg_total = 0, n_bins = 0, half_bins = 0;  // k = b - half_bins
  double f_c = 0, k_c = 0;                               // demodulation frequency, f_c * t_coh
  int32_t n_templates = 0, top_k = 0, precision = 1, cut = 1;
  bool local = false;                                    // per-segment templates (t_i0 = 0 in every segment)
  // NUFFT
  int32_t n_fine = 0, w = 0;
  double sigma = 0, beta_es = 0;
  std::vector<int32_t> radices;                          // Stockham passes, product n_fine
  // templates
  std::vector<double> beta;                              // per template
  std::vector<int32_t> nseg;                             // per template
  int64_t n_spectra = 0;
  // mixed form work decomposition
  int32_t threads = 256;                                 // threads per CTA of the mixed spreader
  int32_t run = 0, span = 0, n_anchor = 0;               // samples per thread / per warp / anchors per segment
  bool allow_128 = false;                                // 128-thread CTAs keep the anchor expansion accurate
  int32_t lanes128 = 32;                                 // lanes per FP64 anchor in 128-thread CTAs (32, or 16
                                                         // where a whole warp's span is too long for the expansion)
  bool global_x = false;                                 // spreader reads samples from global memory (no TMA staging)
  int32_t chunk = 0;
  std::vector<Item> items;
  std::vector<int32_t> order;                            // queue position -> item (empty: in item order)
  bool tuned_items = false;                              // items and order are the tuner's choice
  int32_t ctas = 0;                                      // power cube: resident CTAs per SM the tuner chose (0: all that fit)
  std::vector<int32_t> item_off;                         // [n_templates+1] first item of template m
  // tables (FP64, converted by the launcher)
  std::vector<double> corr;                              // [n_bins] deconvolution factor
  std::vector<double> tw_re, tw_im;                      // [n_fine] exp(-2 pi i m / n_fine)
};

// Sec. II Eq. (beta) for chirp mass mc (Msun) at frequency f (Hz), in 1/s.
double chirp_beta(double mc, double f);

// True when SRS_NO_TMA=1 is set in the environment: the mixed spreader then
// stages samples without TMA bulk copies (srs_capi.cpp).
bool tma_disabled();

// Message for k_mixed's error flag (srs_capi.cpp): flag[0] = 1 when a wait for
// a TMA copy gave up (flag[1..4]: item, segment, parity, block), 2 when the
// spreader's cell walk stopped at its bound with samples unused (item,
// segment, the lane's first sample, block).
void err_flag_message(const int* flag, char* buf, size_t n);

// Host planner (srs_plan.cpp).  Returns SRS_OK or an error with `msg` set.
// With betas_in != NULL the templates are given by their chirp parameters
// (mc is ignored); with local = true every segment is resampled with a 0PN
// template that starts at the segment's first sample (spectra mode only).
srs_status make_plan(const srs_params& p, const double* mc, int32_t n_templates,
                     int64_t n_samples, bool need_segments_all, int32_t seg_begin,
                     int32_t seg_end, Plan& out, std::string& msg,
                     const double* betas_in = nullptr, bool local = false);
void fill_info(const Plan& pl, srs_plan_info* info);
// Deconvolution factors of the mixed form in FP32: the plan's factors times
// 2^-E (E = beta_ES log2 e), the constant of the ES kernel that the spreader
// leaves out of its taps.
std::vector<float> mixed_corr(const Plan& pl);
// beta_ES log2 e as the mixed-form kernels use it (FP32).
float mixed_es_e(const Plan& pl);
// Threads per CTA of the mixed spreader and the run / span / anchor layout that
// follows: one FP64 anchor per 32 lanes (per lanes128 lanes in 128-thread CTAs).
void set_cta(Plan& pl, int32_t threads);
// Samples per thread of the mixed spreader for CTAs of `threads` threads (odd).
int32_t run_for(int64_t n_s, int32_t threads);
// Work items of the mixed form for a given chunk size (search: each template's
// first nseg_m segments; spectra: [seg_begin, seg_end) of every template).
// With tail_singles > 0 (search mode, chunk > 1) the last segments of every
// template, about tail_singles in all, become one-segment items queued after
// all the others, so that the persistent kernel's last wave is fine-grained.
void make_items(Plan& pl, int32_t chunk, bool spectra_mode, int32_t seg_begin, int32_t seg_end,
                int32_t tail_singles = 0);

}  // namespace srs
