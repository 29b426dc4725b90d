// srs_slide.h -- kernels of the two-stage search: tracks of the stack-slide
// templates theta = {Mc, t0} and the stack-slide sum over a per-segment power
// cube (Sec. III.C).  Internal to libsrs.
#pragma once

#include <cuda_runtime.h>

#include "../../include/srs.h"

namespace srs {

// Track geometry of one search (all rows share it).
struct TrackArgs {
  double f0;          // frequency at t0 (Hz)
  double f_lo;        // lower band edge (Hz); bin j is f_lo + j / t_coh
  double t_coh;       // segment length (s)
  double beta_min;    // first bank entry (1/s)
  double dbeta;       // bank spacing (1/s); 0 for a one-entry bank
  int n_beta, n_bins, n_total;
  int weighting;      // SRS_WEIGHT_EQUAL or SRS_WEIGHT_AMPLITUDE
  const float* s_eff; // [n_beta][n_bins] effective PSD relative to white noise, or NULL
  int s_in_weights_only;  // 1: the cube is whitened already; s_eff enters the weights alone
};

// One stack-slide pass over the cube chunk that holds segments
// [seg_begin, seg_end) as cube[(k n_bins + j) ld + (i - seg_begin)], ld =
// seg_end - seg_begin.  first: the running sums start at zero; last: the
// n_sigma map and top-k keys are written.
struct SlideArgs {
  int n_rows, n_t0, n_total;
  int seg_begin, seg_end, ld;
  int first, last;
  int weighted;       // 0: equal weights and a white PSD (every coefficient is (1/2, 1))
  int off32;          // 1: every cube index cell * ld + segment fits 32 bits (cube chunk < 2^32 elements)
};

// cell[r][s] = k_s n_bins + j_s of the s-th segment of row r's track, -1 past
// its end; coef[r][s] = (a_s / (2 S_s), a_s) with a_s = A_s^2 / S_s, so that
// the segment's term a_s (P / S_s - 2) / 2 is one FMA; len[r] = the track's
// length; w2[r][L] = sum_{s < L} a_s^2 (n_total + 1 entries per row).
// beta0[r] = beta(Mc_r, f0), frac[r] = the row's t0 fraction c in [0, 1).
cudaError_t launch_slide_tracks(const double* beta0, const double* frac, int n_rows, const TrackArgs& t,
                                int* cell, float2* coef, int* len, double* w2, int n_sm, cudaStream_t st);

// Stack-slide: Z[r][n] (+)= sum over the chunk's track segments of
// a_s (P / S_s - 2) / 2; with a.last, map[r][n] = Z / sqrt(w2[r][N_seg]) (0
// for an empty track) and keys for the top-k.  map may be NULL.
cudaError_t launch_stack_slide(const float* cube, const int* cell, const float2* coef, const int* len,
                               const double* w2, const double* frac, const SlideArgs& a, float* Z, float* map,
                               unsigned long long* keys, cudaStream_t st);

// Whitening of a cube [rows = n_beta n_bins][ld] over its first n_seg
// segments, in place (Sec. III.C): S[r] = mean_i P / 2 (estimate_s), then
// per segment mu_i, sigma_i of P / S over all rows, then
// P <- 2 + 2 (P / S - mu_i) / sigma_i.  mu, sigma (device, n_seg floats) may
// be NULL.  sums is device scratch of 2 n_seg doubles, musig of n_seg float2.
cudaError_t launch_cube_whiten(float* cube, long long rows, int ld, int n_seg, float* S, bool estimate_s,
                               double* sums, float2* musig, float* mu, float* sigma, int n_sm, cudaStream_t st);

}  // namespace srs
