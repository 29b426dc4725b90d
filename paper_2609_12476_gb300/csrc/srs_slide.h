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
};

// One stack-slide pass over the cube chunk that holds segments
// [seg_begin, seg_end) as cube[(k n_bins + j) ld + (i - seg_begin)], ld =
// seg_end - seg_begin.  first: the running sums start at zero; last: the
// n_sigma map and top-k keys are written.
struct SlideArgs {
  int n_rows, n_t0, n_total;
  int seg_begin, seg_end, ld;
  int first, last;
};

// cell[r][s] = k_s n_bins + j_s of the s-th segment of row r's track, -1 past
// its end; len[r] = the track's length.  beta0[r] = beta(Mc_r, f0), frac[r] =
// the row's t0 fraction c in [0, 1).
cudaError_t launch_slide_tracks(const double* beta0, const double* frac, int n_rows, const TrackArgs& t,
                                int* cell, int* len, int n_sm, cudaStream_t st);

// Stack-slide: Z[r][n] (+)= sum over the chunk's track segments of (P - 2) / 2;
// with a.last, map[r][n] = Z / sqrt(N_seg) (0 for an empty track) and keys for
// the top-k.  map may be NULL.
cudaError_t launch_stack_slide(const float* cube, const int* cell, const int* len, const double* frac,
                               const SlideArgs& a, float* Z, float* map, unsigned long long* keys,
                               cudaStream_t st);

}  // namespace srs
