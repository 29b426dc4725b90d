// srs_kernels.h -- kernel argument blocks and launchers of libsrs (internal).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "srs_internal.h"

namespace srs {

constexpr int kTopkTile = 4096;  // keys per top-k tile (k <= kTopkTile / 2)
// at most this many k_reduce_mixed_top32 blocks per SM; each leaves 32 keys in
// the caller's scratch, which must hold kTop32BlocksPerSm * n_sm * 32 keys
constexpr int kTop32BlocksPerSm = 8;

struct AnchorArgs {
  double fs, t_coh, f_c;
  long long n_s;
  int span, n_anchor;
  int local;                      // 1: every segment's template starts at its first sample (t_i0 = 0)
};

struct MixedArgs {
  int n_s, n_fine, n_bins, half_bins;
  int run, span, n_anchor, n_pass;
  int ns4, nb4;                   // n_s, n_bins rounded up to multiples of 4 (shared-memory layout)
  int chunk;                      // most segments in one item
  int use_tma;                    // 1: samples staged by TMA bulk copies (n_s % 4 == 0, 16-byte aligned strain);
                                  // 0: samples read straight from the strain in global memory
  int threads;                    // threads per CTA (128 or 256); run, span and n_anchor follow it
  int fft_fixed;                  // 1200: the compile-time in-place 10-10-12 transform applies; 0: generic passes
  int seg_begin, seg_range;       // spectra output: first segment, segments per template
  AnchorArgs aa;                  // FP64 anchor inputs
  float kc;                       // f_c * t_coh
  int kc_int;                     // f_c * t_coh when it is a whole number in [1, 2^30), else 0
  float inv_ns;                   // 1 / n_s
  float es_beta_log2e;            // ES shape parameter * log2(e)
  float two_over_w;
  unsigned long long wofs;        // W / (2 n_fine) periods in 2^-64 fixed point (half the kernel's footprint)
  unsigned long long inv_n64;     // 2^64 / n_fine rounded: one fine-grid cell in 2^-64 periods
  const float* corr;              // [n_bins] deconvolution factors
  const float* tw;                // [2 n_fine] interleaved exp(-2 pi i m / n_fine)
  const int* order;               // [n_items] queue position -> item, or NULL (item order)
  float2* grid_out;               // spectra mode: write the spread grid [template][segment][n_fine]
  float* cube_out;                // spectra mode: write P = 2|F|^2/n_s to [template][bin][segment - seg_begin]
                                  // here and skip FFT / deconvolution (the cuFFT comparison), or NULL
  int8_t radices[16];
};

struct PlainArgs {
  double fs, t_coh, f_c, beta_es;
  int n_s, n_fine, n_bins, half_bins;
  int w, n_pass, seg_begin, seg_range;
  const double* corr;             // [n_bins]
  const double* tw;               // [2 n_fine]
  int8_t radices[16];
};

size_t mixed_smem_bytes(const MixedArgs& a);

// The fixed-point constants of the mixed spreader's time map for a plan:
// W / (2 n_fine) periods and one fine-grid cell (1 / n_fine periods), both in
// 2^-64 periods, rounded to nearest.
inline void mixed_fixed_point(const Plan& pl, MixedArgs& a) {
  const unsigned __int128 one = (unsigned __int128)1 << 64;
  const unsigned __int128 n = (unsigned __int128)pl.n_fine;
  a.wofs = (unsigned long long)(((unsigned __int128)pl.w * one + n) / (2 * n));
  a.inv_n64 = (unsigned long long)((2 * one + n) / (2 * n));
}

cudaError_t launch_anchors(const Item* items, int n_items, const double* betas, const AnchorArgs& aa,
                           Anchor* out, long long total, int n_sm, cudaStream_t st);
cudaError_t launch_to_f32(const double* in, float* out, long long n, int n_sm, cudaStream_t st);
cudaError_t launch_mixed(bool spectra, int w, const float* strain, const Item* items, int n_items,
                         const double* betas, int* queue, const MixedArgs& a, float* partial, double2* Fout,
                         int* err, int n_sm, int ctas_per_sm, cudaStream_t st);
cudaError_t launch_plain(bool f64_in, bool spectra, const void* strain, const double* betas, const int* nseg,
                         const PlainArgs& p, int grid_x, int n_templates, double* S, double2* Fout,
                         cudaStream_t st);
cudaError_t launch_reduce_mixed(const float* partial, const int* item_off, const int* nseg, int n_templates,
                                int n_bins, float* map, unsigned long long* keys, int n_sm, cudaStream_t st);
// k <= 32: the same reduction with the top k selected on the way (warp lists,
// block lists in scratch[blocks * 32], the last block writes cands); *ticket
// starts at zero and is left at zero.  Blocks: at most 4 per SM.
cudaError_t launch_reduce_mixed_top32(const float* partial, const int* item_off, const int* nseg, int n_templates,
                                      int n_bins, float* map, int k, unsigned long long* scratch, int* ticket,
                                      srs_candidate* cands, int n_sm, cudaStream_t st);
// F[s][b] = G[s][k(b)] * corr[b] for the grids G of n_spec spectra (after an
// external FFT), k(b) = b - half_bins wrapped into [0, n_fine).
// Arms an mbarrier for a transfer that never comes and waits on it with the
// spreader's bounded wait: err[0] = 1 once the wait gives up (about 1 s).
cudaError_t launch_wait_selftest(int* err, cudaStream_t st);
cudaError_t launch_grid_deconv(const float2* grid, long long n_spec, int n_fine, int n_bins, int half_bins,
                               const float* corr, double2* F, int n_sm, cudaStream_t st);
cudaError_t launch_finish_plain(const double* S, const int* nseg, int n_templates, int n_bins, float* map,
                                unsigned long long* keys, int n_sm, cudaStream_t st);
long long topk_scratch_keys(long long n, int k);
cudaError_t launch_topk(const unsigned long long* keys, long long n, int k, unsigned long long* buf_a,
                        unsigned long long* buf_b, const unsigned long long** result, int* launches,
                        cudaStream_t st);
cudaError_t launch_keys_to_cands(const unsigned long long* keys, int k, int n_bins, srs_candidate* out,
                                 cudaStream_t st);
cudaError_t launch_time_map_mixed(const Anchor* anchors, int n_items, const MixedArgs& a, double* psi,
                                  double* th, cudaStream_t st);
cudaError_t launch_time_map_plain(const int* item_m, const int* item_i, int n_items, const double* betas,
                                  const PlainArgs& p, double* psi, double* th, cudaStream_t st);

}  // namespace srs
