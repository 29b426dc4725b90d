// srs_learn.h -- sizes, argument blocks and launchers of the learned-proposal
// kernels (internal; the public constants are in include/srs.h).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "srs_kernels.h"

namespace srs {

constexpr int kPatchTemplates = SRS_MLP_TEMPLATES;  // 9 coarse templates
constexpr int kPatchBins = SRS_MLP_BINS;            // 33 bins
constexpr int kPatchSize = SRS_MLP_INPUTS;          // 297
constexpr int kHidden = SRS_MLP_HIDDEN;             // 64
constexpr int kParams = SRS_MLP_PARAMS;             // W1, b1, w2, b2
static_assert(kPatchSize == kPatchTemplates * kPatchBins, "patch size");
static_assert(kParams == kHidden * kPatchSize + 2 * kHidden + 1, "parameter count");
constexpr int kSparseMaxBins = 8;                   // bins per refinement work item
constexpr int kSparseChunk = 16;                    // segments per refinement work item
// Above this many requested bins a template is refined through the NUFFT
// (one spectrum gives every bin) instead of direct sums.  A direct-sum pass
// over a segment costs about a sixth of a NUFFT spectrum plus, per bin, a
// sine and cosine (or, for the next bin up, one complex rotation): two groups
// of eight bins cost about as much as the spectrum.
constexpr int kDirectMaxBins = 16;

struct InjectionDev {
  double beta, f0, amp, phi0_cyc, t_end;
};

struct AdamArgs {
  float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
};

struct SparseItem {
  int m, i0, i1, b0, nb, pad0, pad1, pad2;
};

struct SparseArgs {
  int n_s, span, half_bins;
  int run;                        // samples per lane (consecutive), span = 32 run
  int kc_int;                     // f_c t_coh when it is a whole number in [1, 2^30), else 0
  float kc, inv_ns;
  AnchorArgs aa;
};

cudaError_t launch_make_strain(float* out, long long n, double fs, unsigned long long seed, int noise,
                               const InjectionDev* inj, int n_inj, int n_sm, cudaStream_t st);
cudaError_t launch_patches(const float* map, int n_templates, int n_bins, const int* cm, const int* cb, int n,
                           float* out, int n_sm, cudaStream_t st);
cudaError_t launch_mlp_forward(const float* X, int n, const __half* W1h, const float* b1, const __half* w2h,
                               const float* b2, float* logits, float* Z1, int n_sm, cudaStream_t st);
// The network's logit for every cell of a [n_templates][n_bins] map on the
// tensor cores (srs_score_tc.cu): one persistent CTA of 128 threads per SM,
// score_tc_smem_bytes() of dynamic shared memory.  err[0] = 1 (err[1] = the
// tile) if a wait for the tensor cores gave up.
size_t score_tc_smem_bytes();
cudaError_t launch_score_tc(const float* map, int n_templates, int n_bins, const __half* W1h, const float* b1,
                            const __half* w2h, const float* b2, float* scores, int* err, int n_sm,
                            cudaStream_t st);
cudaError_t launch_bce(const float* logits, const float* y, int n, float* dz, float* loss_terms, cudaStream_t st);
cudaError_t launch_mlp_grad(const float* X, int n, const float* Z1, const float* dz, const __half* w2h, float* g,
                            cudaStream_t st);
cudaError_t launch_adam(float* w, const float* g, float* m1, float* m2, const AdamArgs& a, __half* W1h, __half* w2h,
                        cudaStream_t st);
cudaError_t launch_weights_to_half(const float* w, __half* W1h, __half* w2h, cudaStream_t st);
cudaError_t launch_gather_batch(const float* X, const float* y, const int* idx, int n, float* Xb, float* yb,
                                int n_sm, cudaStream_t st);
cudaError_t launch_sparse_bins(const float* strain, const SparseItem* items, int n_items, const double* betas,
                               const int* bins, const SparseArgs& a, float* partial, int n_sm, cudaStream_t st);
cudaError_t launch_sparse_reduce(const float* partial, const int* cell_item0, const int* cell_nitems,
                                 const int* cell_slot, const int* cell_nseg, int n_cells, float* out, cudaStream_t st);

}  // namespace srs
