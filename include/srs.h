/*
 * srs.h -- C ABI of the GB300 semicoherent resampling search (libsrs.so).
 *
 * The search follows arXiv:2609.12476 (Lu, Palomba, Piccinni, Sun):
 *   Sec. III.B  resample each coherent segment with the 0PN time tau(t; beta)
 *               (Eq. new_t) so that a chirp becomes monochromatic
 *               (Eq. monochromatic), and take the segment's spectrum with a
 *               type-1 non-uniform FFT;
 *   Sec. III.C  normalise the powers (Eq. normalized_power), sum them over
 *               segments with equal weights (Eq. weights) into the
 *               semicoherent statistic n_sigma (Eq. semicoherent_statistic);
 *   and keep the top-k (template, bin) cells.
 *
 * Conventions shared by every call
 *   - Templates are chirp masses mc[m] (solar masses) quoted at f_ref; the
 *     resampling parameter is beta_m = beta(f_ref, mc[m]) of Eq. (beta).
 *   - Time t = 0 is the first strain sample; segment i covers samples
 *     [i*n_s, (i+1)*n_s) with n_s = t_coh*fs.  Within segment i the
 *     resampled time is delta_j = tau(t_i0 + j/fs) - tau(t_i0) (Eq. new_t,
 *     referenced to the segment start).
 *   - Bins b = 0..n_bins-1 are the frequencies f_b = f_lo + b/t_coh with
 *     n_bins = (f_hi - f_lo)*t_coh.  The spectrum of a segment is
 *     F_b = sum_j x_j exp(-2 pi i f_b delta_j), no 1/N factor.
 *   - Power P = 2 |F_b|^2 / n_s (Eq. normalized_power for unit-variance white
 *     noise); template m sums its first nseg_m segments, nseg_m = whole
 *     30 s segments its 0PN track spends below f_hi (Sec. II duration,
 *     Sec. V), clamped to [1, segments in the data]; with equal weights and
 *     mu = sigma = 2, n_sigma[m][b] = (sum_i P - 2 nseg_m) / (2 sqrt(nseg_m)).
 *   - Top-k ordering: n_sigma descending, then template ascending, then bin
 *     ascending.
 *
 * Ownership and memory
 *   - The caller owns every buffer passed in or out.  With
 *     params.io_on_device = 1 the strain, map, candidate and spectra
 *     pointers are device pointers on the context's device; with 0 they are
 *     host pointers and the call copies them.  Template lists (mc) are always
 *     host pointers.
 *   - The context owns its device workspace (allocated on first use, grown
 *     when a larger problem arrives, freed by srs_destroy) and its stream.
 *   - Every call is synchronous with respect to the host: it returns after
 *     the results are in the caller's buffers.
 *
 * Errors
 *   - Every call returns an srs_status; nothing throws or aborts across the
 *     ABI.  srs_last_error() gives the context's last message.
 *   - SRS_ERR_ARG: a NULL pointer where one is needed, a non-integer
 *     t_coh*fs or band width, f_hi > fs/2, eps outside [1e-12, 1e-1], top_k
 *     outside [1, 1024] or larger than the map, fewer samples than one
 *     segment.
 *   - SRS_ERR_DOMAIN: a computed segment reaches coalescence
 *     (1 - (8/3) beta t <= 0, Sec. II), possible with cut_segments = 0.
 *   - SRS_ERR_UNSUPPORTED: a combination this build does not run (e.g. the
 *     mixed form below its FP32 floor, eps < 2e-7, or a template chirping
 *     too fast for the mixed form's anchor spacing, such as Mc = 0.1 in a
 *     band that starts at 80 Hz or above; SRS_PLAIN_FP64 runs those; or
 *     more than 2^31 - 1 segment spectra in one call).
 *   - SRS_ERR_CUDA / SRS_ERR_OOM: a CUDA call failed / device memory ran out;
 *     the context stays usable for smaller problems.
 *   - SRS_ERR_TIMEOUT: a device-side bound was reached and the kernel
 *     returned instead of waiting on: a wait for a TMA copy gave up, or the
 *     spreader's cell walk stopped at its cell bound (possible only with a
 *     time map that steps back, which the planner's range excludes); the
 *     message names the item and segment and the context stays usable.
 *   - Threading: one context per host thread.
 */
#ifndef SRS_H
#define SRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srs_ctx srs_ctx;

typedef enum {
  SRS_OK = 0,
  SRS_ERR_ARG = -1,
  SRS_ERR_OOM = -2,
  SRS_ERR_CUDA = -3,
  SRS_ERR_TIMEOUT = -4,
  SRS_ERR_UNSUPPORTED = -5,
  SRS_ERR_DOMAIN = -6
} srs_status;

/* Element type of the strain buffer. */
typedef enum { SRS_F32 = 0, SRS_F64 = 1 } srs_dtype;

/* Arithmetic of the segment transform.
 * SRS_PLAIN_FP64: every step in FP64, one CTA per spectrum, tau evaluated
 *   per sample (the comparison form).
 * SRS_MIXED: tau and the per-segment phase reference in FP64 at a few anchor
 *   samples per segment, sample offsets as 32-bit fixed-point phase plus an
 *   FP32 polynomial, spreading / FFT / power in FP32 with FP32 accumulation,
 *   persistent kernels over (template, segment-chunk) work. */
typedef enum { SRS_PLAIN_FP64 = 0, SRS_MIXED = 1 } srs_precision;

/* Search parameters (Sec. III; defaults in brackets are the paper's search). */
typedef struct {
  double fs;           /* strain sample rate [Hz] */
  double t_coh;        /* coherent segment length [s] [30]; t_coh*fs integer */
  double f_lo;         /* band start [Hz] [40] */
  double f_hi;         /* band end (exclusive) [Hz] [60] */
  double f_ref;        /* frequency at which template chirp masses give beta [Hz] [40] */
  double eps;          /* NUFFT relative tolerance (FINUFFT sense) [1e-6] */
  double sigma;        /* fine-grid oversampling; 0 = choose from eps and shared memory */
  int32_t top_k;       /* candidates to return [32] */
  int32_t precision;   /* srs_precision */
  int32_t cut_segments;/* 1: template m sums its nseg_m in-band segments; 0: all segments */
  int32_t io_on_device;/* 1: strain / outputs are device pointers; 0: host pointers */
  int32_t chunk;       /* segments per work item in the mixed form; 0 = autotune */
  int32_t deterministic; /* reserved, must be 0 or 1; the reduction is always ordered */
} srs_params;

/* Host-side plan (no GPU needed): what srs_plan chose. */
typedef struct {
  int64_t n_s;            /* samples per segment */
  int32_t n_seg_total;    /* whole segments in the strain */
  int32_t n_bins;         /* bins per spectrum */
  int32_t n_fine;         /* fine (oversampled) grid size, a 2^a 3^b 5^c number */
  int32_t w;              /* spreading kernel width in fine-grid cells */
  double beta_es;         /* exponential-of-semicircle shape parameter */
  double sigma;           /* n_fine / n_bins */
  int64_t n_spectra;      /* sum over templates of nseg_m */
  int32_t chunk;          /* segments per work item (mixed form) */
  int32_t n_items;        /* work items (mixed form) */
} srs_plan_info;

/* One candidate cell of the statistic map. */
typedef struct {
  float value;            /* n_sigma */
  int32_t template_idx;   /* m */
  int32_t bin;            /* b, frequency f_lo + b/t_coh */
} srs_candidate;

/* Timings and choices of the last call (all optional to read). */
typedef struct {
  double device_ms;       /* device time of the transform + statistic + top-k */
  double spectra_per_s;   /* n_spectra / device time */
  int64_t n_spectra;
  int32_t w;
  int32_t n_fine;
  double sigma;
  double beta_es;
  int32_t chunk;
  int32_t n_items;
  int32_t kernel_launches;/* kernels this call launched */
  double spread_ms;       /* device time of the transform kernel alone (k_mixed / k_plain) */
  int32_t cta_threads;    /* threads per CTA of the transform kernel */
  int32_t staging;        /* mixed form: 1 = samples staged by TMA bulk copies, 0 = read from global memory */
  int32_t ctas_per_sm;    /* mixed form: resident CTAs per SM the search asked for (0 = as many as fit) */
  double fft_ms;          /* srs_segment_spectra_cufft only: device time of the cuFFT transforms */
  double slide_ms;        /* two-stage calls: device time of the stack-slide kernels */
  int64_t slide_reads;    /* two-stage calls: cube powers the stack-slide summed (track segments over all templates) */
} srs_report;

/* Environment variables read by the library (diagnostics and profiling):
 *   SRS_NO_TMA=1          never stage samples with TMA bulk copies;
 *   SRS_MIXED_LAYOUT=T:S[:C:K]  restrict the autotuner to T threads per CTA
 *                         (128 or 256) and staging S (tma or global), and with
 *                         C:K to C segments per item and K CTAs per SM;
 *   SRS_NO_GRAPHS=1       launch a search's kernels directly instead of
 *                         replaying a captured CUDA graph (read at srs_create). */

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * the context will use (NULL: the context creates its own non-blocking
 * stream).  *out receives the context.  Errors: SRS_ERR_ARG, SRS_ERR_CUDA. */
srs_status srs_create(srs_ctx** out, int device, void* cuda_stream);

/* Free the workspace and the context (NULL is allowed). */
void srs_destroy(srs_ctx* ctx);

/* Last error message of `ctx` (static text when ctx is NULL).  Owned by the
 * context; valid until the next call on it. */
const char* srs_last_error(const srs_ctx* ctx);

/* Host-only planner (Sec. II Eq. beta and duration; Sec. III.B NUFFT sizes):
 * fills `info`, beta_out[n_templates] (may be NULL) and nseg_out[n_templates]
 * (may be NULL) for a strain of n_samples.  No GPU is touched. */
srs_status srs_plan(const srs_params* params, const double* mc, int32_t n_templates,
                    int64_t n_samples, srs_plan_info* info, double* beta_out,
                    int32_t* nseg_out);

/* The semicoherent search (Sec. III.B-C): for every template m and its
 * nseg_m segments, the segment spectra, powers, their sum, n_sigma and the
 * top-k cells.
 *   strain     [n_samples] of `dtype`, host or device per params.io_on_device
 *   mc         [n_templates] host, chirp masses (solar masses) at f_ref
 *   stat_map   [n_templates][n_bins] float n_sigma, or NULL to skip
 *   cands      [top_k] candidates, ordered as above
 *   n_cands    host int32: number of candidates written (min(top_k, map size))
 *   report     host, may be NULL */
srs_status srs_search(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                      const double* mc, int32_t n_templates, const srs_params* params,
                      float* stat_map, srs_candidate* cands, int32_t* n_cands,
                      srs_report* report);

/* Stream-ordered form of srs_search.  Enqueues the same device sequence on
 * the context's stream and returns without waiting; *n_cands is set at once.
 * Outputs are valid, and a device-side failure (a staging wait that gave up)
 * is reported, only after srs_sync; keep every buffer alive and the strain
 * unchanged until then.  Calls may be queued back to back; a new shape's
 * first call still plans and tunes synchronously.  Errors found on the host
 * (arguments, planning) return at once.
 *   params->io_on_device = 1: strain, stat_map and cands are device pointers.
 *   params->io_on_device = 0: host pointers.  The strain goes up on a second
 *     stream into one of two device staging buffers, so a queued call's
 *     upload overlaps the previous call's search; the results come back
 *     when the stream reaches them.  Page-locked (pinned) host buffers are
 *     needed for the copies to overlap; pageable ones work, without overlap. */
srs_status srs_search_async(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                            const double* mc, int32_t n_templates, const srs_params* params,
                            float* stat_map, srs_candidate* cands, int32_t* n_cands);

/* Wait for the context's stream and settle every srs_search_async since the
 * last srs_sync: SRS_ERR_TIMEOUT if any of them failed on the device.  With
 * report != NULL: the last call's sizes, and device_ms / spread_ms averaged
 * over the settled calls (CUDA events around each call's sequence and its
 * transform kernel).  More than 256 unsettled calls settle the oldest 256
 * internally; a failure among them is returned here. */
srs_status srs_sync(srs_ctx* ctx, srs_report* report);

/* Segment spectra F_b for templates [0, n_templates) and segments
 * [seg_begin, seg_end) (Sec. III.B), through the same time map, spreader,
 * FFT and deconvolution as srs_search.
 *   F  [n_templates][seg_end-seg_begin][n_bins] complex double (re, im
 *      interleaved), host or device per params.io_on_device.
 * Segments past a template's nseg_m are still computed (the cut applies
 * only to the sum); SRS_ERR_DOMAIN if any reaches coalescence. */
srs_status srs_segment_spectra(srs_ctx* ctx, const void* strain, int64_t n_samples,
                               int32_t dtype, const double* mc, int32_t n_templates,
                               int32_t seg_begin, int32_t seg_end, const srs_params* params,
                               double* F, srs_report* report);

/* Detection statistics (host only; no context or GPU needed).
 * Threshold (Sec. III.C Eq. n_sigma^th): the n_sigma^th with
 * P(n_sigma > n_sigma^th | H0) = p_fa for one template whose track has n_seg
 * segments with weights w[n_seg] (any positive scale; normalised here so that
 * sum w^2 = 1), or equal weights when w is NULL.  Under H0,
 * n_sigma = sum w_i (E_i - 1) with E_i ~ Exp(1) (P_i ~ chi^2 with 2 dof):
 * for equal weights a scaled chi^2 with 2 n_seg dof, otherwise a generalised
 * chi^2, evaluated as a mixture of Gamma laws (Moschopoulos 1985), or, for
 * weights spread so widely that the mixture would need too many terms, by
 * Imhof's inversion of the characteristic function (whichever is cheaper).
 * SRS_ERR_ARG for n_seg < 1, p_fa outside (0, 1) or a weight <= 0;
 * SRS_ERR_UNSUPPORTED when both routes would take about 1e12 operations or
 * more (unequal weights on tracks of about a million segments). */
srs_status srs_nsigma_threshold(const double* w, int32_t n_seg, double p_fa, double* n_sigma_th);

/* Detection non-centrality (Eq. non-centrality_threshold): the total
 * non-centrality Lambda = sum_i lambda_i for which n_sigma exceeds the p_fa
 * threshold with probability p_det.  Equal weights (w NULL): sum P is
 * non-central chi^2 with 2 n_seg dof, evaluated exactly.  Weights w[n_seg]:
 * the signal's share of segment i is lambda_i = Lambda w_i / sum w (weights
 * that follow A_i^2 / S_i follow the signal power), and the weighted sum is
 * evaluated by Imhof's inversion of its characteristic function inside a
 * bisection on Lambda (about 40 evaluations, each costing order n_seg^2).
 * The paper quotes Lambda_1 = 46.5 for n_seg = 1, p_fa = 1e-6, p_det = 0.95.
 * SRS_ERR_ARG for n_seg < 1, p_fa or p_det outside (0, 1) or a weight <= 0. */
srs_status srs_detection_noncentrality(const double* w, int32_t n_seg, double p_fa, double p_det, double* lambda);

/* Receiver operating characteristic of one signal (Sec. III.C, Fig. roc for a
 * single signal; the left side of Eq. non-centrality_threshold):
 *   p_det[q] = P(n_sigma > n_sigma^th(p_fa[q]) | lambda, w),  q < n_points,
 * for one template whose track has n_seg segments with weights w[n_seg] (any
 * positive scale; NULL: equal weights) and signal non-centralities
 * lambda[n_seg] >= 0 per segment (the signal's normalised power there; NULL:
 * no signal, so p_det = p_fa).  Equal weights: exact (sum P is non-central
 * chi^2 with 2 n_seg dof and non-centrality sum lambda_i).  Unequal weights:
 * the threshold from the exact central law, then Imhof's integral, whose
 * absolute error stays below about 1e-9; its cost grows as n_seg^2 per point.
 * All arrays are host memory owned by the caller; p_det has n_points entries.
 * SRS_ERR_ARG for n_seg < 1, n_points < 1, a p_fa outside (0, 1), a weight
 * <= 0 or a lambda that is negative or not finite. */
srs_status srs_detection_probability(const double* w, const double* lambda, int32_t n_seg, const double* p_fa,
                                     int32_t n_points, double* p_det);

/* Diagnostic: runs the spreader's bounded staging wait on a transfer that never
 * comes (one thread, about one second) and returns what a search would:
 * SRS_ERR_TIMEOUT with the give-up recorded in srs_last_error().  The wait
 * ends by its own limit, so no kernel hangs and the context stays usable. */
srs_status srs_selftest_wait(srs_ctx* ctx);

/* Timed comparison only: the same segment spectra as srs_segment_spectra()
 * in the mixed form, computed unfused.  k_mixed writes each segment's spread
 * grid (n_fine complex float, Sec. III.B spreading step) to device memory,
 * cuFFT's batched single-precision C2C forward transform runs on it, and a
 * third kernel deconvolves and selects the band.  Arguments, layout and
 * ownership as srs_segment_spectra(); params->precision must be SRS_MIXED.
 * The grid scratch (n_templates * (seg_end-seg_begin) * n_fine * 8 bytes) and
 * the cuFFT plan belong to the context.  report->spread_ms is the spreading
 * kernel (after the FP32 strain copy, for float64 strain), report->fft_ms the
 * transforms, report->device_ms everything.
 * SRS_ERR_UNSUPPORTED when libcufft cannot be loaded at run time (the rest of
 * the library does not depend on it); SRS_ERR_ARG for another precision. */
srs_status srs_segment_spectra_cufft(srs_ctx* ctx, const void* strain, int64_t n_samples,
                                     int32_t dtype, const double* mc, int32_t n_templates,
                                     int32_t seg_begin, int32_t seg_end, const srs_params* params,
                                     double* F, srs_report* report);

/* The time map alone (Sec. III.B Eq. new_t), as the chosen precision form
 * evaluates it inside the spreader, for n_items (template, segment) pairs:
 *   psi_out   [n_items][n_s]  delta_j / t_coh modulo 1 (fine-grid phase, periods)
 *   theta_out [n_items][n_s]  f_c delta_j modulo 1, f_c = (f_lo + f_hi)/2 (cycles)
 * both host double arrays; item_m / item_i host int32 arrays.  The mixed
 * form steps each lane's 64-bit fixed-point phase from the lane's first
 * sample; this call uses the lanes of the default 256-thread layout (a tuned
 * search may start its lanes elsewhere, which moves the values by rounding
 * only, below 1e-13 periods). */
srs_status srs_time_map(srs_ctx* ctx, const double* mc, int32_t n_templates,
                        const int32_t* item_m, const int32_t* item_i, int32_t n_items,
                        const srs_params* params, int64_t n_samples, double* psi_out,
                        double* theta_out);

/* ------------------------------------------------------------------------
 * Two-stage search (Sec. III.B local bank, Sec. III.C stack-slide, Sec. VI).
 * Stage one resamples every segment with each entry of a bank of 0PN
 * templates that start at the segment's first sample and stores the powers
 * P = 2|F|^2/n_s (Eq. normalized_power, white unit-variance noise) as a cube.
 * Stage two sums, for each template theta = {Mc, t0} whose frequency passes
 * f0 at t0, the powers along its track: in every segment that starts at or
 * after t0, the bin nearest the 0PN frequency at the segment's first sample
 * (Eq. f) and the bank entry nearest the local chirp parameter beta(Mc, f)
 * (Eq. beta); the track ends where that bin leaves the band, at coalescence,
 * or at the end of the data.  n_sigma = sum w (P - 2)/2 with sum w^2 = 1
 * (Eq. semicoherent_statistic, mu = sigma = 2; equal weights 1/sqrt(N_seg),
 * or the amplitude / PSD weights of srs_slide_grid); 0 when the track has no
 * segment in the data.
 * ------------------------------------------------------------------------ */

/* The local resampling bank: n_beta chirp parameters uniform over
 * [beta_min, beta_max] (1/s); the paper's search uses 69 over 3e-8 .. 7e-4. */
typedef struct {
  double beta_min, beta_max;
  int32_t n_beta;
} srs_bank;

/* Stack-slide templates theta = {Mc, t0}.  Row r has chirp mass mc[r] (Msun)
 * and t0 fraction c[r] in [0, 1); column n has t0 = (n + c[r]) t_coh, so the
 * map is [n_rows][n_t0].  mc and c are host arrays.  f0 in [f_lo, f_hi) is
 * the frequency at t0 (the paper: the band's lower edge).
 * Weights (Sec. III.C Eq. weights, rectangular window Gamma = 1): segment s
 * of a track gets a_s = A_s^2 / S_s, normalised so that sum a_s^2 = 1 over
 * the track's segments in the data, where
 *   A_s^2 = 1 (SRS_WEIGHT_EQUAL), or the segment average of (f / f0)^(4/3)
 *           along the track (SRS_WEIGHT_AMPLITUDE; Sec. II Eq. h0, h0 ~ f^(2/3));
 *   S_s   = s_eff[k_s][j_s], the effective PSD of bank entry k, bin j
 *           relative to white unit-variance noise (host [n_beta][n_bins],
 *           every entry > 0), or 1 when s_eff is NULL.
 * The powers are normalised by the same S (Eq. normalized_power):
 * n_sigma = sum_s a_s (P_s / S_s - 2) / 2 / sqrt(sum_s a_s^2).
 * whiten = 1: the powers are whitened (srs_cube_whiten: divided by the
 * effective PSD, then centred and scaled per segment by the empirical
 * background mean and deviation mu_i, sigma_i), so S enters the weights
 * alone.  srs_slide_search whitens every cube chunk itself, with s_eff if
 * given, else with the PSD it estimates from the first chunk (which then
 * also enters the amplitude weights); srs_stack_slide takes the cube as
 * already whitened. */
enum { SRS_WEIGHT_EQUAL = 0, SRS_WEIGHT_AMPLITUDE = 1 };
typedef struct {
  double f0;
  const double* mc;
  const double* c;
  int32_t n_rows;
  int32_t n_t0;
  int32_t weighting;
  const float* s_eff;
  int32_t whiten;
} srs_slide_grid;

/* Flags of srs_stack_slide. */
enum { SRS_SLIDE_FIRST = 1, SRS_SLIDE_LAST = 2 };

/* Stage one for segments [seg_begin, seg_end):
 *   cube [n_beta][n_bins][seg_end - seg_begin] float, segment innermost,
 * host or device per params->io_on_device (caller-owned).  Mixed form only
 * (SRS_ERR_UNSUPPORTED otherwise); params->f_ref is not used (the bank gives
 * beta directly).  SRS_ERR_DOMAIN if a bank entry coalesces within one
 * segment.  report: device_ms, spread_ms (the transform kernel), sizes. */
srs_status srs_power_cube(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                          const srs_bank* bank, int32_t seg_begin, int32_t seg_end,
                          const srs_params* params, float* cube, srs_report* report);

/* Whitening of a power cube in place (Sec. III.C Eqs. normalized_power,
 * semicoherent_statistic, with the effective PSD and the background moments
 * taken from the data).  Device pointers:
 *   cube   [n_beta][n_bins][n_seg] float (srs_power_cube's layout);
 *   s_eff  [n_beta][n_bins] float: estimate = 1 writes
 *          S = mean over segments of P / 2 into it; estimate = 0 reads it;
 *   mu, sigma [n_seg] float or NULL: each segment's mean and (population)
 *          standard deviation of P / S over all (beta, bin).
 * Afterwards P = 2 + 2 (P / S - mu_i) / sigma_i, so the stack-slide's
 * (P - 2) / 2 is (P / S - mu_i) / sigma_i.  Queued on the context's stream
 * and waited for. */
srs_status srs_cube_whiten(srs_ctx* ctx, float* cube, int32_t n_beta, int32_t n_bins, int32_t n_seg,
                           float* s_eff, int32_t estimate, float* mu, float* sigma);

/* Stage two over one cube chunk holding segments [seg_begin, seg_end) of data
 * with n_seg_total segments, in srs_power_cube's layout (host or device per
 * params->io_on_device).  The running sums live in the context: flags
 * SRS_SLIDE_FIRST starts them at zero, SRS_SLIDE_LAST finishes the search and
 * writes nsigma_map [n_rows][n_t0] (may be NULL) and the top params->top_k
 * candidates (template_idx = row r, bin = column n), ordered by value
 * descending, then row, then column.  Chunks may come in any order between a
 * FIRST and a LAST call; a single call may carry both flags.  Uses t_coh,
 * f_lo, f_hi, top_k and io_on_device of params.  report: slide_ms.
 * SRS_ERR_UNSUPPORTED when n_beta * n_bins reaches 2^31 (32-bit track cells)
 * or the track table or map would hold more than 2e9 entries. */
srs_status srs_stack_slide(srs_ctx* ctx, const float* cube, int32_t seg_begin, int32_t seg_end,
                           int32_t n_seg_total, const srs_bank* bank, const srs_slide_grid* grid,
                           const srs_params* params, int32_t flags, float* nsigma_map,
                           srs_candidate* cands, int32_t* n_cands, srs_report* report);

/* Both stages over all whole segments of the strain.  cube_budget_bytes > 0
 * bounds the device cube: the data is processed in chunks of segments that
 * fit, and the running sums carry over between chunks (the partial-sum
 * caching of Sec. VI); 0 = one chunk.  Outputs as srs_stack_slide's LAST
 * call.  report: device_ms (everything), spread_ms (cube kernels), slide_ms
 * (stack-slide kernels), n_spectra (n_beta x segments). */
srs_status srs_slide_search(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                            const srs_bank* bank, const srs_slide_grid* grid, const srs_params* params,
                            int64_t cube_budget_bytes, float* nsigma_map, srs_candidate* cands,
                            int32_t* n_cands, srs_report* report);

/* ------------------------------------------------------------------------
 * Learned proposal.  A small network looks at a coarse-template n_sigma map
 * and proposes which fine (template, bin) cells to compute; the full
 * fine-template search stays the fallback and the yardstick.
 *   input   a 9 x 33 patch of the coarse map around a cell (templates m-4..m+4,
 *           bins b-16..b+16, zero outside the map), each value through asinh
 *   network 297 -> 64 (ReLU) -> 1 logit; weights used in FP16, sums in FP32;
 *           parameters travel as FP32 master values, one vector of
 *           SRS_MLP_PARAMS floats: W1[64][297] row-major, b1[64], w2[64], b2
 *   loss    binary cross entropy with logits, mean over the batch
 * ------------------------------------------------------------------------ */
#define SRS_MLP_TEMPLATES 9
#define SRS_MLP_BINS 33
#define SRS_MLP_INPUTS 297
#define SRS_MLP_HIDDEN 64
#define SRS_MLP_PARAMS 19137

/* One injected 0PN chirp (Sec. III.A Eqs. f and phi): chirp mass mc (Msun),
 * frequency f0 at t = 0, amplitude amp per sample, phase phi0 (rad). */
typedef struct {
  double mc;
  double f0;
  double amp;
  double phi0;
} srs_injection;

typedef struct {
  int32_t epochs;
  int32_t batch;
  float lr;          /* Adam step size */
  float beta1;       /* Adam first-moment decay */
  float beta2;       /* Adam second-moment decay */
  float adam_eps;
  uint64_t seed;     /* minibatch order */
} srs_train_cfg;

typedef struct {
  double device_ms;          /* coarse search + scoring + refinement */
  int64_t coarse_spectra;    /* spectra of the coarse search */
  int32_t proposed_coarse;   /* coarse cells above the score threshold */
  int32_t fine_cells;        /* fine (template, bin) cells evaluated */
  int64_t fine_segment_bins; /* (segment, bin) direct sums evaluated */
  int32_t fine_templates;    /* distinct fine templates touched */
} srs_proposal_report;

/* Synthetic strain for training and evaluation, written on the device:
 * out[j] = (noise ? N(0,1) : 0) + sum over injections of
 * amp cos(phi(j/fs)), where each chirp starts at t = 0 with frequency f0 and
 * stops where its 0PN frequency (Eq. f) reaches f_hi.  The noise is a
 * counter-based Philox-4x32 (10 rounds) stream `seed` with Box-Muller.
 *   out  device, [n] float; inj host, [n_inj]. */
srs_status srs_make_strain(srs_ctx* ctx, float* out, int64_t n, double fs, uint64_t seed, int32_t noise,
                           const srs_injection* inj, int32_t n_inj, double f_hi);

/* Network inputs for listed cells of a map [n_templates][n_bins]:
 * out[k][r][c] = asinh(map[cell_m[k] + r - 4][cell_b[k] + c - 16]) (0 outside).
 * map, cell_m, cell_b, out on the device when io_on_device = 1, else host. */
srs_status srs_patches(srs_ctx* ctx, const float* map, int32_t n_templates, int32_t n_bins,
                       const int32_t* cell_m, const int32_t* cell_b, int32_t n_cells, float* out,
                       int32_t io_on_device);

/* Logits of n inputs X[n][297]; params host [SRS_MLP_PARAMS]. */
srs_status srs_mlp_forward(srs_ctx* ctx, const float* X, int32_t n, const float* params, float* logits,
                           int32_t io_on_device);

/* Loss and its gradient with respect to every parameter (same layout as
 * params) over the batch X[n][297], labels y[n] in {0, 1}; grad and loss are
 * host pointers. */
srs_status srs_mlp_grad(srs_ctx* ctx, const float* X, const float* y, int32_t n, const float* params,
                        float* grad, float* loss, int32_t io_on_device);

/* Train in place: shuffled minibatches of the device set X[n][297], y[n],
 * Adam on the FP32 master parameters (host, in/out); mean training loss of
 * each epoch in loss_per_epoch (host, [cfg->epochs], may be NULL). */
srs_status srs_mlp_train(srs_ctx* ctx, const float* X, const float* y, int32_t n, const srs_train_cfg* cfg,
                         float* params, float* loss_per_epoch);

/* Network score (logit) of every cell of a device map; scores on the device,
 * [n_templates][n_bins]. */
srs_status srs_score_map(srs_ctx* ctx, const float* map, int32_t n_templates, int32_t n_bins,
                         const float* params, float* scores);

/* n_sigma of listed (template, bin) cells, each over its template's nseg_m
 * segments, from direct sums of the segment samples at those bins (the
 * transform the NUFFT approximates, Sec. III.B), in the mixed precision
 * (FP64 anchors, fixed-point phase, FP32 sums).  nsigma host, [n_cells]. */
srs_status srs_refine(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype, const double* mc,
                      int32_t n_templates, const srs_params* params, const int32_t* cell_m,
                      const int32_t* cell_b, int32_t n_cells, float* nsigma, srs_report* report);

/* How proposed coarse cells become fine cells. */
typedef struct {
  float score_threshold;   /* a coarse cell is proposed when its logit exceeds this */
  int32_t nms_templates;   /* non-maximum suppression half-window in coarse templates (0: off) */
  int32_t nms_bins;        /* ... and in bins (0: off) */
  int32_t fine_rows;       /* fine templates of coarse rows within this many of the cell (0: its own) */
  int32_t component_top;   /* > 0: of each 8-connected group of cells above the threshold, propose only
                              the component_top cells with the highest coarse n_sigma (suppression off) */
  int32_t nms_by_nsigma;   /* 1: the suppression window compares coarse n_sigma instead of scores */
  int32_t template_budget; /* > 0: refine at most this many fine templates -- those whose best proposing
                              coarse cell has the highest score (ties: lower template index); the
                              others' proposed cells are dropped.  0: no budget */
} srs_proposal_params;

/* The proposal search: the coarse search over coarse_mc, network scores of
 * all its cells; a cell scoring above the threshold (and, with suppression
 * on, highest within its window; with component_top > 0, among the
 * component_top highest coarse n_sigma of its group of adjacent
 * above-threshold cells) proposes the fine templates whose nearest
 * coarse template (in log Mc) is within fine_rows of it, at bins within one of
 * its bin; those fine cells are evaluated with srs_refine.  Outputs (host):
 * up to max_cells evaluated cells (cell_m, cell_b, cell_nsigma; *n_cells_out
 * = how many were evaluated, possibly more than max_cells), the top-k of them
 * in cands, and a report. */
srs_status srs_search_proposed(srs_ctx* ctx, const void* strain, int64_t n_samples, int32_t dtype,
                               const double* coarse_mc, int32_t n_coarse, const double* fine_mc,
                               int32_t n_fine, const srs_params* params, const float* mlp_params,
                               const srs_proposal_params* prop, int32_t max_cells, int32_t* cell_m,
                               int32_t* cell_b, float* cell_nsigma, int32_t* n_cells_out,
                               srs_candidate* cands, int32_t* n_cands, srs_proposal_report* report);

/* Size of the fixed device scratch used by srs_segment_spectra_static(). */
#define SRS_STATIC_SCRATCH_BYTES (16u << 20)

/* Segment spectra without allocating device memory.  The paper has no
 * counterpart: this is a service for callers that must not let a library
 * call cudaMalloc / cudaFree -- pipelines whose device memory is all handed
 * to their own allocator at start-up, and low-latency paths that cannot take
 * the stall or the device-wide synchronisation of allocating and freeing.
 *
 * It computes exactly what srs_segment_spectra() computes in the mixed form
 * (params->precision must be SRS_MIXED), with the same kernel, but the
 * kernel's scratch -- its tables, work queue and error flag, and the float32
 * copy of float64 strain -- lives in one fixed array of
 * SRS_STATIC_SCRATCH_BYTES that is part of the library and is held on every
 * GPU that loads the library until the process exits.  No context is used.
 *   cuda_stream  cudaStream_t to run on (NULL: the legacy default stream), on
 *                the current device
 *   strain       device pointer, [n_samples] of `dtype`
 *   mc           host, [n_templates] chirp masses at params->f_ref
 *   F            device pointer, [n_templates][seg_end-seg_begin][n_bins]
 *                complex double (re, im interleaved), caller-owned
 *   err_msg      optional host buffer of err_len bytes for a message
 * Returns SRS_ERR_ARG (with a message) when the request needs more scratch
 * than SRS_STATIC_SCRATCH_BYTES (many templates x segments, or many float64
 * segments: only [seg_begin, seg_end) is converted, 4 B per sample), when
 * strain or F is not device memory of the current device, or for any
 * argument srs_segment_spectra() would reject.  SRS_NO_TMA=1 selects the
 * same sample staging as in srs_segment_spectra().  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) for that device; make
 * that first call before any stream capture.  Every call reuses the same
 * array and clears what must start at zero; calls that overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller.  Synchronous with respect to the host. */
srs_status srs_segment_spectra_static(void* cuda_stream, const void* strain, int64_t n_samples,
                                      int32_t dtype, const double* mc, int32_t n_templates,
                                      int32_t seg_begin, int32_t seg_end, const srs_params* params,
                                      double* F, char* err_msg, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* SRS_H */
