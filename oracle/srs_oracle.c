/*
 * srs_oracle.c -- plain FP64 CPU oracle for the semicoherent NUFFT resampling
 * search (arXiv:2609.12476).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path: every quantity is
 * written out again here from the paper's equations.
 *
 * What it computes (all FP64, no approximation beyond libm rounding):
 *   - beta(f0, Mc)                         Sec. II, Eq. (beta)
 *   - 0PN duration f0 -> f_end             Sec. II (text above Eq. (beta))
 *   - 0PN frequency f(t)                   Sec. III.A, Eq. (f)
 *   - resampled time tau(t)                Sec. III.B, Eq. (new_t)
 *   - segment-local offset delta = tau(t) - tau(t_i0), written without the
 *     constant -(3/5)/beta so that no digits cancel (same equation, offset
 *     removed; a constant shift of tau changes only a per-bin phase)
 *   - the segment spectrum as the plain non-uniform DFT that a type-1 NUFFT
 *     approximates (Sec. III.B):  F(f_b) = sum_j x_j exp(-2 pi i f_b delta_j)
 * The power, semicoherent sum, n_sigma and top-k are done in numpy on top of
 * these spectra (oracle/__init__.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

/* Physical constants (SI / IAU nominal).  G*Msun = 1.32712440018e20 m^3 s^-2,
 * c = 299792458 m/s, so G*Msun/c^3 = 4.925490947...e-6 s. */
static const double ORC_GMSUN = 1.32712440018e20;
static const double ORC_C = 299792458.0;
static const double ORC_PI = 3.14159265358979323846264338327950288;

/* Sec. II, Eq. (beta): beta = (96/5) pi^(8/3) (G/c^3)^(5/3) Mc^(5/3) f0^(8/3),
 * with Mc in solar masses (G*Mc -> G*Msun*Mc), f0 in Hz; beta in 1/s. */
double orc_beta(double mc_msun, double f0) {
  double gm_c3 = ORC_GMSUN * mc_msun / (ORC_C * ORC_C * ORC_C);
  return (96.0 / 5.0) * pow(ORC_PI, 8.0 / 3.0) * pow(gm_c3, 5.0 / 3.0) * pow(f0, 8.0 / 3.0);
}

/* Sec. II: 0PN time to chirp from f0 to f_end,
 * t = 3/(8 beta) * (1 - (f0/f_end)^(8/3)). */
double orc_duration(double beta, double f0, double f_end) {
  return 3.0 / (8.0 * beta) * (1.0 - pow(f0 / f_end, 8.0 / 3.0));
}

/* Sec. III.A, Eq. (f): f(t) = f0 [1 - (8/3) beta (t - t0)]^(-3/8), t0 = 0. */
double orc_freq(double beta, double f0, double t) {
  return f0 * pow(1.0 - (8.0 / 3.0) * beta * t, -3.0 / 8.0);
}

/* Sec. III.B, Eq. (new_t), literally (t0 = 0):
 * tau(t) = -(3/5) [1 - (8/3) beta t]^(5/8) / beta. */
double orc_tau(double beta, double t) {
  return -(3.0 / 5.0) * pow(1.0 - (8.0 / 3.0) * beta * t, 5.0 / 8.0) / beta;
}

/* Segment-local resampled time delta(s) = tau(t_i0 + s) - tau(t_i0), Eq. (new_t)
 * with the common factor taken out:
 *   a = 1 - (8/3) beta t_i0,  x = (8/3) beta s / a,
 *   delta = (3 a^(5/8) / (5 beta)) * (1 - (1 - x)^(5/8))
 *         = (3 a^(5/8) / (5 beta)) * (-expm1((5/8) log1p(-x))).
 * Returns NAN when the sample lies at or past coalescence (1 - (8/3) beta t <= 0). */
double orc_delta(double beta, double t_i0, double s) {
  double a = 1.0 - (8.0 / 3.0) * beta * t_i0;
  double x = (8.0 / 3.0) * beta * s / a;
  if (!(a > 0.0) || !(x < 1.0)) return NAN;
  return (3.0 * pow(a, 5.0 / 8.0) / (5.0 * beta)) * (-expm1((5.0 / 8.0) * log1p(-x)));
}

/* Number of 30 s segments a template spends in band: the 0PN track that starts
 * at f_ref at t = 0 leaves the band at f_hi after orc_duration(beta, f_ref, f_hi)
 * (Sec. II); whole segments only (Sec. V counts 35 segments for 1060 s), at
 * least one, at most the number of segments in the data. */
int32_t orc_nseg(double beta, double f_ref, double f_hi, double t_coh, int32_t n_total, int cut) {
  if (!cut) return n_total;
  double t = orc_duration(beta, f_ref, f_hi);
  double k = floor(t / t_coh);
  if (k < 1.0) k = 1.0;
  if (k > (double)n_total) k = (double)n_total;
  return (int32_t)k;
}

/* The spectrum the type-1 NUFFT approximates (Sec. III.B), written as the plain
 * non-uniform DFT over the segment's samples:
 *   F(f_b) = sum_{j=0}^{n_s-1} x_j exp(-2 pi i f_b delta_j),  f_b = f_lo + b / t_coh,
 *   delta_j = delta(s_j) for s_j = j / fs, segment start t_i0.
 * The phase f_b * delta_j (cycles) is reduced to [0, 1) in FP64 before sin/cos. */
static void spectrum(const double* x, int64_t n_s, double fs, double beta, double t_i0,
                     double f_lo, double t_coh, int32_t n_b, double* re, double* im) {
  for (int32_t b = 0; b < n_b; ++b) { re[b] = 0.0; im[b] = 0.0; }
  for (int64_t j = 0; j < n_s; ++j) {
    double d = orc_delta(beta, t_i0, (double)j / fs);
    for (int32_t b = 0; b < n_b; ++b) {
      double fb = f_lo + (double)b / t_coh;
      double cyc = fb * d;
      cyc -= floor(cyc);
      double ang = 2.0 * ORC_PI * cyc;
      re[b] += x[j] * cos(ang);
      im[b] -= x[j] * sin(ang);
    }
  }
}

/* One job = one (template, segment) spectrum. */
typedef struct {
  const double* strain; int64_t n_s; double fs; double t_coh; double f_lo; int32_t n_b;
  const double* betas; const int32_t* item_m; const int32_t* item_i; int32_t n_items;
  double* out_re; double* out_im; int32_t next; pthread_mutex_t mu; int local;
} orc_job;

static void* worker(void* arg) {
  orc_job* J = (orc_job*)arg;
  for (;;) {
    pthread_mutex_lock(&J->mu);
    int32_t k = J->next++;
    pthread_mutex_unlock(&J->mu);
    if (k >= J->n_items) break;
    int32_t m = J->item_m[k], i = J->item_i[k];
    /* local: the 0PN template starts at the segment's own first sample (the
     * per-segment resampling of Sec. III.C's stack-slide), so t_i0 = 0 */
    double t_i0 = J->local ? 0.0 : (double)i * (double)J->n_s / J->fs;
    spectrum(J->strain + (int64_t)i * J->n_s, J->n_s, J->fs, J->betas[m], t_i0, J->f_lo,
             J->t_coh, J->n_b, J->out_re + (int64_t)k * J->n_b, J->out_im + (int64_t)k * J->n_b);
  }
  return NULL;
}

/* Spectra for a list of (template m, segment i) items; segment i covers samples
 * [i n_s, (i+1) n_s) of `strain`.  With local = 0 the template's track starts at
 * t = 0 (delta referenced to t_i0 = i T); with local = 1 each segment is
 * resampled with a 0PN template that starts at the segment's first sample.
 * Each item is computed by one thread start to finish, so the result does not
 * depend on n_threads.  Returns 0, or -1 on a bad argument. */
int orc_spectra_ex(const double* strain, int64_t n_samples, double fs, double t_coh, double f_lo,
                   int32_t n_b, const double* betas, const int32_t* item_m, const int32_t* item_i,
                   int32_t n_items, int n_threads, int local, double* out_re, double* out_im) {
  int64_t n_s = (int64_t)llround(t_coh * fs);
  if (n_s <= 0 || n_b <= 0 || n_items < 0 || n_threads <= 0) return -1;
  for (int32_t k = 0; k < n_items; ++k)
    if (item_i[k] < 0 || (int64_t)(item_i[k] + 1) * n_s > n_samples) return -1;
  orc_job J = {strain, n_s, fs, t_coh, f_lo, n_b, betas, item_m, item_i, n_items,
               out_re, out_im, 0, PTHREAD_MUTEX_INITIALIZER, local ? 1 : 0};
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < n_threads; ++t)
    if (pthread_create(&th[t], NULL, worker, &J) == 0) ++started;
  if (started == 0) worker(&J);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  return 0;
}

int orc_spectra(const double* strain, int64_t n_samples, double fs, double t_coh, double f_lo,
                int32_t n_b, const double* betas, const int32_t* item_m, const int32_t* item_i,
                int32_t n_items, int n_threads, double* out_re, double* out_im) {
  return orc_spectra_ex(strain, n_samples, fs, t_coh, f_lo, n_b, betas, item_m, item_i, n_items,
                        n_threads, 0, out_re, out_im);
}
