// srs_plan.cpp -- host planner of libsrs (FP64, no GPU).
//
// Sec. II Eq. (beta) and the 0PN duration give each template's resampling
// parameter and in-band segment count; Sec. III.B's type-1 NUFFT needs an
// oversampled grid, an exponential-of-semicircle (ES) spreading kernel and
// its Fourier-transform deconvolution factors.  The ES kernel and its width /
// shape rule follow Barnett, Magland & af Klinteberg (2019), the NUFFT the
// paper uses (its reference for FINUFFT).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>

#include "srs_internal.h"

namespace srs {
namespace {

constexpr double kPi = 3.14159265358979323846;
// G * Msun / c^3 [s] from the IAU nominal G*Msun and the defined speed of light.
constexpr double kGMsunC3 = 1.32712440018e20 / (299792458.0 * 299792458.0 * 299792458.0);


// Smallest 2^a 3^b 5^c >= n.
int32_t next_smooth(int32_t n) {
  for (int32_t m = std::max(n, 1);; ++m) {
    int32_t r = m;
    for (int p : {2, 3, 5})
      while (r % p == 0) r /= p;
    if (r == 1) return m;
  }
}

std::vector<int32_t> radix_plan(int32_t n) {
  std::vector<int32_t> r;
  int32_t m = n;
  while (m % 4 == 0) { r.push_back(4); m /= 4; }
  while (m % 2 == 0) { r.push_back(2); m /= 2; }
  while (m % 3 == 0) { r.push_back(3); m /= 3; }
  while (m % 5 == 0) { r.push_back(5); m /= 5; }
  return r;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_N).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
  x.assign(n, 0.0);
  wt.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // refresh p1, p0 at the converged node for the weight
        p0 = 1.0; p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Fourier transform of the ES kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on
// [-1, 1]:  phihat(xi) = int_{-1}^{1} phi(z) cos(xi z) dz, evaluated with z =
// sin(t) (t in [-pi/2, pi/2]) so the integrand is analytic, by Gauss-Legendre.
double es_hat(double beta, double xi, const std::vector<double>& gx, const std::vector<double>& gw) {
  double s = 0.0;
  for (size_t q = 0; q < gx.size(); ++q) {
    double t = 0.5 * kPi * gx[q];
    double c = std::cos(t);
    s += gw[q] * std::exp(beta * (c - 1.0)) * std::cos(xi * std::sin(t)) * c;
  }
  return 0.5 * kPi * s;
}

bool is_int(double v, double tol) { return std::fabs(v - std::round(v)) <= tol * std::max(1.0, std::fabs(v)); }

}  // namespace

// Eq. (beta): beta = (96/5) pi^(8/3) (G Mc / c^3)^(5/3) f^(8/3)  [1/s].
double chirp_beta(double mc, double f) {
  return 96.0 / 5.0 * std::pow(kPi, 8.0 / 3.0) * std::pow(kGMsunC3 * mc, 5.0 / 3.0) *
         std::pow(f, 8.0 / 3.0);
}

srs_status make_plan(const srs_params& p, const double* mc, int32_t n_templates, int64_t n_samples,
                     bool spectra_mode, int32_t seg_begin, int32_t seg_end, Plan& pl, std::string& msg,
                     const double* betas_in, bool local) {
  char buf[256];
  auto fail = [&](srs_status s, const char* m) { msg = m; return s; };
  if ((!mc && !betas_in) || n_templates <= 0) return fail(SRS_ERR_ARG, "need at least one template (mc != NULL)");
  if (local && !spectra_mode) return fail(SRS_ERR_ARG, "per-segment templates are a spectra-mode plan");
  if (!(p.fs > 0) || !(p.t_coh > 0)) return fail(SRS_ERR_ARG, "fs and t_coh must be positive");
  double ns_d = p.t_coh * p.fs;
  if (!is_int(ns_d, 1e-9) || ns_d < 1) return fail(SRS_ERR_ARG, "t_coh * fs must be a positive integer");
  double nb_d = (p.f_hi - p.f_lo) * p.t_coh;
  if (!(p.f_hi > p.f_lo) || !is_int(nb_d, 1e-9)) return fail(SRS_ERR_ARG, "(f_hi - f_lo) * t_coh must be a positive integer");
  if (p.f_hi > 0.5 * p.fs * (1 + 1e-12) || p.f_lo < -0.5 * p.fs * (1 + 1e-12))
    return fail(SRS_ERR_ARG, "band must lie within [-fs/2, fs/2]");
  if (!(p.eps >= 1e-12 && p.eps <= 1e-1)) return fail(SRS_ERR_ARG, "eps must be in [1e-12, 1e-1]");
  if (!(p.f_ref > 0)) return fail(SRS_ERR_ARG, "f_ref must be positive");
  if (p.precision != SRS_PLAIN_FP64 && p.precision != SRS_MIXED) return fail(SRS_ERR_ARG, "unknown precision");
  if (p.deterministic != 0 && p.deterministic != 1) return fail(SRS_ERR_ARG, "deterministic must be 0 or 1");
  if (p.sigma != 0 && !(p.sigma >= 1.2 && p.sigma <= 4.0)) return fail(SRS_ERR_ARG, "sigma must be 0 (auto) or in [1.2, 4]");
  if (p.chunk < 0) return fail(SRS_ERR_ARG, "chunk must be in [0, 16]");

  pl = Plan();
  pl.fs = p.fs; pl.t_coh = p.t_coh; pl.f_lo = p.f_lo; pl.f_hi = p.f_hi; pl.f_ref = p.f_ref; pl.eps = p.eps;
  pl.n_samples = n_samples;
  pl.n_s = (int64_t)std::llround(ns_d);
  pl.n_bins = (int32_t)std::llround(nb_d);
  pl.half_bins = pl.n_bins / 2;
  pl.f_c = p.f_lo + pl.half_bins / p.t_coh;
  pl.k_c = pl.f_c * p.t_coh;
  pl.precision = p.precision;
  pl.cut = p.cut_segments ? 1 : 0;
  pl.local = local;
  pl.n_templates = n_templates;
  if (n_samples < pl.n_s) return fail(SRS_ERR_ARG, "strain shorter than one segment");
  if (pl.n_s > (1 << 24)) return fail(SRS_ERR_UNSUPPORTED, "segments longer than 2^24 samples");
  pl.n_seg_total = (int32_t)std::min<int64_t>(n_samples / pl.n_s, INT32_MAX);
  if (!spectra_mode) {
    if (p.top_k < 1 || p.top_k > 1024) return fail(SRS_ERR_ARG, "top_k must be in [1, 1024]");
    if ((int64_t)n_templates * pl.n_bins > (int64_t)UINT32_MAX - 1) return fail(SRS_ERR_UNSUPPORTED, "statistic map too large");
  } else {
    if (seg_begin < 0 || seg_end <= seg_begin || seg_end > pl.n_seg_total)
      return fail(SRS_ERR_ARG, "need 0 <= seg_begin < seg_end <= segments in the strain");
  }
  pl.top_k = p.top_k;

  // Templates: beta_m (Eq. beta at f_ref) and in-band segments (Sec. II duration).
  pl.beta.resize(n_templates);
  pl.nseg.resize(n_templates);
  pl.n_spectra = 0;
  // Eq. (beta) with its Mc-independent factor taken once
  const double beta_scale = 96.0 / 5.0 * std::pow(kPi, 8.0 / 3.0) * std::pow(p.f_ref, 8.0 / 3.0);
  const double exit_frac = 1.0 - std::pow(p.f_ref / p.f_hi, 8.0 / 3.0);
  for (int32_t m = 0; m < n_templates; ++m) {
    double b;
    if (betas_in) {
      b = betas_in[m];
      if (!(b > 0) || !std::isfinite(b)) return fail(SRS_ERR_ARG, "chirp parameters beta must be positive and finite");
    } else {
      if (!(mc[m] > 0) || !std::isfinite(mc[m])) return fail(SRS_ERR_ARG, "chirp masses must be positive and finite");
      b = beta_scale * std::pow(kGMsunC3 * mc[m], 5.0 / 3.0);
    }
    pl.beta[m] = b;
    int32_t ns = pl.n_seg_total;
    if (pl.cut) {
      double t_exit = 3.0 / (8.0 * b) * exit_frac;
      double k = std::floor(t_exit / p.t_coh);
      ns = (int32_t)std::max(1.0, std::min(k, (double)pl.n_seg_total));
    }
    pl.nseg[m] = ns;
    int32_t last_seg = spectra_mode ? seg_end : ns;
    // the last sample's time on the template's own clock (segment-local: within one segment)
    double t_last = ((double)(local ? 1 : last_seg) * (double)pl.n_s - 1.0) / p.fs;
    if (!(1.0 - 8.0 / 3.0 * b * t_last > 0.0)) {
      std::snprintf(buf, sizeof buf, "template %d reaches coalescence inside its segments (Sec. II: 1 - 8/3 beta t <= 0)", m);
      msg = buf;
      return SRS_ERR_DOMAIN;
    }
    pl.n_spectra += spectra_mode ? (seg_end - seg_begin) : ns;
  }
  // work items, their first-segment rows and the kernels' item indices are
  // 32-bit: one call covers at most 2^31 - 1 segment spectra
  if (pl.n_spectra > (int64_t)INT32_MAX)
    return fail(SRS_ERR_UNSUPPORTED, "more than 2^31 - 1 segment spectra in one call; split the template list");

  // ES kernel width and shape from eps (Barnett et al. 2019): with
  // oversampling sigma the aliasing error falls like exp(-pi w sqrt(1 - 1/sigma));
  // for sigma = 2 the rule is w = ceil(log10(1/eps)) + 1, beta = 2.30 w; otherwise
  // w = ceil(ln(1/eps) / (pi sqrt(1 - 1/sigma))), beta = 0.97 pi (1 - 1/(2 sigma)) w.
  auto es_params = [&](double sigma, int32_t& w, double& beta_es) {
    if (std::fabs(sigma - 2.0) < 1e-12) {
      w = (int32_t)std::ceil(std::log10(1.0 / p.eps) - 1e-12) + 1;
      beta_es = 2.30 * w;
    } else {
      w = (int32_t)std::ceil(std::log(1.0 / p.eps) / (kPi * std::sqrt(1.0 - 1.0 / sigma)) - 1e-12);
      beta_es = 0.97 * kPi * (1.0 - 0.5 / sigma) * w;
    }
    w = std::max(w, 2);
  };
  const size_t smem_cap = 200 * 1024;
  if (p.precision == SRS_MIXED) {
    // FP32 samples, phases and grid leave a floor of about 1.2e-6 relative L2
    // error per spectrum, so 10 eps must stay above it
    if (p.eps < kMixedMinEps)
      return fail(SRS_ERR_UNSUPPORTED, "the mixed (FP32) form needs eps >= 2e-7; use SRS_PLAIN_FP64");
    pl.sigma = p.sigma > 0 ? p.sigma : 2.0;
    es_params(pl.sigma, pl.w, pl.beta_es);
    if (pl.w > kMixedMaxW) return fail(SRS_ERR_UNSUPPORTED, "kernel width above the mixed form's maximum (raise eps or sigma)");
    pl.n_fine = next_smooth(std::max((int32_t)std::ceil(pl.sigma * pl.n_bins - 1e-9), 2 * pl.w));
    // shared memory of the mixed spreader: staged samples + grid + FFT scratch
    // (none for the in-place 1200-point FFT; counted here for any size) + Z
    // + anchors of one item (at most 16 segments)
    size_t need = (size_t)pl.n_s * 4 + (size_t)pl.n_fine * 16 + (size_t)pl.n_bins * 4 + 16 * 8 * sizeof(Anchor) + 1024;
    if (need > smem_cap) return fail(SRS_ERR_UNSUPPORTED, "segment too long or band too wide for the mixed form's shared memory");
  } else {
    const double sig_try[3] = {2.0, 1.5, 1.25};
    bool ok = false;
    for (double s : sig_try) {
      if (p.sigma > 0 && std::fabs(s - p.sigma) > 1e-12) continue;
      int32_t w; double be;
      es_params(s, w, be);
      int32_t n = next_smooth(std::max((int32_t)std::ceil(s * pl.n_bins - 1e-9), 2 * w));
      if ((size_t)n * 32 + 1024 <= smem_cap && w <= kPlainMaxW) {
        pl.sigma = s; pl.w = w; pl.beta_es = be; pl.n_fine = n; ok = true;
        break;
      }
    }
    if (!ok && p.sigma > 0) {
      es_params(p.sigma, pl.w, pl.beta_es);
      pl.sigma = p.sigma;
      pl.n_fine = next_smooth(std::max((int32_t)std::ceil(p.sigma * pl.n_bins - 1e-9), 2 * pl.w));
      ok = (size_t)pl.n_fine * 32 + 1024 <= smem_cap && pl.w <= kPlainMaxW;
    }
    if (!ok) return fail(SRS_ERR_UNSUPPORTED, "band too wide for the FP64 form's shared-memory FFT");
  }
  pl.sigma = (double)pl.n_fine / pl.n_bins;
  pl.radices = radix_plan(pl.n_fine);

  // Mixed form: run of samples per thread, one FP64 anchor per warp span.
  set_cta(pl, kSpreadThreads);
  if (p.precision == SRS_MIXED) {
    // Local degree-5 expansion over one span must be accurate to 1e-9 cycles at
    // the band edge: bound the first omitted term, coef_6 beta^5 A^(-43/8) / 6!
    // (d^6 delta / ds^6 / 6!), at the smallest A = 1 - 8/3 beta t of any segment.
    // Checked for 256-thread CTAs (required) and for 128-thread CTAs, whose
    // runs are twice as long: with an anchor per warp if that holds, else with
    // an anchor per half-warp (the 256-thread span again); 128-thread CTAs are
    // allowed if either holds.
    double fmax = std::max(std::fabs(p.f_lo), std::fabs(p.f_hi));
    const double ds_half = 32.0 * (double)run_for(pl.n_s, 128) / p.fs;
    const double ds_quarter = 16.0 * (double)run_for(pl.n_s, 128) / p.fs;
    const double ds = pl.span / p.fs;
    // d^6 delta / ds^6 / 6! = coef_6 beta^5 A^(-43/8) / 720 and d^2 delta / ds^2 / 2 = beta A^(-11/8) / 2,
    // through logarithms (one log of beta and of A per template)
    const double c6 = 2438.3333333333333 / 720.0;
    const double lim6_half = 1e-9 / (std::pow(ds_half, 6) * fmax), lim2_half = 0.25 * p.t_coh / (ds_half * ds_half);
    const double lim6 = 1e-9 / (std::pow(ds, 6) * fmax), lim2 = 0.25 * p.t_coh / (ds * ds);
    const double lim6_q = 1e-9 / (std::pow(ds_quarter, 6) * fmax), lim2_q = 0.25 * p.t_coh / (ds_quarter * ds_quarter);
    bool warp_anchor_128 = true;
    pl.allow_128 = true;
    for (int32_t m = 0; m < n_templates; ++m) {
      int32_t last_seg = local ? 1 : (spectra_mode ? seg_end : pl.nseg[m]);
      double A = 1.0 - 8.0 / 3.0 * pl.beta[m] * (((double)last_seg * pl.n_s) / p.fs);
      A = std::max(A, 1e-300);
      const double lb = std::log(pl.beta[m]), la = std::log(A);
      const double e6 = c6 * std::exp(5.0 * lb - 43.0 / 8.0 * la);
      const double e2 = 0.5 * std::exp(lb - 11.0 / 8.0 * la);
      if (e6 > lim6_half || e2 > lim2_half) warp_anchor_128 = false;
      if (e6 > lim6_q || e2 > lim2_q) pl.allow_128 = false;
      if (e6 > lim6 || e2 > lim2) {
        std::snprintf(buf, sizeof buf, "template %d chirps too fast for the mixed form's anchor spacing; use SRS_PLAIN_FP64", m);
        msg = buf;
        return SRS_ERR_UNSUPPORTED;
      }
    }
    pl.lanes128 = warp_anchor_128 ? 32 : 16;
  }

  // Deconvolution: with fine grid spacing h = 2 pi / n and kernel half-width
  // alpha = w h / 2, sum_l psi(l h - x) exp(-i k l h) ~= exp(-i k x) alpha phihat(k alpha) / h,
  // so F_k = G_k * (2 / w) / phihat(k pi w / n).
  // The tables depend on (beta_ES, w, n_fine, n_bins) only; the last few are
  // kept, so that re-planning a template list costs no quadrature.
  {
    struct Tables {
      double beta_es;
      int32_t w, n_fine, n_bins;
      std::vector<double> corr, tw_re, tw_im;
    };
    static std::mutex mu;
    static std::vector<Tables> cache;
    std::lock_guard<std::mutex> lock(mu);
    const Tables* hit = nullptr;
    for (const Tables& t : cache)
      if (t.beta_es == pl.beta_es && t.w == pl.w && t.n_fine == pl.n_fine && t.n_bins == pl.n_bins) hit = &t;
    if (!hit) {
      Tables t;
      t.beta_es = pl.beta_es;
      t.w = pl.w;
      t.n_fine = pl.n_fine;
      t.n_bins = pl.n_bins;
      std::vector<double> gx, gw;
      gauss_legendre(128, gx, gw);
      t.corr.resize(pl.n_bins);
      for (int32_t b = 0; b < pl.n_bins; ++b) {
        double k = (double)(b - pl.half_bins);
        double ph = es_hat(pl.beta_es, k * kPi * pl.w / pl.n_fine, gx, gw);
        t.corr[b] = (2.0 / pl.w) / ph;
      }
      t.tw_re.resize(pl.n_fine);
      t.tw_im.resize(pl.n_fine);
      for (int32_t m = 0; m < pl.n_fine; ++m) {
        double a = -2.0 * kPi * (double)m / pl.n_fine;
        t.tw_re[m] = std::cos(a);
        t.tw_im[m] = std::sin(a);
      }
      if (cache.size() >= 8) cache.erase(cache.begin());
      cache.push_back(std::move(t));
      hit = &cache.back();
    }
    pl.corr = hit->corr;
    pl.tw_re = hit->tw_re;
    pl.tw_im = hit->tw_im;
  }

  // Default chunk: enough items to keep ~8 per resident CTA of a 152-SM part.
  if (p.chunk > 16) return fail(SRS_ERR_ARG, "chunk must be in [0, 16]");
  int32_t chunk = p.chunk;
  if (chunk == 0) {
    int64_t per = pl.n_spectra / (8 * 152 * 4);
    chunk = (int32_t)std::max<int64_t>(1, std::min<int64_t>(16, per));
  }
  make_items(pl, chunk, spectra_mode, seg_begin, seg_end);
  return SRS_OK;
}

void make_items(Plan& pl, int32_t chunk, bool spectra_mode, int32_t seg_begin, int32_t seg_end,
                int32_t tail_singles) {
  pl.chunk = chunk;
  pl.items.clear();
  pl.order.clear();
  pl.item_off.assign(pl.n_templates + 1, 0);
  const bool tail = !spectra_mode && chunk > 1 && tail_singles > 0 && pl.n_spectra > 0;
  std::vector<int32_t> singles;
  int64_t g = 0;
  for (int32_t m = 0; m < pl.n_templates; ++m) {
    pl.item_off[m] = (int32_t)pl.items.size();
    int32_t a = spectra_mode ? seg_begin : 0;
    int32_t e = spectra_mode ? seg_end : pl.nseg[m];
    int32_t e_multi = e;
    if (tail) {
      const int64_t s_m = ((int64_t)(e - a) * tail_singles + pl.n_spectra - 1) / pl.n_spectra;
      e_multi = e - (int32_t)std::min<int64_t>(s_m, e - a);
    }
    for (int32_t i = a; i < e; ) {
      Item it;
      it.m = m;
      it.i0 = i;
      it.i1 = i < e_multi ? std::min(e_multi, i + chunk) : i + 1;
      it.g0 = (int32_t)g;
      g += it.i1 - it.i0;
      if (tail && i >= e_multi) singles.push_back((int32_t)pl.items.size());
      else if (tail) pl.order.push_back((int32_t)pl.items.size());
      pl.items.push_back(it);
      i = it.i1;
    }
  }
  pl.item_off[pl.n_templates] = (int32_t)pl.items.size();
  if (tail) pl.order.insert(pl.order.end(), singles.begin(), singles.end());
}

int32_t run_for(int64_t n_s, int32_t threads) {
  // samples per thread, odd: lane l reads xs[l run + m], so an odd run puts
  // the 32 lanes of a warp on 32 different shared-memory banks
  int32_t run = (int32_t)((n_s + threads - 1) / threads);
  return run | 1;
}

void set_cta(Plan& pl, int32_t threads) {
  pl.threads = threads;
  pl.run = run_for(pl.n_s, threads);
  pl.span = (threads == 128 ? pl.lanes128 : 32) * pl.run;
  pl.n_anchor = (int32_t)((pl.n_s + pl.span - 1) / pl.span);
}

void fill_info(const Plan& pl, srs_plan_info* info) {
  if (!info) return;
  info->n_s = pl.n_s;
  info->n_seg_total = pl.n_seg_total;
  info->n_bins = pl.n_bins;
  info->n_fine = pl.n_fine;
  info->w = pl.w;
  info->beta_es = pl.beta_es;
  info->sigma = pl.sigma;
  info->n_spectra = pl.n_spectra;
  info->chunk = pl.chunk;
  info->n_items = (int32_t)pl.items.size();
}

}  // namespace srs

namespace srs {

float mixed_es_e(const Plan& pl) { return (float)(pl.beta_es * 1.4426950408889634074); }

std::vector<float> mixed_corr(const Plan& pl) {
  // the spreader's taps are 2^(E sqrt(1 - z^2)), the ES kernel times 2^E
  const double scale = std::exp2(-(double)mixed_es_e(pl));
  std::vector<float> c(pl.corr.size());
  for (size_t b = 0; b < c.size(); ++b) c[b] = (float)(pl.corr[b] * scale);
  return c;
}

}  // namespace srs
