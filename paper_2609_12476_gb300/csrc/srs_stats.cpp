// srs_stats.cpp -- detection statistics of the semicoherent search (host only):
// the n_sigma threshold at a false-alarm probability (Sec. III.C Eq.
// n_sigma^th) and the total non-centrality a signal needs to be detected
// (Eq. non-centrality_threshold).
//
// Under H0 each normalised power P_i is chi^2 with 2 degrees of freedom, so
// (P_i - 2)/2 = E_i - 1 with E_i ~ Exp(1), and for weights w (sum w^2 = 1)
//   n_sigma = sum_i w_i E_i - sum_i w_i.
// Equal weights: sum E_i ~ Gamma(N, 1), whose survival function for a whole
// number N is the Poisson sum Q(N, x) = e^-x sum_{k<N} x^k / k!.  Unequal
// weights: a sum of exponentials with different scales, whose survival
// function is the mixture of Gamma(N + k) survival functions of Moschopoulos
// (1985): with b = min w_i, C = prod (b / w_i),
//   gamma_k = sum_i (1 - b / w_i)^k / k,  delta_0 = 1,
//   delta_{k+1} = 1/(k+1) sum_{j=1}^{k+1} j gamma_j delta_{k+1-j},
//   P(sum w_i E_i > q) = C sum_k delta_k Q(N + k, q / b),
// every term positive.  The mixture weights C delta_k are carried as scaled
// deltas with C in logs (see ExpMixture).
// With a signal, P_i is non-central chi^2 (2 dof, non-centrality lambda_i);
// for equal weights sum P_i is non-central chi^2 with 2N dof and total
// non-centrality Lambda, a Poisson(Lambda/2) mixture of central chi^2 with
// 2(N + j) dof.  For unequal weights the signal's share of segment i is
// lambda_i = Lambda w_i / sum w (the weights follow A_i^2 / S_i, the signal
// power per segment), and P(sum_i w_i P_i > x) is evaluated by Imhof's
// (1961) inversion of the characteristic function:
//   P(Q > x) = 1/2 + (1/pi) int_0^inf sin(theta(u)) / (u rho(u)) du,
//   theta(u) = sum_i [arctan(w_i u) + lambda_i w_i u / (1 + w_i^2 u^2)] - x u / 2,
//   rho(u)   = prod_i (1 + w_i^2 u^2)^(1/2) exp(sum_i lambda_i w_i^2 u^2 / (2 (1 + w_i^2 u^2))),
// accurate at the detection probabilities asked for here (not at 1e-6 tails,
// where the threshold comes from the exact central mixture).  Weights that
// are all equal take the exact equal-weight route.  The ROC of one signal
// (Fig. roc: p_det against p_fa) is the same probability at the thresholds of
// a list of p_fa, with the per-segment non-centralities lambda_i given.
#include <cmath>
#include <vector>

#include "../../include/srs.h"

namespace {

using ld = long double;

// Q(m, x) for m = m0, m0 + 1, ..., m0 + count - 1 (whole m >= 1): the upper
// regularized incomplete gamma function, by Q(m + 1, x) = Q(m, x) + p(m, x)
// with the Poisson term p(m, x) = e^-x x^m / m!, in logs.
void gamma_q_run(int64_t m0, int64_t count, ld x, std::vector<ld>& out) {
  out.assign((size_t)count, 0.0L);
  if (x <= 0) {
    for (auto& v : out) v = 1.0L;
    return;
  }
  const ld lx = std::log(x);
  // Q(m0, x) = sum_{k < m0} p(k, x): add from the largest term outwards
  const int64_t kmax = m0 - 1;
  const int64_t kpk = std::min<int64_t>(kmax, (int64_t)std::floor(x));
  auto logp = [&](int64_t k) { return -x + (ld)k * lx - std::lgamma((ld)k + 1.0L); };
  const ld lref = logp(kpk);
  ld s = 0;
  for (int64_t k = kpk; k >= 0; --k) {
    const ld t = std::exp(logp(k) - lref);
    s += t;
    if (t < 1e-22L * s) break;
  }
  for (int64_t k = kpk + 1; k <= kmax; ++k) {
    const ld t = std::exp(logp(k) - lref);
    s += t;
    if (t < 1e-22L * s) break;
  }
  ld q = s * std::exp(lref);
  for (int64_t c = 0; c < count; ++c) {
    out[(size_t)c] = std::min<ld>(q, 1.0L);
    q += std::exp(logp(m0 + c));
  }
}

// The law of sum_i w_i E_i for positive weights as a mixture of Gamma(N + k,
// scale b) laws: mixture weights d_k = C delta_k (Moschopoulos 1985), built
// once; sf(q) = sum_k d_k Q(N + k, q / b).  C = prod (b / w_i) leaves every
// floating-point range on long tracks with spread weights (e^-17500 for a
// 26-day 0PN track over 40-60 Hz), so the recurrence runs on
// deltas scaled by e^shift, rescaled whenever they grow past 1e250, and C
// enters in logs: d_k = exp(logC - shift) delta_hat_k.
struct ExpMixture {
  int64_t n = 0;
  ld b = 1;
  std::vector<double> dh;   // delta_k e^shift
  double log_factor = 0;    // logC - shift: d_k = exp(log_factor) dh_k
  bool converged = false;   // the terms left out are negligible (false: kcap was reached first)

  ExpMixture(const std::vector<ld>& w, int64_t kcap) {
    n = (int64_t)w.size();
    b = w[0];
    for (ld v : w) b = std::min(b, v);
    double logC = 0;
    std::vector<double> r(w.size()), rk(w.size(), 1.0);
    for (size_t i = 0; i < w.size(); ++i) {
      logC += (double)std::log(b / w[i]);
      r[i] = (double)(1.0L - b / w[i]);
    }
    double shift = 0;                 // dh_k = delta_k e^shift
    dh.push_back(1.0);
    std::vector<double> gam(1, 0.0);
    double sum_dh = 1.0, peak = 1.0;
    auto total = [&]() { return std::exp(logC - shift + std::log(sum_dh)); };
    for (int64_t k = 1; k <= kcap; ++k) {
      double g = 0;
      for (size_t i = 0; i < w.size(); ++i) {
        rk[i] *= r[i];
        g += rk[i];
      }
      gam.push_back(g / (double)k);
      double dk = 0;
      for (int64_t j = 1; j <= k; ++j) dk += (double)j * gam[(size_t)j] * dh[(size_t)(k - j)];
      dk /= (double)k;
      dh.push_back(dk);
      sum_dh += dk;
      peak = std::max(peak, dk);
      if (peak > 1e250) {             // rescale the stored deltas
        for (double& v : dh) v *= 1e-250;
        sum_dh *= 1e-250;
        peak *= 1e-250;
        shift -= 250.0 * std::log(10.0);
      }
      if (dk < 1e-30 * peak && dk < dh[(size_t)(k - 1)] && total() > 0.5) {   // past the mode, negligible
        converged = true;
        break;
      }
    }
    log_factor = logC - shift;
  }

  ld sf(ld q) const {
    std::vector<ld> Q;
    gamma_q_run(n, (int64_t)dh.size(), q / b, Q);
    ld s = 0;
    for (size_t k = 0; k < dh.size(); ++k) s += (ld)dh[k] * Q[k];
    if (!(s > 0)) return 0.0L;
    return std::min<ld>(std::exp((ld)log_factor + std::log(s)), 1.0L);
  }
};

// P(chi^2_{2N}(Lambda) > x): Poisson(Lambda / 2) mixture of Q(N + j, x / 2).
ld noncentral_sf(int64_t n, ld lambda, ld x) {
  const ld mu = lambda / 2;
  const int64_t jpk = (int64_t)std::floor(mu);
  const int64_t span = (int64_t)(12.0L * std::sqrt(mu + 1.0L)) + 30;
  const int64_t j0 = std::max<int64_t>(0, jpk - span), j1 = jpk + span;
  std::vector<ld> Q;
  gamma_q_run(n + j0, j1 - j0 + 1, x / 2, Q);
  ld s = 0;
  for (int64_t j = j0; j <= j1; ++j) {
    const ld lp = mu > 0 ? -mu + (ld)j * std::log(mu) - std::lgamma((ld)j + 1.0L) : (j == 0 ? 0.0L : -INFINITY);
    s += std::exp(lp) * Q[(size_t)(j - j0)];
  }
  return std::min<ld>(s, 1.0L);
}

// P(sum_i w_i P_i > x) with P_i ~ chi^2_2(lam_i), by Imhof's integral over
// [0, U]: 15-point Gauss-Legendre panels half a period of the integrand's
// fastest oscillation wide, and U where the tail bound
// int_U^inf du / (u rho(u)) <= 1 / (n U^n prod w_i) drops below `tail`.
struct Imhof {
  const std::vector<double>& w;
  const std::vector<double>& lam;
  double x;
  double tail = 1e-9;

  double integrand(double u) const {
    if (u <= 0) {
      // u -> 0: theta(u) / u -> sum (w + lam w / 2) - x / 2, rho -> 1
      double s = 0;
      for (size_t i = 0; i < w.size(); ++i) s += w[i] * (1.0 + 0.5 * lam[i]);
      return s - 0.5 * x;
    }
    double th = -0.5 * x * u, lr = 0;
    for (size_t i = 0; i < w.size(); ++i) {
      const double wu = w[i] * u, d = 1.0 + wu * wu;
      th += std::atan(wu) + 0.5 * lam[i] * wu / d;
      lr += 0.5 * std::log(d) + 0.5 * lam[i] * wu * wu / d;
    }
    if (lr > 700) return 0.0;
    return std::sin(th) / (u * std::exp(lr));
  }
  double sf() const {
    static const double gx[8] = {0.0, 0.201194093997434522, 0.394151347077563370, 0.570972172608538848,
                                 0.724417731360170047, 0.848206583410427216, 0.937273392400705904,
                                 0.987992518020485428};
    static const double gw[8] = {0.202578241925561273, 0.198431485327111576, 0.186161000015562211,
                                 0.166269205816993934, 0.139570677926154314, 0.107159220467171935,
                                 0.070366047488108125, 0.030753241996117268};
    const double n = (double)w.size();
    double lw = 0;
    for (double v : w) lw += std::log(v);
    const double U = std::max(1.0, std::exp((-std::log(n * tail) - lw) / n));
    const double kPi = 3.14159265358979323846;
    // theta'(u) is at most x / 2 + sum w_i (1 + lambda_i / 2) in magnitude:
    // panels of half its period
    double rate = 0.5 * x;
    for (size_t i = 0; i < w.size(); ++i) rate += w[i] * (1.0 + 0.5 * lam[i]);
    const double width = std::min(kPi / std::max(rate, 1e-3), U);
    const long long panels = std::min<long long>(20000000, (long long)std::ceil(U / width));
    const double h = U / (double)panels;
    double acc = 0;
    for (long long k = 0; k < panels; ++k) {
      const double c = (k + 0.5) * h, r = 0.5 * h;
      double pv = gw[0] * integrand(c);
      for (int j = 1; j < 8; ++j) pv += gw[j] * (integrand(c - r * gx[j]) + integrand(c + r * gx[j]));
      acc += pv * r;
    }
    return 0.5 + acc / kPi;
  }
};

// The q >= 0 with sf(q) = p for a decreasing sf with sf(0) = 1 (the law of
// a sum of non-negative terms), by bisection on log sf; [lo, hi] is a first
// bracket, widened as needed.
template <typename F>
ld invert_sf(F sf, ld lo, ld hi, ld p) {
  if (sf(lo) <= p) {
    hi = lo;
    lo = 0;
  } else {
    while (sf(hi) > p) {
      const ld d = hi - lo;
      lo = hi;
      hi += 2 * d;
    }
  }
  const ld lp = std::log(p);
  for (int it = 0; it < 200; ++it) {
    const ld mid = 0.5L * (lo + hi);
    const ld v = sf(mid);
    if ((v > 0 ? std::log(v) : -INFINITY) > lp) lo = mid; else hi = mid;
    if (hi - lo <= 1e-15L * hi) break;
  }
  return 0.5L * (lo + hi);
}

// Weights normalised to sum w^2 = 1 (w NULL: equal weights).  False when a
// weight is not positive and finite; *unequal says whether any two differ.
bool unit_weights(const double* w, int32_t n, std::vector<double>& ww, bool* unequal) {
  ww.assign((size_t)n, 1.0 / std::sqrt((double)n));
  *unequal = false;
  if (!w) return true;
  double s2 = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (!(w[i] > 0) || !std::isfinite(w[i])) return false;
    s2 += w[i] * w[i];
    if (std::fabs(w[i] - w[0]) > 1e-12 * std::fabs(w[0])) *unequal = true;
  }
  for (int32_t i = 0; i < n; ++i) ww[(size_t)i] = w[i] / std::sqrt(s2);
  return true;
}

// Equal weights: the threshold on S = sum P (chi^2 with 2N dof under H0) and
// its exact false-alarm probability.
ld sum_threshold(int64_t n, double p_fa, ld* sf_at) {
  auto sf0 = [&](ld s) {
    std::vector<ld> Q;
    gamma_q_run(n, 1, s / 2, Q);
    return Q[0];
  };
  const ld s_th = invert_sf(sf0, 2.0L * n, 2.0L * n + 10.0L * std::sqrt((ld)n), (ld)p_fa);
  if (sf_at) *sf_at = sf0(s_th);
  return s_th;
}

}  // namespace

extern "C" {

srs_status srs_nsigma_threshold(const double* w, int32_t n_seg, double p_fa, double* n_sigma_th) {
  if (!n_sigma_th || n_seg < 1 || n_seg > 10000000 || !(p_fa > 0 && p_fa < 1)) return SRS_ERR_ARG;
  std::vector<ld> ww((size_t)n_seg, 1.0L);
  if (w) {
    ld s2 = 0;
    for (int32_t i = 0; i < n_seg; ++i) {
      if (!(w[i] > 0) || !std::isfinite(w[i])) return SRS_ERR_ARG;
      ww[(size_t)i] = w[i];
      s2 += (ld)w[i] * w[i];
    }
    const ld inv = 1.0L / std::sqrt(s2);
    for (auto& v : ww) v *= inv;
  } else {
    for (auto& v : ww) v = 1.0L / std::sqrt((ld)n_seg);
  }
  ld sum_w = 0, b = ww[0];
  for (ld v : ww) {
    sum_w += v;
    b = std::min(b, v);
  }
  const ld mean = sum_w;   // E[sum w E] = sum w; its variance is sum w^2 = 1
  // The mixture index K is a sum of independent negative binomials with
  // success probabilities b / w_i: mean sum (w_i / b - 1), variance
  // sum (w_i / b)(w_i / b - 1).  Building K terms costs about K^2 + K n;
  // Imhof's integral costs about n times its panel count per evaluation.
  // Weights spread so widely that the mixture costs more take the integral.
  const ld n = (ld)n_seg;
  ld km = 0, kv = 0, lw = 0;
  for (ld v : ww) {
    km += v / b - 1;
    kv += (v / b) * (v / b - 1);
    lw += std::log(v);
  }
  const ld k_need = km + 12.0L * std::sqrt(kv) + 100.0L;
  const ld U = std::max(1.0L, std::exp((-std::log(n * 1e-14L) - lw) / n));
  const ld x_typ = 2.0L * (mean + 5.0L);
  const ld panels = std::max(1.0L, U * x_typ / (2.0L * 3.14159265358979323846L));
  const ld cost_mix = k_need * k_need + k_need * n;
  const ld cost_imhof = 60.0L * 15.0L * 10.0L * panels * n;   // evaluations x nodes x (atan, log) per weight
  if (std::min(cost_mix, cost_imhof) > 1e12L) return SRS_ERR_UNSUPPORTED;   // many minutes either way
  if (cost_mix <= cost_imhof) {
    const ExpMixture mix(ww, (int64_t)std::min<ld>(2.0L * k_need + 1000.0L, 5e7L));
    if (mix.converged) {
      auto sf = [&](ld q) { return mix.sf(q); };
      const ld q = invert_sf(sf, mean, mean + 10.0L, (ld)p_fa);
      *n_sigma_th = (double)(q - sum_w);
      return SRS_OK;
    }
  }
  if (cost_imhof > 1e12L) return SRS_ERR_UNSUPPORTED;   // the mixture did not converge either
  // sum w E > q  <=>  sum w P > 2 q with P = 2 E ~ chi^2_2
  std::vector<double> wd(ww.begin(), ww.end()), zero(ww.size(), 0.0);
  auto sf = [&](ld q) {
    Imhof im{wd, zero, (double)(2.0L * q)};
    im.tail = 1e-14;
    return (ld)std::max(0.0, im.sf());
  };
  const ld q = invert_sf(sf, mean, mean + 10.0L, (ld)p_fa);
  *n_sigma_th = (double)(q - sum_w);
  return SRS_OK;
}

srs_status srs_detection_noncentrality(const double* w, int32_t n_seg, double p_fa, double p_det, double* lambda) {
  if (!lambda || n_seg < 1 || n_seg > 10000000 || !(p_fa > 0 && p_fa < 1) || !(p_det > 0 && p_det < 1))
    return SRS_ERR_ARG;
  bool unequal = false;
  std::vector<double> ww;
  if (!unit_weights(w, n_seg, ww, &unequal)) return SRS_ERR_ARG;
  if (unequal) {
    // unequal weights: the threshold on n_sigma from the exact central law,
    // then Lambda from Imhof's integral with lambda_i = Lambda w_i / sum w
    double s1 = 0;
    for (double v : ww) s1 += v;
    double th = 0;
    srs_status s = srs_nsigma_threshold(ww.data(), n_seg, p_fa, &th);
    if (s != SRS_OK) return s;
    // n_sigma = sum w (P - 2) / 2 > th  <=>  Q = sum w P > 2 th + 2 sum w
    const double x = 2.0 * th + 2.0 * s1;
    std::vector<double> lam((size_t)n_seg, 0.0);
    auto pdet = [&](double L) {
      for (int32_t i = 0; i < n_seg; ++i) lam[(size_t)i] = L * ww[(size_t)i] / s1;
      return Imhof{ww, lam, x}.sf();
    };
    if (pdet(0.0) >= p_det) {
      *lambda = 0.0;
      return SRS_OK;
    }
    double lo = 0, hi = 1;
    while (pdet(hi) < p_det) hi *= 2;
    for (int it = 0; it < 100; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (pdet(mid) < p_det) lo = mid; else hi = mid;
      if (hi - lo <= 1e-10 * hi) break;
    }
    *lambda = 0.5 * (lo + hi);
    return SRS_OK;
  }
  const int64_t n = n_seg;
  ld sf_th = 0;
  const ld s_th = sum_threshold(n, p_fa, &sf_th);
  if ((ld)p_det <= sf_th) {
    *lambda = 0.0;
    return SRS_OK;
  }
  // the Lambda with P(S > s_th | Lambda) = p_det: increasing in Lambda
  ld lo = 0, hi = 1;
  while (noncentral_sf(n, hi, s_th) < p_det) hi *= 2;
  for (int it = 0; it < 200; ++it) {
    const ld mid = 0.5L * (lo + hi);
    if (noncentral_sf(n, mid, s_th) < p_det) lo = mid; else hi = mid;
    if (hi - lo <= 1e-13L * hi) break;
  }
  *lambda = (double)(0.5L * (lo + hi));
  return SRS_OK;
}

srs_status srs_detection_probability(const double* w, const double* lambda, int32_t n_seg, const double* p_fa,
                                     int32_t n_points, double* p_det) {
  if (!p_fa || !p_det || n_seg < 1 || n_seg > 10000000 || n_points < 1) return SRS_ERR_ARG;
  for (int32_t q = 0; q < n_points; ++q)
    if (!(p_fa[q] > 0 && p_fa[q] < 1)) return SRS_ERR_ARG;
  std::vector<double> ww, lam((size_t)n_seg, 0.0);
  bool unequal = false;
  if (!unit_weights(w, n_seg, ww, &unequal)) return SRS_ERR_ARG;
  double total = 0;
  if (lambda) {
    for (int32_t i = 0; i < n_seg; ++i) {
      if (!(lambda[i] >= 0) || !std::isfinite(lambda[i])) return SRS_ERR_ARG;
      lam[(size_t)i] = lambda[i];
      total += lambda[i];
    }
  }
  for (int32_t q = 0; q < n_points; ++q) {
    if (!unequal) {
      // sum P is non-central chi^2 with 2N dof and non-centrality sum lambda_i
      ld sf_th = 0;
      const ld s_th = sum_threshold(n_seg, p_fa[q], &sf_th);
      p_det[q] = (double)(total > 0 ? noncentral_sf(n_seg, (ld)total, s_th) : sf_th);
      continue;
    }
    double th = 0;
    const srs_status s = srs_nsigma_threshold(ww.data(), n_seg, p_fa[q], &th);
    if (s != SRS_OK) return s;
    double s1 = 0;
    for (double v : ww) s1 += v;
    // n_sigma = sum w (P - 2) / 2 > th  <=>  sum w P > 2 th + 2 sum w
    const double v = Imhof{ww, lam, 2.0 * th + 2.0 * s1}.sf();
    p_det[q] = std::min(1.0, std::max(0.0, v));
  }
  return SRS_OK;
}

}  // extern "C"
