"""Detection statistics of the semicoherent search (oracle side).

TEST INFRASTRUCTURE ONLY (same rule as the rest of `oracle`).

Passages followed (Sec. III.C):
  Eq. (semicoherent_statistic) under H0: with P_i ~ chi^2_2 (mu = sigma = 2),
    n_sigma = sum_i w_i (P_i - 2) / 2 = sum_i w_i E_i - sum_i w_i,
    E_i ~ Exp(1), sum w^2 = 1.
  Eq. (n_sigma^th): the threshold with P(n_sigma > th | H0) = p_fa.
  Eq. (non-centrality_threshold): the total non-centrality Lambda that
    crosses the threshold with probability p_det (equal weights: sum P_i is
    non-central chi^2 with 2N dof).
  ROC (the detection probability against p_fa for a signal with per-segment
    non-centralities lambda_i, Fig. roc's ordinate for one signal):
    P(n_sigma > n_sigma^th(p_fa) | lambda_i, w).
Equal weights use scipy's chi^2 and non-central chi^2 routines.  Unequal
weights use the exact survival function of a sum of exponentials with
distinct scales (the hypoexponential law),
  P(sum_i w_i E_i > q) = sum_i prod_{j != i} w_i / (w_i - w_j) exp(-q / w_i),
in 60-digit decimal arithmetic, so small inputs only.  With a signal and
unequal weights, Q = sum_i w_i P_i (P_i non-central chi^2, 2 dof) has the
characteristic function
  phi(t) = prod_i exp(i lambda_i w_i t / (1 - 2 i w_i t)) / (1 - 2 i w_i t),
and P(Q > x) = 1/2 + (1/pi) int_0^inf Im[exp(-i t x) phi(t)] / t dt
(Gil-Pelaez 1951), integrated with scipy's adaptive and Fourier quadratures.
"""
from decimal import Decimal, getcontext

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq
from scipy.stats import chi2, ncx2


def nsigma_threshold_equal(n_seg, p_fa):
    """(chi^2_{2N} isf(p_fa) - 2N) / (2 sqrt(N))."""
    s = chi2.isf(p_fa, 2 * n_seg)
    return (s - 2.0 * n_seg) / (2.0 * np.sqrt(n_seg))


def detection_noncentrality(n_seg, p_fa, p_det):
    """Lambda with P(chi^2_{2N}(Lambda) > chi^2_{2N} isf(p_fa)) = p_det."""
    s = chi2.isf(p_fa, 2 * n_seg)
    return brentq(lambda lam: ncx2.sf(s, 2 * n_seg, lam) - p_det, 1e-9, 1e5, xtol=1e-12, rtol=1e-14)


def weighted_exp_sf(w, q, digits=60):
    """P(sum_i w_i E_i > q) for distinct positive w (hypoexponential law)."""
    getcontext().prec = digits
    W = [Decimal(repr(float(v))) for v in w]
    Q = Decimal(repr(float(q)))
    total = Decimal(0)
    for i, wi in enumerate(W):
        c = Decimal(1)
        for j, wj in enumerate(W):
            if j != i:
                c *= wi / (wi - wj)
        total += c * (-Q / wi).exp()
    return float(total)


def nsigma_threshold_weighted(w, p_fa):
    """The threshold for distinct positive weights (normalised to sum w^2 = 1)."""
    w = np.asarray(w, dtype=np.float64)
    w = w / np.sqrt(np.sum(w * w))
    mean = float(np.sum(w))
    lo, hi = 0.0, mean + 40.0          # q > 0: the law of a sum of positive terms starts there
    f = lambda q: np.log(weighted_exp_sf(w, q)) - np.log(p_fa)
    q = brentq(f, lo, hi, xtol=1e-13)
    return q - mean


def detection_probability_mc(w, lam_total, threshold, n_draws, seed):
    """Monte Carlo P(n_sigma > threshold) for weights w (normalised to
    sum w^2 = 1) and a signal of total non-centrality lam_total split as
    lambda_i = lam_total w_i / sum w: P_i ~ non-central chi^2 with 2 dof."""
    w = np.asarray(w, dtype=np.float64)
    w = w / np.sqrt(np.sum(w * w))
    lam = lam_total * w / np.sum(w)
    r = np.random.default_rng(seed)
    hits = 0
    done = 0
    while done < n_draws:
        m = min(500_000, n_draws - done)
        P = r.noncentral_chisquare(2.0, lam, size=(m, w.size))
        ns = (P - 2.0) / 2.0 @ w
        hits += int(np.sum(ns > threshold))
        done += m
    return hits / n_draws


def weighted_noncentral_sf(w, lam, x):
    """P(sum_i w_i P_i > x), P_i ~ non-central chi^2 (2 dof, lambda_i), by the
    Gil-Pelaez inversion of the characteristic function (weights as given)."""
    w = np.asarray(w, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)

    def phi(t):
        z = 1.0 - 2.0j * w * t
        return np.prod(np.exp(1j * lam * w * t / z) / z)

    def g(t):
        if t == 0.0:
            return float(np.sum(w * (2.0 + lam))) - x      # the t -> 0 limit of Im[e^{-itx} phi] / t
        return (np.exp(-1j * t * x) * phi(t)).imag / t

    a = 20.0 / x
    head, _ = quad(g, 0.0, a, limit=400, epsabs=1e-13, epsrel=1e-12)
    # beyond a: Im[e^{-itx} phi] = Im phi cos(xt) - Re phi sin(xt), Fourier integrals on [a, inf)
    c, _ = quad(lambda t: phi(t).imag / t, a, np.inf, weight="cos", wvar=x, limlst=200, epsabs=1e-13)
    s, _ = quad(lambda t: phi(t).real / t, a, np.inf, weight="sin", wvar=x, limlst=200, epsabs=1e-13)
    return 0.5 + (head + c - s) / np.pi


def detection_probability(w, lam, p_fa):
    """P(n_sigma > n_sigma^th(p_fa) | lambda) for weights w (normalised to
    sum w^2 = 1; None or all equal: equal weights) and per-segment
    non-centralities lam.  n_sigma > th  <=>  sum_i w_i P_i > 2 th + 2 sum w."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.size
    if w is None or np.all(np.asarray(w) == np.asarray(w)[0]):
        s = chi2.isf(p_fa, 2 * n)
        total = float(np.sum(lam))
        return float(chi2.sf(s, 2 * n) if total == 0.0 else ncx2.sf(s, 2 * n, total))
    w = np.asarray(w, dtype=np.float64)
    w = w / np.sqrt(np.sum(w * w))
    th = nsigma_threshold_weighted(w, p_fa)
    return float(weighted_noncentral_sf(w, lam, 2.0 * th + 2.0 * np.sum(w)))
