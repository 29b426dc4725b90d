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
Equal weights use scipy's chi^2 and non-central chi^2 routines.  Unequal
weights use the exact survival function of a sum of exponentials with
distinct scales (the hypoexponential law),
  P(sum_i w_i E_i > q) = sum_i prod_{j != i} w_i / (w_i - w_j) exp(-q / w_i),
in 60-digit decimal arithmetic, so small inputs only.
"""
from decimal import Decimal, getcontext

import numpy as np
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
    lo, hi = mean, mean + 40.0
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
