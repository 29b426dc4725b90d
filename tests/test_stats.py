"""Detection statistics: the oracle (oracle.stats) pinned by the printed
detection non-centrality, a closed form, textbook laws and Monte Carlo; then
the library's host functions (srs_nsigma_threshold,
srs_detection_noncentrality, srs_detection_probability) against the oracle.
CPU only: these functions need no GPU."""
import json
import os

import numpy as np
import pytest

from oracle import stats
from scipy.stats import chi2, ncx2

from paper_2609_12476_gb300 import SrsError, detection_noncentrality, detection_probability, nsigma_threshold

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_oracle_detection_noncentrality_matches_paper():
    g = GOLD["detection_noncentrality"]
    lam = stats.detection_noncentrality(g["n_seg"], g["p_fa"], g["p_det"])
    assert round(lam, 1) == g["lambda_printed"]


def test_oracle_one_segment_threshold_closed_form():
    # one segment: n_sigma = E - 1 with E ~ Exp(1), so th = -ln(p_fa) - 1
    for p in (0.9, 0.5, 1e-2, 1e-6, 1e-9):
        assert stats.nsigma_threshold_equal(1, p) == pytest.approx(-np.log(p) - 1.0, rel=1e-10)
        assert stats.nsigma_threshold_weighted([1.0], p) == pytest.approx(-np.log(p) - 1.0, rel=1e-9)


def test_oracle_weighted_law_monte_carlo():
    """The hypoexponential survival function against 4e6 seeded draws."""
    w = np.array([0.3, 0.5, 0.9, 1.4, 2.0])
    e = np.random.default_rng(17).exponential(1.0, size=(4_000_000, w.size))
    q_all = e @ w
    for q in (4.0, 7.0, 10.0):
        emp = np.mean(q_all > q)
        sf = stats.weighted_exp_sf(w, q)
        assert abs(emp - sf) <= 4 * np.sqrt(sf * (1 - sf) / q_all.size) + 1e-7, (q, emp, sf)


def test_oracle_weighted_threshold_tends_to_equal():
    n = 12
    w = 1.0 + 1e-3 * np.arange(n)
    assert stats.nsigma_threshold_weighted(w, 1e-6) == pytest.approx(stats.nsigma_threshold_equal(n, 1e-6), rel=2e-3)


@pytest.mark.parametrize("n", [1, 2, 7, 35, 240, 2880])
@pytest.mark.parametrize("p_fa", [1e-2, 1e-6, 1e-9])
def test_library_equal_weight_threshold(n, p_fa):
    assert nsigma_threshold(n, p_fa) == pytest.approx(stats.nsigma_threshold_equal(n, p_fa), rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_library_weighted_threshold(seed):
    r = np.random.default_rng(seed)
    n = int(r.integers(2, 16))
    w = np.sort(r.uniform(0.4, 2.5, n))
    w[1:] += 1e-3 * np.arange(1, n)          # distinct, for the oracle's closed form
    for p in (1e-3, 1e-6):
        assert nsigma_threshold(n, p, w) == pytest.approx(stats.nsigma_threshold_weighted(w, p), rel=1e-8)


def test_library_weighted_threshold_scale_free_and_long_tracks():
    # weights are normalised: any common scale gives the same threshold
    w = np.linspace(1.0, 1.72, 300)
    assert nsigma_threshold(300, 1e-6, w) == pytest.approx(nsigma_threshold(300, 1e-6, 7.5 * w), rel=1e-12)
    # amplitude-like weights over a long track stay close to (and above) the equal-weight threshold
    w = np.linspace(1.0, 1.72, 2880)
    a, b = nsigma_threshold(2880, 1e-6, w), nsigma_threshold(2880, 1e-6)
    assert b <= a <= 1.05 * b


@pytest.mark.parametrize("n", [1, 3, 35, 100])
def test_library_detection_noncentrality(n):
    assert detection_noncentrality(n, 1e-6, 0.95) == pytest.approx(stats.detection_noncentrality(n, 1e-6, 0.95),
                                                                   rel=1e-9)


def test_library_statistics_reject_bad_arguments():
    with pytest.raises(SrsError):
        nsigma_threshold(0, 1e-6)
    with pytest.raises(SrsError):
        nsigma_threshold(3, 1.5)
    with pytest.raises(SrsError):
        nsigma_threshold(3, 1e-6, [1.0, -1.0, 2.0])
    with pytest.raises(SrsError):
        detection_noncentrality(10, 1e-6, 1.0)


def test_library_weighted_detection_noncentrality_monte_carlo():
    """With unequal weights the library's Lambda^det gives p_det = 0.95 under
    2e6 seeded draws of the weighted non-central sum (threshold from the
    oracle's exact hypoexponential law)."""
    w = np.array([0.6, 0.8, 1.0, 1.3, 1.7, 2.2])
    p_fa, p_det = 1e-4, 0.95
    lam = detection_noncentrality(w.size, p_fa, p_det, weights=w)
    th = stats.nsigma_threshold_weighted(w, p_fa)
    est = stats.detection_probability_mc(w, lam, th, 2_000_000, seed=31)
    assert abs(est - p_det) < 4 * np.sqrt(p_det * (1 - p_det) / 2_000_000), (lam, est)
    # equal weights given explicitly take the exact route; nearly equal ones agree with it
    n = 12
    exact = detection_noncentrality(n, 1e-6, 0.95)
    assert detection_noncentrality(n, 1e-6, 0.95, weights=np.ones(n)) == exact
    near = detection_noncentrality(n, 1e-6, 0.95, weights=1.0 + 1e-4 * np.arange(n))
    assert near == pytest.approx(exact, rel=1e-5)


def test_library_weighted_threshold_on_a_month_long_track():
    """A 26-day track (Mc = 1e-3 across 40-60 Hz: 76 158 segments) with
    segment-averaged f^(4/3) weights: the mixture's constant C = prod b / w_i
    is e^-17500 there, far outside floating-point range, and the threshold
    still comes out just above the equal-weight one."""
    import srs_synth
    b0 = srs_synth.chirp_beta(1e-3, 40.0)
    L = int(3 / (8 * b0) * (1 - (40 / 60) ** (8 / 3)) / 30.0)
    s = np.arange(L)
    a = 2.0 / (np.sqrt(1 - 8 / 3 * b0 * s * 30.0) + np.sqrt(np.maximum(1 - 8 / 3 * b0 * (s + 1) * 30.0, 0.0)))
    assert L > 70000 and a.max() / a.min() > 1.7
    te, tw = nsigma_threshold(L, 1e-6), nsigma_threshold(L, 1e-6, a)
    assert te < tw < 1.01 * te


def test_oracle_weighted_noncentral_law_reduces_to_textbook_laws():
    """The characteristic-function inversion with equal weights is scipy's
    non-central chi^2 with 2N dof and total non-centrality sum lambda_i,
    however the signal is split; without a signal and unequal weights it is
    the hypoexponential law (sum w P = 2 sum w E)."""
    for n, lam, x in [(1, [5.0], 12.0), (3, [1.0, 2.0, 7.0], 20.0), (4, [30.0, 0.0, 0.0, 0.0], 25.0),
                      (2, [0.4, 0.6], 60.0)]:
        got = stats.weighted_noncentral_sf(np.ones(n), lam, x)
        assert got == pytest.approx(ncx2.sf(x, 2 * n, sum(lam)), rel=1e-6, abs=1e-14), (n, lam, x)
    assert stats.weighted_noncentral_sf(np.ones(6), np.zeros(6), 15.0) == pytest.approx(chi2.sf(15.0, 12), rel=1e-12)
    w = np.array([0.3, 0.5, 0.9, 1.4, 2.0])
    for q in (4.0, 10.0, 40.0, 60.0):
        got = stats.weighted_noncentral_sf(w, np.zeros(5), q)
        assert got == pytest.approx(stats.weighted_exp_sf(w, q / 2), rel=1e-8, abs=1e-15), q


def test_oracle_detection_probability_monte_carlo():
    """Unequal weights and an unequal signal split against 2e6 seeded draws of
    the weighted non-central sum."""
    w = np.array([0.5, 0.9, 1.1, 1.6, 2.3])
    lam = np.array([0.5, 6.0, 2.0, 9.0, 1.0])
    r = np.random.default_rng(41)
    n_draws = 2_000_000
    P = r.noncentral_chisquare(2.0, lam, size=(n_draws, w.size))
    wn = w / np.sqrt(np.sum(w * w))
    ns = (P - 2.0) / 2.0 @ wn
    for p_fa in (1e-3, 1e-2, 1e-1):
        th = stats.nsigma_threshold_weighted(w, p_fa)
        emp = float(np.mean(ns > th))
        pd = stats.detection_probability(w, lam, p_fa)
        assert abs(emp - pd) <= 4 * np.sqrt(pd * (1 - pd) / n_draws), (p_fa, emp, pd)


@pytest.mark.parametrize("n", [1, 3, 35, 300])
def test_library_detection_probability_equal_weights(n):
    r = np.random.default_rng(n)
    lam = r.uniform(0.0, 2.0, n) * (60.0 / n)
    pf = [1e-8, 1e-6, 1e-3, 0.1]
    got = detection_probability(n, pf, lam)
    want = [stats.detection_probability(None, lam, p) for p in pf]
    assert got == pytest.approx(want, rel=1e-9, abs=1e-15)
    # equal weights given explicitly take the same exact route
    assert np.array_equal(detection_probability(n, pf, lam, weights=np.full(n, 3.0)), got)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_library_detection_probability_weighted(seed):
    r = np.random.default_rng(100 + seed)
    n = int(r.integers(2, 9))
    w = np.sort(r.uniform(0.4, 2.5, n))
    w[1:] += 1e-3 * np.arange(1, n)          # distinct, for the oracle's threshold
    lam = r.uniform(0.0, 12.0, n)
    pf = [1e-6, 1e-4, 1e-2]
    got = detection_probability(n, pf, lam, weights=w)
    want = [stats.detection_probability(w, lam, p) for p in pf]
    assert got == pytest.approx(want, rel=1e-6, abs=1e-9)


def test_library_roc_properties():
    """No signal gives p_det = p_fa; p_det rises with p_fa and with the
    signal; at the library's Lambda^det with lambda_i = Lambda w_i / sum w it
    is p_det."""
    w = np.array([0.6, 0.8, 1.0, 1.3, 1.7, 2.2])
    pf = np.logspace(-9, -1, 9)
    for weights in (None, w):
        assert detection_probability(6, pf, None, weights) == pytest.approx(pf, rel=1e-6, abs=1e-11)
        lo = detection_probability(6, pf, np.full(6, 2.0), weights)
        hi = detection_probability(6, pf, np.full(6, 4.0), weights)
        assert np.all(np.diff(lo) > 0) and np.all(hi > lo)
    for weights in (None, w):
        lam_det = detection_noncentrality(6, 1e-6, 0.95, weights=weights)
        ww = np.ones(6) if weights is None else weights / np.sqrt(np.sum(weights ** 2))
        assert detection_probability(6, 1e-6, lam_det * ww / ww.sum(), weights) == pytest.approx(0.95, abs=1e-8)
    # the paper's one-segment number: Lambda = 46.5 at p_fa = 1e-6 gives p_det = 0.95
    g = GOLD["detection_noncentrality"]
    assert detection_probability(1, g["p_fa"], [g["lambda_printed"]]) == pytest.approx(g["p_det"], abs=2e-3)


def test_library_detection_probability_rejects_bad_arguments():
    with pytest.raises(SrsError):
        detection_probability(3, 0.0)
    with pytest.raises(SrsError):
        detection_probability(3, [1e-6, 1.0])
    with pytest.raises(SrsError):
        detection_probability(3, 1e-6, [1.0, -0.5, 2.0])
    with pytest.raises(SrsError):
        detection_probability(3, 1e-6, [1.0, np.nan, 2.0])
    with pytest.raises(SrsError):
        detection_probability(3, 1e-6, None, [1.0, 0.0, 2.0])
    with pytest.raises(SrsError):
        detection_probability(0, 1e-6)


def test_library_two_routes_agree_on_long_tracks():
    """On tracks too long for the 60-digit oracle, the library's two unequal-
    weight routes check each other: the threshold from the Gamma mixture must
    have false-alarm probability p_fa under Imhof's integral (no signal)."""
    for n in (300, 2880):
        w = np.linspace(1.0, 1.72, n)
        for p_fa in (1e-2, 1e-4, 1e-6):
            assert detection_probability(n, p_fa, None, w) == pytest.approx(p_fa, rel=1e-5)


@pytest.mark.parametrize("n,spread", [(20, 1e3), (10, 1e4), (6, 1e6)])
def test_library_threshold_for_widely_spread_weights(n, spread):
    """Weights spread over 3 to 6 decades: the Gamma mixture would need far
    too many terms, and the library takes Imhof's integral instead; the
    threshold still matches the oracle's exact hypoexponential law."""
    w = np.linspace(1.0, spread, n)
    for p in (1e-3, 1e-6):
        assert nsigma_threshold(n, p, w) == pytest.approx(stats.nsigma_threshold_weighted(w, p), rel=1e-8)


def test_library_refuses_weighted_thresholds_it_cannot_finish():
    """Unequal weights on a two-million-segment track would take either route
    far too long: the call says so instead of running for hours."""
    n = 2_000_000
    with pytest.raises(SrsError) as e:
        nsigma_threshold(n, 1e-6, np.linspace(1.0, 2.0, n))
    assert e.value.status == -5          # SRS_ERR_UNSUPPORTED
    assert nsigma_threshold(n, 1e-6) > 0  # equal weights stay exact and cheap


def test_library_thresholds_across_the_whole_p_fa_range():
    """p_fa from 0.9 (a threshold below the mean) down to 1e-20, equal and
    unequal weights, against the oracle."""
    w = np.array([0.5, 0.9, 1.1, 1.6, 2.3])
    for p in (0.9, 0.5, 1e-12, 1e-15, 1e-20):
        assert nsigma_threshold(5, p, w) == pytest.approx(stats.nsigma_threshold_weighted(w, p), rel=1e-9, abs=1e-12)
        assert nsigma_threshold(7, p) == pytest.approx(stats.nsigma_threshold_equal(7, p), rel=1e-9, abs=1e-12)
    for n, p_fa, p_det in ((1, 0.5, 0.99), (3, 0.9, 0.95), (40, 0.7, 0.8), (1, 1e-12, 0.9999)):
        assert detection_noncentrality(n, p_fa, p_det) == pytest.approx(stats.detection_noncentrality(n, p_fa, p_det),
                                                                        rel=1e-9)


def test_library_detection_probability_loud_and_uneven_signals():
    """A loud signal (lambda 300 per segment) and signals concentrated in a few
    segments: the integral's panels follow the fastest oscillation."""
    w = np.array([0.5, 0.9, 1.1, 1.6, 2.3])
    pf = [1e-9, 1e-6, 1e-3, 0.5]
    for lam in ([300.0] * 5, [50.0, 0.0, 0.0, 0.0, 80.0], [20.0, 5.0, 1.0, 0.0, 3.0]):
        got = detection_probability(5, pf, np.array(lam), w)
        want = [stats.detection_probability(w, np.array(lam), p) for p in pf]
        assert got == pytest.approx(want, rel=1e-6, abs=1e-9), lam
