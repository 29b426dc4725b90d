"""Pins of the FP64 oracle against the paper's printed numbers, closed forms,
library routines in limiting cases, and statistics.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
import srs_synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _one_sig(x):
    e = np.floor(np.log10(abs(x)))
    return round(x / 10 ** e) * 10 ** e


def test_beta_range_matches_paper():
    g = GOLD["beta_range"]
    lo = oracle.beta(g["mc_lo"], g["f_lo"])
    hi = oracle.beta(g["mc_hi"], g["f_hi"])
    assert _one_sig(lo) == pytest.approx(g["beta_lo_printed"])
    assert _one_sig(hi) == pytest.approx(g["beta_hi_printed"])


def test_injection_segment_count_matches_paper():
    g = GOLD["injection_segments"]
    b = oracle.beta(g["mc"], g["f0"])
    assert oracle.nseg(b, g["f0"], g["f_end"], g["t_coh"], 10 ** 6) == g["n_seg"]
    # 35 whole segments = 1050 s < 0PN band time < 36 segments
    t = oracle.duration(b, g["f0"], g["f_end"])
    assert 35 * 30.0 < t < 36 * 30.0


def test_band_crossing_times_match_paper():
    g = GOLD["band_crossing_times"]
    b1 = oracle.beta(g["cases"][0]["mc"], g["f_lo"])
    hours = oracle.duration(b1, g["f_lo"], g["f_hi"]) / 3600.0
    assert round(hours) == g["cases"][0]["hours_printed"]
    b2 = oracle.beta(g["cases"][1]["mc"], g["f_lo"])
    years = oracle.duration(b2, g["f_lo"], g["f_hi"]) / (365.25 * 86400.0)
    assert round(years) == g["cases"][1]["years_printed"]


def test_nseg_cut_rule_and_clamps():
    b = oracle.beta(0.1, 40.0)
    assert oracle.nseg(b, 40.0, 60.0, 30.0, 10) == 10      # clamped to the data
    assert oracle.nseg(b, 40.0, 60.0, 30.0, 100, cut=False) == 100
    heavy = oracle.beta(5.0, 40.0)                            # leaves band in < 30 s
    assert oracle.nseg(heavy, 40.0, 60.0, 30.0, 100) == 1


def test_frequency_reaches_f_end_after_duration():
    """Eq. (f) and the Sec. II duration are two separate formulas; they must agree."""
    for mc in (5e-4, 1e-2, 1e-1):
        b = oracle.beta(mc, 40.0)
        t = oracle.duration(b, 40.0, 60.0)
        assert oracle.freq(b, 40.0, t) == pytest.approx(60.0, rel=1e-12)


def test_delta_matches_high_precision_eq_new_t():
    """delta = tau(t_i0 + s) - tau(t_i0) with tau from Eq. (new_t) evaluated
    literally at 60 digits; the oracle's cancellation-free form must agree to
    ~1e-15 relative."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    for mc, i0 in ((5e-4, 2879), (1e-2, 100), (1e-1, 34), (3e-2, 0)):
        b = oracle.beta(mc, 40.0)
        t_i0 = i0 * 30.0
        B = mpmath.mpf(b)
        tau = lambda t: -mpmath.mpf(3) / 5 * (1 - mpmath.mpf(8) / 3 * B * t) ** (mpmath.mpf(5) / 8) / B
        for s in (0.0, 1.0 / 256, 7.3, 29.99609375):
            ref = tau(mpmath.mpf(t_i0) + mpmath.mpf(s)) - tau(mpmath.mpf(t_i0))
            got = oracle.delta(b, t_i0, s)[0]
            assert abs(got - float(ref)) <= 2e-15 * max(abs(float(ref)), 1e-300) + 1e-300


def test_delta_derivative_is_frequency_ratio():
    """d tau / dt = f(t) / f0 (Eq. (new_t) differentiated against Eq. (f))."""
    b = oracle.beta(1e-1, 40.0)
    t_i0, h = 900.0, 1e-3
    for s in (0.5, 12.0, 29.0):
        d = oracle.delta(b, t_i0, [s - h, s + h])
        slope = (d[1] - d[0]) / (2 * h)
        assert slope == pytest.approx(oracle.freq(b, 40.0, t_i0 + s) / 40.0, rel=1e-8)


def _theta_mp(beta, t_i0, fs, n, f):
    """2 pi f delta_j for j < n, computed at high precision from Eq. (new_t)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    B = mpmath.mpf(beta)
    tau = lambda t: -mpmath.mpf(3) / 5 * (1 - mpmath.mpf(8) / 3 * B * t) ** (mpmath.mpf(5) / 8) / B
    t0 = tau(mpmath.mpf(t_i0))
    out = np.empty(n)
    for j in range(n):
        cyc = mpmath.mpf(f) * (tau(mpmath.mpf(t_i0) + mpmath.mpf(j) / fs) - t0)
        out[j] = float(2 * mpmath.pi * (cyc - mpmath.floor(cyc)))
    return out


def test_tone_in_tau_gives_exactly_n():
    """Monochromatic in tau (Eq. (monochromatic)): x = cos(theta), y = sin(theta),
    theta_j = 2 pi f_b delta_j.  Then F_x(f_b) + i F_y(f_b) = sum_j 1 = N exactly,
    and F_x - i F_y = sum_j exp(-2 i theta_j)."""
    fs, T, f_lo, n_b = 64.0, 4.0, 10.0, 40
    n = int(fs * T)
    b = oracle.beta(0.05, 12.0)
    t_i0 = 3 * T
    bin0 = 9
    f0 = f_lo + bin0 / T
    th = _theta_mp(b, t_i0, fs, n, f0)
    strain = np.zeros(4 * n)
    strain[3 * n:] = np.cos(th)
    Fx = oracle.spectra(strain, fs, T, f_lo, n_b, [b], [(0, 3)])[0]
    strain[3 * n:] = np.sin(th)
    Fy = oracle.spectra(strain, fs, T, f_lo, n_b, [b], [(0, 3)])[0]
    assert abs(Fx[bin0] + 1j * Fy[bin0] - n) < 1e-9
    assert abs((Fx[bin0] - 1j * Fy[bin0]) - np.exp(-2j * th).sum()) < 1e-9


def test_tiny_spectra_against_brute_force():
    """Brute force on a tiny input: 3 segments of 64 samples of seeded noise,
    12 bins, two templates, global (t_i0 = i T) and segment-local (t_i0 = 0)
    time maps.  Every term x_j exp(-2 pi i f_b delta_j) is evaluated at 40
    digits with delta_j from Eq. (new_t) literally; the oracle must agree to
    1e-12 of the spectrum's norm."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    fs, T, f_lo, n_b = 16.0, 4.0, 1.0, 12
    n = int(fs * T)
    x = srs_synth.white_noise(3 * n, seed=23)
    betas = [4e-3, 2.5e-2]                 # (8/3) beta t < 1 over the 12 s
    items = [(m, i) for m in range(2) for i in range(3)]
    for local in (False, True):
        F = oracle.spectra(x, fs, T, f_lo, n_b, betas, items, local=local)
        for q, (m, i) in enumerate(items):
            B = mpmath.mpf(betas[m])
            tau = lambda t: -mpmath.mpf(3) / 5 * (1 - mpmath.mpf(8) / 3 * B * t) ** (mpmath.mpf(5) / 8) / B
            t_i0 = mpmath.mpf(0 if local else i * T)
            d = [tau(t_i0 + mpmath.mpf(j) / fs) - tau(t_i0) for j in range(n)]
            ref = np.empty(n_b, dtype=complex)
            for b in range(n_b):
                fb = mpmath.mpf(f_lo) + mpmath.mpf(b) / T
                acc = mpmath.mpc(0)
                for j in range(n):
                    acc += mpmath.mpf(float(x[i * n + j])) * mpmath.expjpi(-2 * fb * d[j])
                ref[b] = complex(acc)
            assert np.max(np.abs(F[q] - ref)) <= 1e-12 * np.linalg.norm(ref), (local, m, i)


def test_uniform_limit_is_the_fft():
    """beta -> 0 makes delta_j = j / fs, so with the full mode set the NDFT is the
    plain DFT: F(f_b) = fft(x)[(b - N/2) mod N] for f_b = (b - N/2) / T."""
    fs, T = 32.0, 8.0
    n = int(fs * T)
    x = srs_synth.white_noise(n, seed=3)
    F = oracle.spectra(x, fs, T, -fs / 2, n, [1e-30], [(0, 0)])[0]
    ref = np.fft.fft(x)
    k = (np.arange(n) - n // 2) % n
    assert np.max(np.abs(F - ref[k])) < 1e-9 * np.max(np.abs(ref))
    # Parseval over the full mode set
    assert np.sum(np.abs(F) ** 2) == pytest.approx(n * np.sum(x ** 2), rel=1e-12)


def test_real_input_conjugate_symmetry():
    """Real x: F(-f) = conj F(f) for any beta."""
    fs, T = 32.0, 4.0
    n = int(fs * T)
    x = srs_synth.white_noise(2 * n, seed=5)
    b = oracle.beta(0.08, 8.0)
    F = oracle.spectra(x, fs, T, -8.0, 65, [b], [(0, 1)])[0]   # f_b = -8 .. +8 Hz
    assert np.max(np.abs(F[::-1] - np.conj(F))) < 1e-9 * np.max(np.abs(F))


def test_noiseless_exact_template_chirp_concentrates_power():
    """A 0PN chirp resampled with its own beta is a tone at f0 in every segment
    (Sec. III.B): the peak bin is f0's and its power is A^2 N / 2 up to the
    O(1/N) cross term."""
    fs, T, f_lo, f_hi = 256.0, 30.0, 40.0, 60.0
    mc, f0, A = 3e-2, 45.0, 0.05
    n_s = int(fs * T)
    nseg = 6
    x = srs_synth.chirp(nseg * n_s, fs, mc, f0, A)
    b = oracle.beta(mc, f0)
    n_b = int((f_hi - f_lo) * T)
    F = oracle.spectra(x, fs, T, f_lo, n_b, [b], [(0, i) for i in range(nseg)])
    P = oracle.power(F, n_s)
    b0 = int(round((f0 - f_lo) * T))
    assert np.all(np.argmax(P, axis=1) == b0)
    assert np.allclose(P[:, b0], A * A * n_s / 2, rtol=5e-3)
    # everything off the peak is leakage-free to O(A^2): a tiny fraction
    off = np.delete(P, b0, axis=1)
    assert off.max() < 1e-3 * P[:, b0].min()


def test_noise_power_moments_and_n_sigma_null():
    """Gaussian N(0,1) noise: P ~ chi^2_2 (mean 2, std 2), n_sigma ~ (0, 1)."""
    g = GOLD["noise_power_moments"]
    fs, T, f_lo, f_hi = 256.0, 30.0, 40.0, 60.0
    n_s = int(fs * T)
    nseg = 8
    x = srs_synth.white_noise(nseg * n_s, seed=11)
    bets = [oracle.beta(m, 40.0) for m in (1e-3, 2e-2, 9e-2)]
    n_b = 600
    items = [(m, i) for m in range(3) for i in range(nseg)]
    P = oracle.power(oracle.spectra(x, fs, T, f_lo, n_b, bets, items), n_s)
    se = g["std"] / np.sqrt(P.size)
    assert abs(P.mean() - g["mean"]) < 4 * se * 2
    assert abs(P.std() - g["std"]) < 0.05 * g["std"]
    S = P.reshape(3, nseg, n_b).sum(axis=1)
    ns = oracle.n_sigma(S, [nseg] * 3)
    assert abs(ns.mean()) < 0.1 and abs(ns.std() - 1.0) < 0.1


def test_topk_order_against_brute_force():
    r = np.random.default_rng(0)
    M = r.integers(0, 6, size=(7, 9)).astype(np.float64)   # many ties
    v, m, b = oracle.topk(M, 20)
    brute = sorted(((-M[i, j], i, j) for i in range(7) for j in range(9)))[:20]
    assert [(-a, i, j) for a, i, j in brute] == list(zip(v, m, b))


def test_tau_literal_matches_high_precision_eq_new_t():
    """orc_tau is Eq. (new_t) as printed (t0 = 0); at 60 digits the same formula
    must agree with the FP64 evaluation to a few ulps of tau itself."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    for mc, t in ((5e-4, 0.0), (5e-4, 86399.0), (1e-2, 4321.5), (1e-1, 1000.0), (3e-2, 7199.99609375)):
        b = oracle.beta(mc, 40.0)
        B = mpmath.mpf(b)
        ref = -mpmath.mpf(3) / 5 * (1 - mpmath.mpf(8) / 3 * B * mpmath.mpf(t)) ** (mpmath.mpf(5) / 8) / B
        got = oracle.tau(b, t)
        assert abs(got - float(ref)) <= 4e-16 * abs(float(ref))


def test_tau_derivative_is_frequency_ratio():
    """d tau / dt = f(t) / f0 (Sec. III.B: the resampled signal is monochromatic at
    f0), with f from Eq. (f), a separate formula."""
    for mc in (1e-2, 1e-1):
        b = oracle.beta(mc, 40.0)
        for t, h in ((0.0, 0.25), (500.0, 0.25), (900.0, 0.125)):
            slope = (oracle.tau(b, t + h) - oracle.tau(b, t - h)) / (2 * h)
            assert slope == pytest.approx(oracle.freq(b, 40.0, t) / 40.0, rel=1e-7)


def test_tau_difference_is_the_segment_local_delta():
    """tau(t_i0 + s) - tau(t_i0) from the literal Eq. (new_t) equals the oracle's
    cancellation-free delta to the rounding of the large constant -(3/5)/beta."""
    for mc, t_i0 in ((2e-2, 3000.0), (1e-1, 600.0), (5e-4, 80000.0)):
        b = oracle.beta(mc, 40.0)
        big = abs(oracle.tau(b, t_i0))
        for s in (0.5, 13.0, 29.99609375):
            diff = oracle.tau(b, t_i0 + s) - oracle.tau(b, t_i0)
            assert abs(diff - oracle.delta(b, t_i0, s)[0]) <= 8e-16 * big


def test_semicoherent_exact_chirp_closed_form():
    """Sec. III.C on a noiseless chirp resampled with its own beta: in each of the
    template's first N_seg segments the chirp is a tone at f0 (Sec. III.B), so the
    power at f0's bin is A^2 n_s / 2 (up to the O(1/n_s) cross term), the sum is
    S = N_seg A^2 n_s / 2 and n_sigma = (S - 2 N_seg) / (2 sqrt(N_seg)) (equal
    weights).  Two templates with different segment counts: the exact one (row 1)
    and a mismatched one (row 0), whose power spreads over many bins."""
    fs, T, f_lo, f_hi = 256.0, 30.0, 40.0, 60.0
    mc, f0, A = 3e-2, 45.0, 0.05
    n_s = int(fs * T)
    x = srs_synth.chirp(6 * n_s, fs, mc, f0, A)
    b_true = oracle.beta(mc, f0)
    betas = [3.0 * b_true, b_true]
    nsegs = [3, 5]
    n_b = int((f_hi - f_lo) * T)
    S, ns = oracle.semicoherent(x, fs, T, f_lo, n_b, betas, nsegs)
    b0 = int(round((f0 - f_lo) * T))
    N = nsegs[1]
    S_ref = N * A * A * n_s / 2.0
    assert S.shape == (2, n_b) and ns.shape == (2, n_b)
    assert S[1, b0] == pytest.approx(S_ref, rel=5e-3)
    assert ns[1, b0] == pytest.approx((S_ref - 2.0 * N) / (2.0 * np.sqrt(N)), rel=1e-2)
    # off the peak the exact row holds leakage only: its n_sigma is -sqrt(N) (S ~ 0)
    off = np.delete(S[1], b0)
    assert off.max() < 1e-3 * S[1, b0]
    assert np.allclose(np.delete(ns[1], b0), -np.sqrt(N), atol=1e-2)
    # the mismatched template's power stays below the exact one's everywhere,
    # and its row is normalised by its own segment count (sum of P >= 0)
    assert S[0].max() < 0.5 * S[1, b0]
    assert ns[0].min() >= -np.sqrt(nsegs[0]) - 1e-12


def test_semicoherent_against_per_item_brute_force():
    """The semicoherent sum assembled item by item on a tiny input: each (m, i)
    spectrum is summed term by term at 40 digits with delta from Eq. (new_t) as
    printed, its power is 2|F|^2/n_s (Eq. normalized_power), template m adds its
    first N_seg(m) segments, n_sigma = (S - 2N)/(2 sqrt N) (Eqs. weights,
    semicoherent_statistic).  Seeded noise plus a chirp, so every segment's
    contribution differs."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    fs, T, f_lo, n_b = 16.0, 4.0, 1.0, 10
    n = int(fs * T)
    x = srs_synth.white_noise(5 * n, seed=29) + srs_synth.chirp(5 * n, fs, 40.0, 3.0, 0.7)
    betas = [4e-3, 1.5e-2]                 # (8/3) beta t < 1 over the 20 s
    nsegs = [2, 4]
    S, ns = oracle.semicoherent(x, fs, T, f_lo, n_b, betas, nsegs)
    S_ref = np.zeros((2, n_b))
    for m in range(2):
        B = mpmath.mpf(betas[m])
        tau = lambda t: -mpmath.mpf(3) / 5 * (1 - mpmath.mpf(8) / 3 * B * t) ** (mpmath.mpf(5) / 8) / B
        for i in range(nsegs[m]):
            t_i0 = mpmath.mpf(i * T)
            d = [tau(t_i0 + mpmath.mpf(j) / fs) - tau(t_i0) for j in range(n)]
            for b in range(n_b):
                fb = mpmath.mpf(f_lo) + mpmath.mpf(b) / T
                acc = mpmath.mpc(0)
                for j in range(n):
                    acc += mpmath.mpf(float(x[i * n + j])) * mpmath.expjpi(-2 * fb * d[j])
                S_ref[m, b] += float(2 * abs(acc) ** 2 / n)
    ns_ref = np.array([(S_ref[m] - 2.0 * nsegs[m]) / (2.0 * np.sqrt(nsegs[m])) for m in range(2)])
    assert np.max(np.abs(S - S_ref)) <= 1e-11 * np.max(S_ref)
    assert np.max(np.abs(ns - ns_ref)) <= 1e-11 * np.max(np.abs(ns_ref))
