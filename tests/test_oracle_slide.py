"""Pins of the two-stage oracle (oracle.slide): the local resampling bank, the
per-segment power cube, the {Mc, t0} tracks and the stack-slide sum, against
printed numbers, identities of the 0PN model, an injected chirp, closed forms
and brute force.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
import srs_synth
from oracle import slide

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
T, F_LO, F_HI, FS = 30.0, 40.0, 60.0, 256.0
N_B = 600


def _bank():
    g = GOLD["local_bank"]
    return slide.local_bank(g["beta_min"], g["beta_max"], g["n_beta"])


def test_bank_is_uniform_over_the_printed_range():
    g = GOLD["local_bank"]
    b = _bank()
    assert b.size == g["n_beta"]
    assert b[0] == g["beta_min"] and b[-1] == pytest.approx(g["beta_max"], rel=1e-15)
    assert np.allclose(np.diff(b), (g["beta_max"] - g["beta_min"]) / (g["n_beta"] - 1), rtol=1e-12)
    # the bank spans the local chirp parameters of the searched chirp masses over the band
    assert oracle.beta(5e-4, F_LO) >= b[0] * 0.9 and oracle.beta(1e-1, F_HI) <= b[-1] * 1.1


def test_cube_size_matches_printed_memory_figures():
    """Sec. VI: a year of spectra is about 200 GB, 80 GB hold about 165 days,
    for a cube of n_beta x band bins of single-precision powers per segment."""
    g = GOLD["cube_memory"]
    per_seg = g["n_beta"] * round((g["f_hi"] - g["f_lo"]) * g["t_coh"]) * g["bytes_per_power"]
    year = 365.25 * 86400.0 / g["t_coh"] * per_seg
    assert round(year / 1e11) * 1e11 == g["year_bytes_printed"]
    days = g["device_bytes"] / per_seg * g["t_coh"] / 86400.0
    assert days == pytest.approx(g["days_printed"], rel=0.03)


@pytest.mark.parametrize("mc,i", [(3e-2, 100), (1e-1, 20), (2e-3, 2000)])
def test_local_map_is_the_global_map_rescaled(mc, i):
    """Within segment i, the track that starts at f_ref at t = 0 and the 0PN
    template that starts at the segment (with beta(Mc, f_i), f_i its frequency
    there) share a phase: f_ref delta_global(s) = f_i delta_local(s)."""
    b = oracle.beta(mc, F_LO)
    t_i0 = i * T
    f_i = oracle.freq(b, F_LO, t_i0)
    b_i = oracle.beta(mc, f_i)
    s = np.linspace(0.0, T, 17)
    g = oracle.delta(b, t_i0, s)
    loc = oracle.delta(b_i, 0.0, s)
    assert np.allclose(F_LO * g, f_i * loc, rtol=1e-12, atol=1e-12)


def _phase(mc, f0, t):
    """Eq. (phi) with t0 = 0, phi0 = 0 (test-side)."""
    b = srs_synth.chirp_beta(mc, f0)
    return -(6.0 * np.pi / 5.0) * f0 * (1.0 - (8.0 / 3.0) * b * t) ** 0.625 / b


@pytest.mark.parametrize("mc,c", [(1e-2, 0.0), (6e-2, 0.25), (1e-1, 0.9), (5e-4, 0.5)])
def test_track_frequency_is_the_phase_derivative(mc, c):
    """The track's frequency in each segment is the chirp's instantaneous
    frequency at the segment's first sample: (1/2 pi) d phi/dt of Eq. (phi),
    by a central difference."""
    k, j = slide.track(mc, c, F_LO, T, F_LO, N_B, _bank(), 400)
    assert len(j) > 0
    off = (1.0 if c > 0 else 0.0) - c
    h = 1e-3
    for s in range(0, len(j), max(1, len(j) // 20)):
        t = (s + off) * T
        f_num = (_phase(mc, F_LO, t + h) - _phase(mc, F_LO, t - h)) / (2 * h) / (2 * np.pi)
        x = (f_num - F_LO) * T
        if abs(x - np.floor(x) - 0.5) > 1e-3:          # away from a rounding tie
            assert j[s] == int(np.rint(x))
    assert np.all(np.diff(j) >= 0)                      # the chirp only rises


@pytest.mark.parametrize("mc,c", [(1e-1, 0.0), (1e-1, 0.5), (4e-2, 0.0), (7e-2, 0.3)])
def test_track_length_matches_band_time(mc, c):
    """The track ends where the nearest bin leaves the band: the last track
    segment starts before the 0PN time (Sec. II duration) from f0 to
    f_hi - 1/(2T) has passed, the next one after."""
    b = oracle.beta(mc, F_LO)
    k, j = slide.track(mc, c, F_LO, T, F_LO, N_B, _bank(), 10 ** 6)
    off = (1.0 if c > 0 else 0.0) - c
    t_edge = oracle.duration(b, F_LO, F_HI - 0.5 / T)
    L = len(j)
    assert (L - 1 + off) * T < t_edge < (L + off) * T
    assert j[-1] == N_B - 1 or j[-1] == N_B - 2 or (L + off) * T - t_edge < T


def test_track_bank_index_is_nearest_local_beta():
    bank = _bank()
    for mc, c in [(1e-2, 0.0), (9e-2, 0.4)]:
        k, j = slide.track(mc, c, F_LO, T, F_LO, N_B, bank, 300)
        b0 = oracle.beta(mc, F_LO)
        off = (1.0 if c > 0 else 0.0) - c
        for s in range(len(k)):
            # local chirp parameter by Eq. (f): beta(t) = beta0 / (1 - 8/3 beta0 t)
            bl = b0 / (1.0 - (8.0 / 3.0) * b0 * (s + off) * T)
            d = np.abs(bank - bl)
            assert d[k[s]] <= d.min() * (1 + 1e-9) + 1e-30


def test_stack_slide_closed_forms():
    bank = _bank()
    rows_mc = np.array([8e-2, 8e-2, 3e-2])
    rows_c = np.array([0.0, 0.5, 0.0])
    n_total, n_t0 = 60, 50
    cube = np.full((len(bank), N_B, n_total), 2.0)
    ns, L = slide.stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B)
    assert np.all(ns == 0.0)
    # raise only the cells of one template's track by 2 c: that template reads c sqrt(N)
    r0, n0, cval = 0, 7, 0.75
    k, j = slide.track(rows_mc[r0], rows_c[r0], F_LO, T, F_LO, N_B, bank, n_total)
    first = slide.first_segment(n0, rows_c[r0])
    Lp = min(len(k), n_total - first)
    cube[k[:Lp], j[:Lp], first + np.arange(Lp)] += 2.0 * cval
    ns, L = slide.stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B)
    assert L[r0, n0] == Lp
    assert ns[r0, n0] == pytest.approx(cval * np.sqrt(Lp), rel=1e-12)
    # the data end truncates tracks: N_seg counts only segments inside the data
    assert L[2, n_t0 - 1] == min(len(slide.track(3e-2, 0.0, F_LO, T, F_LO, N_B, bank, n_total)[0]),
                                 n_total - (n_t0 - 1))


def test_stack_slide_brute_force_on_a_random_cube():
    """A pure-Python loop over templates, track segments and cells against
    oracle.slide.stack_slide on a seeded chi-square cube."""
    bank = slide.local_bank(3e-8, 7e-4, 12)
    n_total, n_t0 = 40, 40
    cube = srs_synth.random_cube(len(bank), N_B, n_total, seed=5).astype(np.float64)
    rows_mc = np.array([1e-1, 1e-1, 5e-2, 2e-2])
    rows_c = np.array([0.0, 0.5, 0.2, 0.0])
    ns, L = slide.stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B)
    for r in range(len(rows_mc)):
        k, j = slide.track(rows_mc[r], rows_c[r], F_LO, T, F_LO, N_B, bank, n_total)
        for n in range(n_t0):
            acc, cnt = 0.0, 0
            i = n + (1 if rows_c[r] > 0 else 0)
            for s in range(len(k)):
                if i + s >= n_total:
                    break
                acc += (cube[k[s], j[s], i + s] - 2.0) / 2.0
                cnt += 1
            want = acc / np.sqrt(cnt) if cnt else 0.0
            assert ns[r, n] == pytest.approx(want, rel=1e-12, abs=1e-12)
            assert L[r, n] == cnt


@pytest.mark.slow
def test_power_cube_concentrates_an_entering_chirp():
    """A noise-free 0PN chirp that enters the band at t0: in each of its
    segments the cube's largest power over (beta bank, bin) sits on the track's
    cell (within one bin and one bank step), at a large share of the coherent
    maximum A^2 n_s / 2."""
    mc, t0, amp = 2e-2, 600.0, 1.0
    n_seg = 30
    x = srs_synth.strain_with_chirps(int(n_seg * T * FS), FS, 0,
                                     [{"mc": mc, "f0": F_LO, "amp": amp, "t_start": t0}], noise=False)
    bank = _bank()
    k, j = slide.track(mc, 0.0, F_LO, T, F_LO, N_B, bank, n_seg)
    segs = [20, 25, 29]
    P = slide.power_cube(x, FS, T, F_LO, N_B, bank, segs[0], segs[-1] + 1)
    n_s = int(T * FS)
    for i in segs:
        s = i - 20                           # t0 = 20 T
        sl = P[:, :, i - segs[0]]
        kk, jj = np.unravel_index(np.argmax(sl), sl.shape)
        assert abs(int(jj) - int(j[s])) <= 1 and abs(int(kk) - int(k[s])) <= 1, (i, kk, jj, k[s], j[s])
        assert sl.max() > 0.35 * amp ** 2 * n_s / 2


@pytest.mark.parametrize("mc,c,s", [(1e-2, 0.0, 0), (1e-2, 0.3, 500), (1e-1, 0.0, 30), (1e-1, 0.6, 34), (3e-3, 0.0, 2000)])
def test_amplitude_average_matches_closed_form(mc, c, s):
    """A^2 ~ f^(4/3) (Eq. h0) with f = f0 A(t)^(-3/8) (Eq. f) is f0^(4/3)
    A(t)^(-1/2); its mean over [dt, dt + T) is 2 / (sqrt(A(dt)) + sqrt(A(dt + T)))
    in units of f0^(4/3).  The oracle integrates numerically."""
    b0 = srs_synth.chirp_beta(mc, F_LO)
    dt = (s + (1.0 if c > 0 else 0.0) - c) * T
    A0, A1 = 1 - 8 / 3 * b0 * dt, 1 - 8 / 3 * b0 * (dt + T)
    want = 2.0 / (np.sqrt(A0) + np.sqrt(A1))
    assert slide.amplitude_sq(mc, c, F_LO, T, s) == pytest.approx(want, rel=1e-10)


def test_weighted_stack_slide_closed_forms():
    bank = _bank()
    rows_mc, rows_c = np.array([9e-2, 4e-2]), np.array([0.25, 0.0])
    n_total, n_t0 = 80, 60
    r = np.random.default_rng(4)
    s_eff = r.uniform(0.5, 3.0, size=(len(bank), N_B))
    # P / S = 2 everywhere: every template reads 0 under any weights
    cube = 2.0 * np.repeat(s_eff[:, :, None], n_total, axis=2)
    ns, L = slide.stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B, weighting=1,
                              s_eff=s_eff)
    assert np.allclose(ns, 0.0, atol=1e-12)
    # P / S = 2 + 2 c on one template's track: c sum(a) / sqrt(sum a^2), a = A^2 / S
    r0, n0, cval = 0, 11, 0.5
    k, j = slide.track(rows_mc[r0], rows_c[r0], F_LO, T, F_LO, N_B, bank, n_total)
    first = slide.first_segment(n0, rows_c[r0])
    Lp = min(len(k), n_total - first)
    cube[k[:Lp], j[:Lp], first + np.arange(Lp)] += 2.0 * cval * s_eff[k[:Lp], j[:Lp]]
    ns, L = slide.stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B, weighting=1,
                              s_eff=s_eff)
    a = np.array([slide.amplitude_sq(rows_mc[r0], rows_c[r0], F_LO, T, s) for s in range(Lp)]) / s_eff[k[:Lp], j[:Lp]]
    assert ns[r0, n0] == pytest.approx(cval * a.sum() / np.sqrt((a * a).sum()), rel=1e-12)
    # equal weights and a white PSD give the unweighted statistic
    cube2 = srs_synth.random_cube(len(bank), N_B, n_total, seed=9).astype(np.float64)
    u, _ = slide.stack_slide(cube2, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B)
    w, _ = slide.stack_slide(cube2, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B,
                             s_eff=np.ones((len(bank), N_B)))
    assert np.allclose(u, w, rtol=1e-12, atol=1e-12)
    # one PSD scale for power and weights cancels
    w1, _ = slide.stack_slide(cube2 * 3.0, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B, weighting=1,
                              s_eff=np.full((len(bank), N_B), 3.0))
    w0, _ = slide.stack_slide(cube2, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B, weighting=1)
    assert np.allclose(w1, w0, rtol=1e-12, atol=1e-12)


def test_weighted_stack_slide_brute_force():
    bank = slide.local_bank(3e-8, 7e-4, 10)
    n_total, n_t0 = 30, 30
    cube = srs_synth.random_cube(len(bank), N_B, n_total, seed=6).astype(np.float64)
    s_eff = np.random.default_rng(2).uniform(0.7, 1.6, size=(len(bank), N_B))
    rows_mc, rows_c = np.array([1e-1, 6e-2]), np.array([0.5, 0.0])
    ns, L = slide.stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B, weighting=1,
                              s_eff=s_eff)
    for r in range(2):
        k, j = slide.track(rows_mc[r], rows_c[r], F_LO, T, F_LO, N_B, bank, n_total)
        for n in range(n_t0):
            num, den = 0.0, 0.0
            for s in range(len(k)):
                i = n + (1 if rows_c[r] > 0 else 0) + s
                if i >= n_total:
                    break
                a = slide.amplitude_sq(rows_mc[r], rows_c[r], F_LO, T, s) / s_eff[k[s], j[s]]
                num += a * (cube[k[s], j[s], i] / s_eff[k[s], j[s]] - 2.0) / 2.0
                den += a * a
            want = num / np.sqrt(den) if den > 0 else 0.0
            assert ns[r, n] == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_whitening_moments_and_psd_estimate():
    """After whitening, every segment's values have mean 2 and standard
    deviation 2 exactly (the identity the normalisation builds in); the PSD
    estimate recovers a coloured-noise pattern; a white chi-square cube with
    one louder segment comes back with that segment's scale divided out."""
    r = np.random.default_rng(3)
    K, B, N = 6, 50, 400
    S_true = r.uniform(0.5, 4.0, size=(K, B))
    cube = srs_synth.random_cube(K, B, N, seed=4).astype(np.float64) * S_true[:, :, None]
    cube[:, :, 7] *= 3.0                        # a non-stationary segment
    out, S, mu, sigma = slide.whiten(cube)
    assert np.allclose(out.mean(axis=(0, 1)), 2.0, atol=1e-12)
    assert np.allclose(out.std(axis=(0, 1)), 2.0, rtol=1e-12)
    assert np.median(np.abs(S / S_true - 1.0)) < 0.05
    # segment 7's mean is 3 x 2, up to 4 standard errors of a mean of K B exponentials
    assert abs(mu[7] - 3.0 * np.median(mu)) < 4 * 6.0 / np.sqrt(K * B)
    # a given table is used as is
    out2, S2, _, _ = slide.whiten(cube, s_eff=S_true)
    assert np.array_equal(S2, S_true)
    # with S in the weights only, a white cube and unit weights reduce to the plain statistic
    bank = _bank()
    rows_mc, rows_c = np.array([8e-2]), np.array([0.0])
    cube_w = srs_synth.random_cube(len(bank), N_B, 40, seed=5).astype(np.float64)
    u, _ = slide.stack_slide(cube_w, rows_mc, rows_c, 30, 40, bank, F_LO, T, F_LO, N_B)
    v, _ = slide.stack_slide(cube_w, rows_mc, rows_c, 30, 40, bank, F_LO, T, F_LO, N_B,
                             s_eff=np.ones((len(bank), N_B)), s_eff_in_weights_only=True)
    assert np.allclose(u, v, rtol=1e-12, atol=1e-12)
