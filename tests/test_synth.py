"""The seeded input generators (srs_synth) against the signal model and the
stated recipes: chirp samples against Eq. (phi) evaluated at 40 digits,
coloured noise against its spectral density, the stack-slide rows' t0 step
rule, and the entering injections' ranges.  CPU only."""
import math

import numpy as np
import pytest

import srs_synth


def test_chirp_samples_follow_eq_phi():
    """A cos(phi(t) - phi(t_start) + phi0), phi from Sec. III.A Eq. (phi) with
    its constant, zero before t_start and after coalescence."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    fs, mc, f0, amp, phi0, t_start = 256.0, 0.09, 47.0, 0.7, 0.4, 12.3
    b = srs_synth.chirp_beta(mc, f0)
    t_c = 3.0 / (8.0 * b)
    n = int((t_start + t_c) * fs) + 50
    x = srs_synth.chirp(n, fs, mc, f0, amp, phi0, t_start)
    B, F0 = mpmath.mpf(b), mpmath.mpf(f0)
    phi = lambda t: -6 * mpmath.pi / 5 * F0 * (1 - mpmath.mpf(8) / 3 * B * t) ** (mpmath.mpf(5) / 8) / B
    for j in (int(t_start * fs) + 1, int(t_start * fs) + 777, n // 2, int((t_start + t_c) * fs) - 3):
        t = mpmath.mpf(j) / mpmath.mpf(fs) - mpmath.mpf(t_start)
        want = amp * float(mpmath.cos(phi(t) - phi(0) + phi0))
        assert x[j] == pytest.approx(want, abs=1e-9), j
    assert np.all(x[:int(t_start * fs)] == 0.0)
    assert np.all(x[int((t_start + t_c) * fs) + 2:] == 0.0)


def test_coloured_noise_has_its_spectral_density():
    """Averaged periodograms of 64 s pieces follow asd(f)^2 (white N(0, 1) has
    one-sided density 2 / fs) to a few percent in every 5 Hz band."""
    fs, n = 256.0, 256 * 4096
    asd = lambda f: 0.5 + (np.maximum(np.abs(f), 30.0) / 40.0) ** -2.0
    x = srs_synth.coloured_noise(n, fs, 21, asd)
    seg = int(64 * fs)
    pieces = x[: (n // seg) * seg].reshape(-1, seg)
    pxx = np.mean(np.abs(np.fft.rfft(pieces, axis=1)) ** 2, axis=0) * 2.0 / (fs * seg)
    f = np.fft.rfftfreq(seg, 1.0 / fs)
    for lo in range(10, 120, 5):
        band = (f >= lo) & (f < lo + 5)
        ratio = np.mean(pxx[band]) / np.mean((2.0 / fs) * asd(f[band]) ** 2)
        assert ratio == pytest.approx(1.0, abs=0.05), lo


def test_slide_rows_t0_step_rule():
    """Q steps of t0 per segment for each chirp mass, with one step moving the
    band-edge frequency by at most bin_step bins (df/dt = f beta(Mc, f),
    Sec. III.A Eq. f), and Q the smallest such count."""
    T, f_hi = 30.0, 60.0
    mcs = srs_synth.log_templates(5e-4, 1e-1, 12)
    for step in (1.0, 2.0, 4.0):
        rows_mc, rows_c = srs_synth.slide_rows(mcs, f_hi, T, bin_step=step)
        for mc in mcs:
            c = rows_c[rows_mc == mc]
            Q = c.size
            assert np.allclose(c, np.arange(Q) / Q)
            fdot = f_hi * srs_synth.chirp_beta(mc, f_hi)
            assert fdot * (T / Q) * T <= step * (1 + 1e-12)
            if Q > 1:
                assert fdot * (T / (Q - 1)) * T > step


def test_entering_injections_ranges():
    inj = srs_synth.entering_injections(200, 4, 5e-4, 1e-1, 86400.0, (0.04, 0.08))
    mc = np.array([i["mc"] for i in inj])
    ts = np.array([i["t_start"] for i in inj])
    assert np.all((mc >= 5e-4) & (mc <= 1e-1)) and np.all((ts >= 0) & (ts <= 0.9 * 86400.0))
    assert all(i["f0"] == 40.0 and 0.04 <= i["amp"] <= 0.08 and 0 <= i["phi0"] < 2 * math.pi for i in inj)
    # log-uniform masses: about half below the geometric mean
    assert 0.4 < np.mean(mc < math.sqrt(5e-4 * 1e-1)) < 0.6
    assert srs_synth.entering_injections(5, 4, 5e-4, 1e-1, 86400.0, 0.05) == \
        srs_synth.entering_injections(5, 4, 5e-4, 1e-1, 86400.0, 0.05)
