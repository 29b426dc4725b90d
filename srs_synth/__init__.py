"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module only makes data: Gaussian noise, Newtonian (0PN) chirps injected
into it, and template lists.  It holds none of the search's arithmetic (no
resampling, transform, power or statistic), so it can feed both the CUDA path
and the oracle without tying them together.

The chirp follows the paper's signal model: Sec. III.A Eq. (f) for the
frequency and Eq. (phi) for the phase, with the chirp parameter of Sec. II
Eq. (beta).  The phase is written with its constant removed
(phi(t) - phi(0)), which only shifts phi0.

Workload shapes (30 s segments, 40-60 Hz band, chirp masses 5e-4..1e-1 Msun)
follow the paper's search (abstract, Sec. III.C, Sec. IV).
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

# G*Msun / c^3 in seconds (IAU nominal G*Msun = 1.32712440018e20 m^3/s^2).
_GMSUN_C3 = 1.32712440018e20 / 299792458.0 ** 3


def chirp_beta(mc_msun, f0):
    """Sec. II Eq. (beta): chirp rate parameter for chirp mass mc at frequency f0."""
    return (96.0 / 5.0) * math.pi ** (8.0 / 3.0) * (_GMSUN_C3 * mc_msun) ** (5.0 / 3.0) * f0 ** (8.0 / 3.0)


def mc_for_beta(beta, f0):
    """Inverse of chirp_beta in mc at fixed f0."""
    k = (96.0 / 5.0) * math.pi ** (8.0 / 3.0) * _GMSUN_C3 ** (5.0 / 3.0) * f0 ** (8.0 / 3.0)
    return (beta / k) ** 0.6


def white_noise(n, seed, dtype=np.float64):
    """n samples of N(0, 1) from numpy's PCG64 stream `seed`."""
    return np.random.default_rng(seed).standard_normal(n).astype(dtype, copy=False)


def coloured_noise(n, fs, seed, asd):
    """n samples of stationary Gaussian noise with amplitude spectral density
    proportional to asd(f) (a callable on an array of frequencies in Hz),
    scaled to unit variance at the asd's value 1: white N(0, 1) noise from
    PCG64 stream `seed`, shaped in the frequency domain."""
    x = white_noise(n, seed)
    X = np.fft.rfft(x)
    f = np.fft.rfftfreq(n, 1.0 / fs)
    return np.fft.irfft(X * np.asarray(asd(f), dtype=np.float64), n)


def chirp(n, fs, mc_msun, f0, amp, phi0=0.0, t_start=0.0):
    """A cos(phi(t)) for t = t_start + j/fs, j < n, zero before t_start.

    phi(t) - phi0 = 2 pi f0 * (3 / (5 beta)) * (1 - (1 - (8/3) beta (t - t_start))^(5/8))
    (Eq. (phi) minus its value at t_start); zero after coalescence."""
    out = np.zeros(n)
    add_chirp(out, fs, mc_msun, f0, amp, phi0, t_start)
    return out


def add_chirp(out, fs, mc_msun, f0, amp, phi0=0.0, t_start=0.0, j_first=0):
    """out[j] += chirp sample j_first + j, evaluated only over the samples where
    the chirp is live (the same values as chirp's, sample by sample)."""
    n = out.size
    beta = chirp_beta(mc_msun, f0)
    j0 = min(n, max(0, int(np.floor(t_start * fs)) - 1 - j_first))
    t_end = t_start + 3.0 / (8.0 * beta)
    j1 = n if not np.isfinite(t_end) or t_end * fs + 2 - j_first >= n else \
        min(n, max(j0, int(np.ceil(t_end * fs)) + 2 - j_first))
    t = np.arange(j_first + j0, j_first + j1, dtype=np.float64) / fs - t_start
    x = (8.0 / 3.0) * beta * t
    live = (t >= 0) & (x < 1.0)
    core = -np.expm1(0.625 * np.log1p(-x[live]))
    phase = 2.0 * np.pi * f0 * (3.0 / (5.0 * beta)) * core + phi0
    seg = out[j0:j1]
    seg[live] += amp * np.cos(phase)


def log_templates(mc_lo, mc_hi, count):
    """count chirp masses log-spaced over [mc_lo, mc_hi]."""
    if count == 1:
        return np.array([float(mc_lo)])
    return np.exp(np.linspace(np.log(mc_lo), np.log(mc_hi), count))


def strain_with_chirps(n, fs, seed, injections, dtype=np.float64, noise=True):
    """Noise (seed) plus the listed chirps; each injection is a dict with keys
    mc, f0, amp and optionally phi0, t_start."""
    x = white_noise(n, seed) if noise else np.zeros(n)
    block = 1 << 20

    def fill(j):                    # every chirp, in order, over samples [j, j + block)
        v = x[j:j + block]
        for inj in injections:
            add_chirp(v, fs, inj["mc"], inj["f0"], inj["amp"], inj.get("phi0", 0.0), inj.get("t_start", 0.0), j)

    if injections:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as pool:
            list(pool.map(fill, range(0, n, block)))
    return x.astype(dtype, copy=False)


def random_injections(count, seed, mc_lo, mc_hi, f_lo, f_hi, amp):
    """count injections: chirp mass log-uniform in [mc_lo, mc_hi], f0 uniform in
    [f_lo, f_hi), phi0 uniform in [0, 2 pi); amp a number or a (lo, hi) pair for
    a uniform draw."""
    r = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        a = amp if np.isscalar(amp) else r.uniform(amp[0], amp[1])
        out.append({"mc": float(np.exp(r.uniform(np.log(mc_lo), np.log(mc_hi)))),
                    "f0": float(r.uniform(f_lo, f_hi)), "amp": float(a),
                    "phi0": float(r.uniform(0, 2 * np.pi))})
    return out


# Workloads of the paper's search shape (T_coh = 30 s, 40-60 Hz).
WORKLOADS = {
    # single segment, single exact template, full mode set at 128 Hz
    "single": dict(fs=128.0, t_obs=30.0, t_coh=30.0, f_lo=-64.0, f_hi=64.0, f_ref=50.0,
                   mc=[1e-2], eps=1e-9, seed=0, dtype="f64",
                   injections=[{"mc": 1e-2, "f0": 50.0, "amp": 0.5}]),
    # 2 h, 64 templates 2e-2..5e-2, one loud chirp
    "semicoherent_2h": dict(fs=256.0, t_obs=7200.0, t_coh=30.0, f_lo=40.0, f_hi=60.0, f_ref=40.0,
                            mc=("log", 2e-2, 5e-2, 64), eps=1e-6, seed=0, dtype="f64", top_k=32,
                            injections=[{"mc": 3e-2, "f0": 45.0, "amp": 0.05}]),
    # 6 h, 1024 templates 5e-4..1e-1, 8 injections
    "batched_6h": dict(fs=256.0, t_obs=21600.0, t_coh=30.0, f_lo=40.0, f_hi=60.0, f_ref=40.0,
                       mc=("log", 5e-4, 1e-1, 1024), eps=1e-6, seed=0, dtype="f64", top_k=32,
                       injections=("random", 8, 1, 0.05)),
    # 24 h float32, 4096 templates, 64 injections
    "large_24h": dict(fs=256.0, t_obs=86400.0, t_coh=30.0, f_lo=40.0, f_hi=60.0, f_ref=40.0,
                      mc=("log", 5e-4, 1e-1, 4096), eps=1e-6, seed=0, dtype="f32", top_k=32,
                      injections=("random", 64, 1, 0.05)),
}


def slide_rows(mc_list, f_hi, t_coh, bin_step=1.0):
    """Rows of a stack-slide template grid theta = {Mc, t0}: for each chirp mass,
    t0 fractions c = q / Q (q < Q) of a segment, with Q chosen so that moving t0
    by T / Q moves the band-edge frequency f_hi by at most bin_step bins:
    Q = max(1, ceil(fdot(f_hi) T^2 / bin_step)), fdot(f) = f beta(Mc, f).
    Returns (mc [R], c [R]) float arrays."""
    mcs, cs = [], []
    for mc in np.asarray(mc_list, dtype=np.float64):
        fdot = f_hi * chirp_beta(float(mc), f_hi)
        q_n = max(1, int(math.ceil(fdot * t_coh * t_coh / bin_step)))
        for q in range(q_n):
            mcs.append(float(mc))
            cs.append(q / q_n)
    return np.asarray(mcs), np.asarray(cs)


def random_cube(n_beta, n_bins, n_seg, seed):
    """A power cube [n_beta][n_bins][n_seg] float32 of independent chi-square
    (2 degrees of freedom) draws, the distribution of P = 2 |F|^2 / n_s for
    white unit-variance noise (mean 2), from numpy's PCG64 stream `seed`."""
    r = np.random.default_rng(seed)
    return r.exponential(2.0, size=(n_beta, n_bins, n_seg)).astype(np.float32)


# Two-stage (cube + stack-slide) workloads: the local resampling bank of the
# paper (69 templates uniform in beta over 3e-8..7e-4 1/s), tracks entering
# the band at f0 = 40 Hz at t0.
SLIDE_WORKLOADS = {
    # 6 h float64, 48 chirp masses 5e-4..1e-1, 4 chirps entering the band after t = 0
    "stackslide_6h": dict(fs=256.0, t_obs=21600.0, t_coh=30.0, f_lo=40.0, f_hi=60.0, eps=1e-6,
                          seed=0, dtype="f64", top_k=32, bank=(3e-8, 7e-4, 69),
                          mc=("log", 5e-4, 1e-1, 48), bin_step=1.0,
                          injections=[{"mc": 2e-2, "t_start": 3000.0, "amp": 0.06},
                                      {"mc": 6e-2, "t_start": 9015.0, "amp": 0.06},
                                      {"mc": 3e-3, "t_start": 600.0, "amp": 0.03},
                                      {"mc": 9e-2, "t_start": 15012.0, "amp": 0.08}]),
    # 24 h float32, 256 chirp masses 5e-4..1e-1, 16 chirps entering at random times
    "stackslide_24h": dict(fs=256.0, t_obs=86400.0, t_coh=30.0, f_lo=40.0, f_hi=60.0, eps=1e-6,
                           seed=0, dtype="f32", top_k=32, bank=(3e-8, 7e-4, 69),
                           mc=("log", 5e-4, 1e-1, 256), bin_step=1.0,
                           injections=("entering", 16, 2, (0.04, 0.08))),
}


def entering_injections(count, seed, mc_lo, mc_hi, t_obs, amp, f0=40.0):
    """count chirps that enter the band at f0 at a time t_start uniform over the
    first 90% of the data; chirp mass log-uniform, phi0 uniform, amp a number or
    a (lo, hi) pair."""
    r = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        a = amp if np.isscalar(amp) else r.uniform(amp[0], amp[1])
        out.append({"mc": float(np.exp(r.uniform(np.log(mc_lo), np.log(mc_hi)))), "f0": f0,
                    "t_start": float(r.uniform(0.0, 0.9 * t_obs)), "amp": float(a),
                    "phi0": float(r.uniform(0, 2 * np.pi))})
    return out


def make_slide_workload(name, **over):
    """Materialise a two-stage workload: strain, bank bounds, stack-slide rows
    (mc, c) and the search parameters."""
    w = dict(SLIDE_WORKLOADS[name]); w.update(over)
    n = int(round(w["t_obs"] * w["fs"]))
    mc = w["mc"]
    if isinstance(mc, tuple) and mc[0] == "log":
        mc = log_templates(mc[1], mc[2], mc[3])
    mc = np.asarray(mc, dtype=np.float64)
    inj = w["injections"]
    if isinstance(inj, tuple) and inj[0] == "entering":
        inj = entering_injections(inj[1], inj[2], 5e-4, 1e-1, w["t_obs"], inj[3], w["f_lo"])
    inj = [dict(i, f0=i.get("f0", w["f_lo"])) for i in inj]
    dtype = np.float32 if w["dtype"] == "f32" else np.float64
    x = strain_with_chirps(n, w["fs"], w["seed"], inj, dtype=dtype)
    rows_mc, rows_c = slide_rows(mc, w["f_hi"], w["t_coh"], w["bin_step"])
    w.update(strain=x, mc=mc, injections=inj, n_samples=n, rows_mc=rows_mc, rows_c=rows_c,
             n_total=n // int(round(w["t_coh"] * w["fs"])))
    return w


def make_workload(name, **over):
    """Materialise a named workload: returns dict with strain (numpy), mc list
    and the search parameters."""
    w = dict(WORKLOADS[name]); w.update(over)
    n = int(round(w["t_obs"] * w["fs"]))
    mc = w["mc"]
    if isinstance(mc, tuple) and mc[0] == "log":
        mc = log_templates(mc[1], mc[2], mc[3])
    mc = np.asarray(mc, dtype=np.float64)
    inj = w["injections"]
    if isinstance(inj, tuple) and inj[0] == "random":
        inj = random_injections(inj[1], inj[2], 5e-4, 1e-1, w["f_lo"], w["f_hi"], inj[3])
    dtype = np.float32 if w["dtype"] == "f32" else np.float64
    x = strain_with_chirps(n, w["fs"], w["seed"], inj, dtype=dtype)
    w.update(strain=x, mc=mc, injections=inj, n_samples=n)
    return w
