"""FP64 CPU oracle for the semicoherent NUFFT resampling search (arXiv:2609.12476).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package; the library path never
does.  It shares no code with the CUDA path.

Each function states the passage of the paper it follows:
  beta, duration, freq, tau, delta, nseg -> Sec. II Eq. (beta), Sec. III.A Eq. (f),
                                             Sec. III.B Eq. (new_t), Sec. V
  spectra                                -> Sec. III.B (the transform a type-1 NUFFT
                                             approximates), direct non-uniform DFT
  power                                  -> Sec. III.C Eq. (normalized_power)
  semicoherent / n_sigma                 -> Sec. III.C Eqs. (weights),
                                             (semicoherent_statistic)
  topk                                   -> ordering (n_sigma desc, template asc, bin asc)
The learned-proposal reference (MLP forward/backward) lives in oracle.mlp, the
two-stage search (power cube, tracks, stack-slide) in oracle.slide, and the
detection thresholds in oracle.stats.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def load(path):
    """Load an oracle library built from srs_oracle.c and declare its functions."""
    L = ctypes.CDLL(path)
    d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
    if True:
        P = ctypes.c_void_p
        L.orc_beta.restype = d; L.orc_beta.argtypes = [d, d]
        L.orc_duration.restype = d; L.orc_duration.argtypes = [d, d, d]
        L.orc_freq.restype = d; L.orc_freq.argtypes = [d, d, d]
        L.orc_tau.restype = d; L.orc_tau.argtypes = [d, d]
        L.orc_delta.restype = d; L.orc_delta.argtypes = [d, d, d]
        L.orc_nseg.restype = i32; L.orc_nseg.argtypes = [d, d, d, d, i32, ctypes.c_int]
        L.orc_spectra.restype = ctypes.c_int
        L.orc_spectra.argtypes = [P, i64, d, d, d, i32, P, P, P, i32, ctypes.c_int, P, P]
        L.orc_spectra_ex.restype = ctypes.c_int
        L.orc_spectra_ex.argtypes = [P, i64, d, d, d, i32, P, P, P, i32, ctypes.c_int, ctypes.c_int, P, P]
    return L


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load(_build.build())
    return _LIB


def beta(mc_msun, f0):
    """Sec. II Eq. (beta): chirp parameter beta(f0, Mc) in 1/s."""
    return lib().orc_beta(float(mc_msun), float(f0))


def duration(beta_, f0, f_end):
    """Sec. II: 0PN time from f0 to f_end."""
    return lib().orc_duration(float(beta_), float(f0), float(f_end))


def freq(beta_, f0, t):
    """Sec. III.A Eq. (f): 0PN frequency at time t (t0 = 0)."""
    return lib().orc_freq(float(beta_), float(f0), float(t))


def tau(beta_, t):
    """Sec. III.B Eq. (new_t), literal form (t0 = 0)."""
    return lib().orc_tau(float(beta_), float(t))


def delta(beta_, t_i0, s):
    """Segment-local resampled time tau(t_i0 + s) - tau(t_i0), Eq. (new_t) without
    the constant offset.  Vectorised over s."""
    L = lib()
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    return np.array([L.orc_delta(float(beta_), float(t_i0), float(v)) for v in s])


def nseg(beta_, f_ref, f_hi, t_coh, n_total, cut=True):
    """Whole segments the template track spends in band (Sec. II duration, Sec. V)."""
    return int(lib().orc_nseg(float(beta_), float(f_ref), float(f_hi), float(t_coh),
                              int(n_total), 1 if cut else 0))


def spectra(strain, fs, t_coh, f_lo, n_b, betas, items, n_threads=None, local=False):
    """Direct non-uniform DFT F(f_b) = sum_j x_j exp(-2 pi i f_b delta_j) for each
    (template m, segment i) in `items`; f_b = f_lo + b / t_coh.  Returns complex
    array [len(items), n_b].  local=True resamples every segment with a 0PN
    template that starts at the segment's first sample (delta_j = tau(s_j) -
    tau(0) with beta_m), the per-segment form of Sec. III.C's stack-slide."""
    strain = np.ascontiguousarray(strain, dtype=np.float64)
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    items = np.asarray(items, dtype=np.int32).reshape(-1, 2)
    im_ = np.ascontiguousarray(items[:, 0]); ii_ = np.ascontiguousarray(items[:, 1])
    n = items.shape[0]
    re = np.zeros((n, n_b)); im = np.zeros((n, n_b))
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    rc = lib().orc_spectra_ex(strain.ctypes.data, strain.size, float(fs), float(t_coh), float(f_lo),
                              int(n_b), betas.ctypes.data, im_.ctypes.data, ii_.ctypes.data, n,
                              int(n_threads), 1 if local else 0, re.ctypes.data, im.ctypes.data)
    if rc != 0:
        raise ValueError("oracle: bad arguments to spectra")
    return re + 1j * im


def power(F, n_s):
    """Sec. III.C Eq. (normalized_power) for white unit-variance noise sampled at fs:
    x~ = F / fs and S_eff = 2 / fs give P = 4 |x~|^2 / (T S_eff) = 2 |F|^2 / n_s."""
    return 2.0 * np.abs(F) ** 2 / n_s


def n_sigma(S, nseg_):
    """Sec. III.C Eq. (semicoherent_statistic) with equal weights w = 1/sqrt(N_seg)
    (so sum w^2 = 1) and mu = sigma = 2: n_sigma = (S - 2 N) / (2 sqrt(N))."""
    nseg_ = np.asarray(nseg_, dtype=np.float64).reshape(-1, 1)
    return (S - 2.0 * nseg_) / (2.0 * np.sqrt(nseg_))


def semicoherent(strain, fs, t_coh, f_lo, n_b, betas, nsegs, n_threads=None):
    """Sum of powers over each template's first N_seg(m) segments: S[m][b], and the
    n_sigma map.  Computes every (m, i) spectrum, so keep it to small inputs."""
    n_s = int(round(t_coh * fs))
    items = [(m, i) for m in range(len(betas)) for i in range(int(nsegs[m]))]
    F = spectra(strain, fs, t_coh, f_lo, n_b, betas, items, n_threads)
    P = power(F, n_s)
    S = np.zeros((len(betas), n_b))
    for k, (m, _i) in enumerate(items):
        S[m] += P[k]
    return S, n_sigma(S, nsegs)


def topk(stat_map, k):
    """The k largest entries of a [templates, bins] map, ordered by value
    descending, then template ascending, then bin ascending.  Returns
    (values, template_idx, bin) arrays."""
    stat_map = np.asarray(stat_map)
    M, B = stat_map.shape
    mm, bb = np.meshgrid(np.arange(M), np.arange(B), indexing="ij")
    order = np.lexsort((bb.ravel(), mm.ravel(), -stat_map.ravel()))[:k]
    return stat_map.ravel()[order], mm.ravel()[order], bb.ravel()[order]
