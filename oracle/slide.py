"""FP64 oracle of the two-stage search: per-segment power cube over a local
0PN resampling bank, then the stack-slide along {Mc, t0} frequency tracks.

TEST INFRASTRUCTURE ONLY (same rule as the rest of `oracle`): tests/,
__graft_entry__.smoke() and bench.py's CPU legs may use it; the library path
never does, and it shares no code with the CUDA path.

Passages followed:
  local_bank   -> Sec. III.B (a bank of 0PN resampling templates placed
                  uniformly in beta; the paper uses 69 over 3e-8..7e-4 1/s)
  power_cube   -> Sec. III.B (segment spectra, each segment resampled with a
                  0PN template that starts at the segment) and Sec. III.C
                  Eq. (normalized_power): P = 2 |F|^2 / n_s for white noise
  track        -> Sec. III.C (the track of theta = {Mc, t0} with f0 at the
                  band's lower edge: frequency f_j and resampling template
                  beta_k in each segment), Sec. III.A Eq. (f), Sec. II Eq. (beta)
  whiten       -> Sec. III.C Eqs. (normalized_power), (semicoherent_statistic)
                  with the effective PSD and the background moments mu_i,
                  sigma_i estimated from the data
  stack_slide  -> Sec. III.C Eqs. (weights), (semicoherent_statistic) with
                  mu = sigma = 2: equal weights w = 1/sqrt(N_seg(theta)), or
                  w proportional to A_i^2 / S_eff (the segment average of the
                  0PN amplitude squared, Sec. II Eq. (h0) h0 ~ f^(2/3), over
                  an effective PSD table; rectangular window, Gamma = 1),
                  normalised so that sum w^2 = 1; powers normalised by S_eff
                  (Eq. (normalized_power))
Readings where the paper leaves a choice (each also listed with the design
notes): the track uses the segments that start at or after t0; its frequency
in a segment is the 0PN frequency at the segment's first sample, rounded to
the nearest bin; the resampling template is the bank entry nearest to the
local chirp parameter beta(Mc, f) there; the track ends at the first segment
whose nearest bin lies above the band, or at the end of the data.
"""
import numpy as np

from . import beta, freq, power, spectra


def local_bank(beta_min, beta_max, n):
    """Sec. III.B: n resampling templates uniform in beta over [beta_min, beta_max]."""
    if n == 1:
        return np.array([float(beta_min)])
    return beta_min + np.arange(n, dtype=np.float64) * ((beta_max - beta_min) / (n - 1))


def power_cube(strain, fs, t_coh, f_lo, n_b, bank, seg_begin, seg_end, n_threads=None):
    """P[k][b][i - seg_begin] = 2 |F_{i,k}(f_b)|^2 / n_s for every bank entry k
    and segment i in [seg_begin, seg_end), each segment resampled with the 0PN
    template beta_k starting at the segment's first sample."""
    K = len(bank)
    n_seg = seg_end - seg_begin
    n_s = int(round(t_coh * fs))
    items = [(k, i) for k in range(K) for i in range(seg_begin, seg_end)]
    F = spectra(strain, fs, t_coh, f_lo, n_b, bank, items, n_threads=n_threads, local=True)
    P = power(F, n_s).reshape(K, n_seg, n_b)
    return np.ascontiguousarray(P.transpose(0, 2, 1))


def first_segment(n, c):
    """Index of the first segment that starts at or after t0 = (n + c) T."""
    return n + (1 if c > 0 else 0)


def track(mc, c, f0, t_coh, f_lo, n_b, bank, n_max):
    """The 0PN track of theta = {Mc, t0 = (n + c) T} (0 <= c < 1), relative to
    its first segment: for the s-th track segment, which starts
    dt_s = (s + [c > 0] - c) T after t0,
      f_s = f(dt_s) by Eq. (f) with beta(Mc, f0) (Eq. (beta)),
      j_s = the nearest bin, rint((f_s - f_lo) T),
      k_s = the bank entry nearest to beta(Mc, f_s).
    The track stops before the first s with j_s > n_b - 1, at coalescence, or
    at s = n_max.  Returns (k [L], j [L]) as int arrays."""
    b0 = beta(mc, f0)
    off = (1.0 if c > 0 else 0.0) - c
    bank = np.asarray(bank, dtype=np.float64)
    ks, js = [], []
    for s in range(n_max):
        dt = (s + off) * t_coh
        if not (1.0 - (8.0 / 3.0) * b0 * dt > 0.0):
            break
        f = freq(b0, f0, dt)
        j = int(np.rint((f - f_lo) * t_coh))
        if j > n_b - 1 or j < 0:
            break
        bl = beta(mc, f)
        ks.append(int(np.argmin(np.abs(bank - bl))))
        js.append(j)
    return np.asarray(ks, dtype=np.int64), np.asarray(js, dtype=np.int64)


def amplitude_sq(mc, c, f0, t_coh, s):
    """Segment average of the squared 0PN amplitude along the track, relative
    to its value at f0 (Sec. II Eq. (h0): h0 ~ f^(2/3), so A^2 ~ f^(4/3)),
    over the s-th track segment [dt_s, dt_s + T): 64-point Gauss-Legendre
    quadrature of (f(t) / f0)^(4/3) by Eq. (f), zero past coalescence."""
    b0 = beta(mc, f0)
    dt = (s + (1.0 if c > 0 else 0.0) - c) * t_coh
    t_c = 3.0 / (8.0 * b0)
    hi = min(dt + t_coh, t_c)
    if hi <= dt:
        return 0.0
    x, wq = np.polynomial.legendre.leggauss(64)
    t = dt + (x + 1.0) * 0.5 * (hi - dt)
    f = np.array([freq(b0, f0, v) for v in t])
    return float(np.sum(wq * (f / f0) ** (4.0 / 3.0)) * 0.5 * (hi - dt) / t_coh)


def n_sigma_track(P_track):
    """Eq. (semicoherent_statistic) over one track's powers with w = 1/sqrt(N)
    (so sum w^2 = 1) and mu = sigma = 2; 0 for an empty track."""
    P_track = np.asarray(P_track, dtype=np.float64)
    n = P_track.size
    if n == 0:
        return 0.0
    return float(np.sum((P_track - 2.0) / 2.0) / np.sqrt(n))


def n_sigma_weighted(P_track, a, s_eff_track):
    """Eq. (semicoherent_statistic) with weights w_s = a_s / sqrt(sum a_s^2)
    (Eq. (weights) normalised), a_s = A_s^2 / S_s, and powers normalised by
    the effective PSD S_s (relative to white unit-variance noise):
    sum_s w_s (P_s / S_s - 2) / 2.  0 for an empty track."""
    P = np.asarray(P_track, dtype=np.float64)
    if P.size == 0:
        return 0.0
    S = np.asarray(s_eff_track, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64) / S
    return float(np.sum(a * (P / S - 2.0) / 2.0) / np.sqrt(np.sum(a * a)))


def whiten(cube, s_eff=None):
    """Normalise a power cube P[k][j][i] for coloured, non-stationary noise
    (Sec. III.C Eqs. (normalized_power), (semicoherent_statistic)):
      S[k][j] = mean_i P[k][j][i] / 2 (white unit-variance noise gives
                E[P] = 2), or the given table;
      Pt = P / S;  mu_i, sigma_i = mean and (population) standard deviation
                of Pt over all (k, j) of segment i;
      out = 2 + 2 (Pt - mu_i) / sigma_i,
    so that (out - 2) / 2 = (Pt - mu_i) / sigma_i, the term of Eq.
    (semicoherent_statistic) with empirical moments.  Returns (out, S, mu,
    sigma)."""
    P = np.asarray(cube, dtype=np.float64)
    S = P.mean(axis=2) / 2.0 if s_eff is None else np.asarray(s_eff, dtype=np.float64)
    Pt = P / S[:, :, None]
    mu = Pt.mean(axis=(0, 1))
    sigma = Pt.std(axis=(0, 1))
    return 2.0 + 2.0 * (Pt - mu) / sigma, S, mu, sigma


def stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, f0, t_coh, f_lo, n_b, with_abs=False,
                weighting=0, s_eff=None, s_eff_in_weights_only=False):
    """n_sigma[r][n] for theta = {rows_mc[r], t0 = (n + rows_c[r]) T} over a
    cube P[k][j][i] that holds every segment i < n_total.  weighting 0: equal
    weights; 1: amplitude weights (amplitude_sq).  s_eff: [n_beta][n_bins]
    effective PSD relative to white noise, or None (white); with
    s_eff_in_weights_only the cube is already normalised by it (whiten) and
    s_eff enters the weights alone.  Also returns the
    number of track segments N_seg[r][n] inside the data, and with
    with_abs=True a bound helper: the sum over the track of
    (|a P / S| + |2 a|) / 2 / sqrt(sum a^2)."""
    R = len(rows_mc)
    out = np.zeros((R, n_t0))
    nseg = np.zeros((R, n_t0), dtype=np.int64)
    absum = np.zeros((R, n_t0))
    for r in range(R):
        k, j = track(rows_mc[r], rows_c[r], f0, t_coh, f_lo, n_b, bank, n_total)
        amp = (np.array([amplitude_sq(rows_mc[r], rows_c[r], f0, t_coh, s) for s in range(len(k))])
               if weighting else np.ones(len(k)))
        S_all = s_eff[k, j] if s_eff is not None else np.ones(len(k))
        for n in range(n_t0):
            first = first_segment(n, rows_c[r])
            L = max(0, min(len(k), n_total - first))
            i = first + np.arange(L)
            P = cube[k[:L], j[:L], i]
            if weighting or s_eff is not None:
                if s_eff_in_weights_only:
                    a = amp[:L] / S_all[:L]
                    out[r, n] = n_sigma_weighted(P, a, np.ones(L))
                else:
                    out[r, n] = n_sigma_weighted(P, amp[:L], S_all[:L])
            else:
                out[r, n] = n_sigma_track(P)
            nseg[r, n] = L
            if L:
                a = amp[:L] / S_all[:L]
                Pn = np.asarray(P, dtype=np.float64) / (1.0 if s_eff_in_weights_only else S_all[:L])
                absum[r, n] = float(np.sum(np.abs(a * Pn) + 2 * np.abs(a)) / 2.0 / np.sqrt(np.sum(a * a)))
    if with_abs:
        return out, nseg, absum
    return out, nseg
