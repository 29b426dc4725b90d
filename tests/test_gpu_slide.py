"""GPU parity of the two-stage search (power cube + stack-slide) against the
FP64 oracle (oracle.slide), through the C ABI.

Tolerances: cube powers within the bound that rel-L2(F) <= 10 eps per
spectrum implies, |dP_b| <= (4 |F_b| d + 2 d^2) / n_s with d = 10 eps ||F||;
stack-slide sums on a given cube within the FP32 summation bound
(L + 2) u sum_s (|a_s P_s / S_s| + 2 |a_s|) / 2 / sqrt(sum a^2) (u = 2^-24, L
track segments; the FMA coefficients are FP32 too) plus the final scaling;
end-to-end n_sigma within the sum of both over the track."""
import numpy as np
import pytest

import oracle
import srs_synth
from oracle import slide
from paper_2609_12476_gb300 import SRS_WEIGHT_AMPLITUDE, Context, Params, SrsError

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FS, T, F_LO, F_HI = 256.0, 30.0, 40.0, 60.0
N_B, N_S = 600, 7680
BANK = (3e-8, 7e-4, 69)
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def _params(**kw):
    return Params(fs=FS, t_coh=T, f_lo=F_LO, f_hi=F_HI, eps=1e-6, top_k=kw.pop("top_k", 32), **kw)


def _p_bound(F, eps):
    """Per-bin |dP| bound from rel-L2(F) <= 10 eps (F: complex [..., n_b])."""
    d = 10 * eps * np.linalg.norm(F, axis=-1, keepdims=True)
    return (4 * np.abs(F) * d + 2 * d ** 2) / N_S


@pytest.fixture(scope="module")
def strain_2h():
    # on the end-to-end test's template grid: its fifth chirp mass, entering at segment 50
    inj = [{"mc": float(srs_synth.log_templates(3e-2, 8e-2, 9)[4]), "f0": F_LO, "amp": 0.08, "t_start": 1500.0,
            "phi0": 0.3}]
    return srs_synth.strain_with_chirps(int(7200 * FS), FS, 7, inj), inj


def test_power_cube_matches_oracle(ctx, strain_2h):
    x, _ = strain_2h
    p = _params()
    bank = slide.local_bank(*BANK)
    cube, rep = ctx.power_cube(x, BANK, 100, 103, p)
    assert cube.shape == (69, N_B, 3) and rep["kernel_launches"] >= 1
    items = [(k, i) for k in range(69) for i in range(100, 103)]
    F = oracle.spectra(x, FS, T, F_LO, N_B, bank, items, local=True).reshape(69, 3, N_B)
    P = oracle.power(F, N_S).transpose(0, 2, 1)
    tol = _p_bound(F, 1e-6).transpose(0, 2, 1) + 1e-6 * P + 1e-6
    err = np.abs(cube - P)
    assert np.all(err <= tol), float(np.max(err / tol))
    # device I/O, the first segments (ragged chunk of one) and the same values
    xd = torch.from_numpy(x).cuda()
    cd, _ = ctx.power_cube(xd, BANK, 101, 102, p)
    assert np.allclose(cd.cpu().numpy()[:, :, 0], cube[:, :, 1], rtol=1e-5, atol=1e-4)
    c0, _ = ctx.power_cube(x, BANK, 0, 1, p)
    F0 = oracle.spectra(x, FS, T, F_LO, N_B, bank[[0, 68]], [(0, 0), (1, 0)], local=True)
    P0 = oracle.power(F0, N_S)
    assert np.all(np.abs(c0[[0, 68], :, 0] - P0) <= _p_bound(F0, 1e-6) + 1e-6 * P0 + 1e-6)


def _random_case(n_total=240, seed=11):
    bank = slide.local_bank(*BANK)
    cube = srs_synth.random_cube(69, N_B, n_total, seed)
    mc = srs_synth.log_templates(5e-4, 1e-1, 12)
    rows_mc, rows_c = srs_synth.slide_rows(mc, F_HI, T, bin_step=4.0)
    return bank, cube, rows_mc, rows_c


def _slide_tol(L, absum, ref):
    return (np.asarray(L, dtype=np.float64) + 2) * U32 * absum + 4 * U32 * np.abs(ref) + 1e-6


def test_stack_slide_matches_oracle_on_a_random_cube(ctx):
    bank, cube, rows_mc, rows_c = _random_case()
    n_total = cube.shape[2]
    n_t0 = n_total
    ref, L, absum = slide.stack_slide(cube, rows_mc, rows_c, n_t0, n_total, bank, F_LO, T, F_LO, N_B,
                                      with_abs=True)
    cands, m, rep = ctx.stack_slide(cube, 0, n_total, BANK, rows_mc, rows_c, n_t0, _params())
    err = np.abs(m - ref)
    tol = _slide_tol(L, absum, ref)
    assert np.all(err <= tol), float(np.max(err / tol))
    assert np.all(m[L == 0] == 0.0)
    # candidates: the largest cells of the returned map, (value desc, row asc, column asc)
    v, rr, nn = oracle.topk(m, 32)
    assert np.array_equal(cands["template_idx"], rr) and np.array_equal(cands["bin"], nn)
    assert np.array_equal(cands["value"], v.astype(np.float32))
    assert rep["slide_ms"] > 0


def test_weighted_stack_slide_matches_oracle(ctx):
    """Amplitude weights (segment-averaged f^(4/3)) over a seeded effective-PSD
    table, on a seeded chi-square cube, against the oracle."""
    bank, cube, rows_mc, rows_c = _random_case(n_total=160, seed=21)
    n_total = cube.shape[2]
    s_eff = np.random.default_rng(8).uniform(0.5, 3.0, size=(69, N_B)).astype(np.float32)
    ref, L, absum = slide.stack_slide(cube, rows_mc, rows_c, 120, n_total, bank, F_LO, T, F_LO, N_B,
                                      with_abs=True, weighting=1, s_eff=s_eff.astype(np.float64))
    cands, m, _ = ctx.stack_slide(cube, 0, n_total, BANK, rows_mc, rows_c, 120, _params(),
                                  weighting=SRS_WEIGHT_AMPLITUDE, s_eff=s_eff)
    err = np.abs(m - ref)
    tol = _slide_tol(L, absum, ref)
    assert np.all(err <= tol), float(np.max(err / tol))
    v, rr, nn = oracle.topk(m, 32)
    assert np.array_equal(cands["template_idx"], rr) and np.array_equal(cands["bin"], nn)
    # equal weights over a white table are the unweighted statistic
    _, m0, _ = ctx.stack_slide(cube, 0, n_total, BANK, rows_mc, rows_c, 120, _params())
    _, m1, _ = ctx.stack_slide(cube, 0, n_total, BANK, rows_mc, rows_c, 120, _params(),
                               s_eff=np.ones((69, N_B), np.float32))
    assert np.allclose(m0, m1, rtol=1e-6, atol=1e-6)


def test_stack_slide_chunks_carry_partial_sums(ctx):
    """The running sums carried between cube chunks (Sec. VI partial sums)
    give the one-pass result; a chunk without FIRST needs an open search."""
    bank, cube, rows_mc, rows_c = _random_case(n_total=200, seed=3)
    n_total = cube.shape[2]
    cd = torch.from_numpy(cube).cuda()
    p = _params()
    c1, m1, _ = ctx.stack_slide(cd, 0, n_total, BANK, rows_mc, rows_c, 150, p)
    bounds = [0, 77, 78, 140, 200]
    for q in range(len(bounds) - 1):
        a, b = bounds[q], bounds[q + 1]
        out = ctx.stack_slide(cd[:, :, a:b].contiguous(), a, n_total, BANK, rows_mc, rows_c, 150, p,
                              first=(q == 0), last=(q == len(bounds) - 2))
    c2, m2, _ = out
    m1h, m2h = m1.cpu().numpy(), m2.cpu().numpy()
    ref, L, absum = slide.stack_slide(cube, rows_mc, rows_c, 150, n_total, bank, F_LO, T, F_LO, N_B, with_abs=True)
    tol = 2 * _slide_tol(L, absum, ref)
    assert np.all(np.abs(m2h - m1h) <= tol)
    assert np.all(np.abs(m2h - ref) <= tol)
    with pytest.raises(SrsError):
        ctx.stack_slide(cd[:, :, 0:10].contiguous(), 0, n_total, BANK, rows_mc, rows_c, 150, p, first=False,
                        last=True)


def _track_nsigma(x, mc, c, n, n_total, bank, eps=1e-6, weighting=0):
    """Oracle n_sigma of one template from its track's spectra, with the
    tolerance those spectra's error bound implies."""
    k, j = slide.track(mc, c, F_LO, T, F_LO, N_B, bank, n_total)
    first = slide.first_segment(n, c)
    L = max(0, min(len(k), n_total - first))
    if L == 0:
        return 0.0, 1e-6, 0
    items = [(int(k[s]), first + s) for s in range(L)]
    F = oracle.spectra(x, FS, T, F_LO, N_B, bank, items, local=True)
    Fj = F[np.arange(L), j[:L]]
    P = oracle.power(Fj, N_S)
    dP = _p_bound(F, eps)[np.arange(L), j[:L]]
    a = (np.array([slide.amplitude_sq(mc, c, F_LO, T, s) for s in range(L)]) if weighting else np.ones(L))
    norm = np.sqrt(np.sum(a * a))
    ref = slide.n_sigma_weighted(P, a, np.ones(L)) if weighting else slide.n_sigma_track(P)
    absum = np.sum(a * (np.abs(P) + 2.0)) / 2.0 / norm
    tol = np.sum(a * dP) / (2 * norm) + (L + 2) * U32 * absum + 1e-5 * abs(ref) + 1e-5
    return ref, tol, L


def test_slide_search_end_to_end(ctx, strain_2h):
    x, inj = strain_2h
    bank = slide.local_bank(*BANK)
    n_total = x.size // N_S
    mc = srs_synth.log_templates(3e-2, 8e-2, 9)
    rows_mc, rows_c = srs_synth.slide_rows(mc, F_HI, T, bin_step=1.0)
    n_t0 = n_total
    cands, m, rep = ctx.slide_search(x, BANK, rows_mc, rows_c, n_t0, _params())
    assert m.shape == (rows_mc.size, n_t0)
    assert rep["n_spectra"] == 69 * n_total and rep["slide_ms"] > 0 and rep["spread_ms"] > 0
    # the entering chirp is the loudest template, at its chirp mass and entry time
    r, n = int(cands["template_idx"][0]), int(cands["bin"][0])
    t0 = (n + rows_c[r]) * T
    assert abs(np.log(rows_mc[r] / inj[0]["mc"])) < 0.15 and abs(t0 - inj[0]["t_start"]) <= T, (r, n, rows_mc[r], t0)
    assert cands["value"][0] > 20
    v, rr, nn = oracle.topk(m, 32)
    assert np.array_equal(cands["template_idx"], rr) and np.array_equal(cands["bin"], nn)
    # the power reads the library reports are the oracle tracks' segments inside the data
    reads = 0
    for r_ in range(rows_mc.size):
        k, _ = slide.track(rows_mc[r_], rows_c[r_], F_LO, T, F_LO, N_B, bank, n_total)
        first = np.arange(n_t0) + (1 if rows_c[r_] > 0 else 0)
        reads += int(np.sum(np.clip(np.minimum(len(k), n_total - first), 0, None)))
    assert rep["slide_reads"] == reads
    # sampled templates against the oracle: the winner, a quiet one, one cut by the data's end
    rng = np.random.default_rng(1)
    picks = [(r, n), (int(rng.integers(rows_mc.size)), int(rng.integers(n_t0))), (0, n_t0 - 3)]
    for r_, n_ in picks:
        ref, tol, L = _track_nsigma(x, rows_mc[r_], rows_c[r_], n_, n_total, bank)
        assert abs(m[r_, n_] - ref) <= tol, (r_, n_, L, m[r_, n_], ref, tol)


def test_weighted_slide_search_end_to_end(ctx, strain_2h):
    """Amplitude weights in the whole search: the entering chirp is still the
    loudest template, and sampled templates match the weighted oracle."""
    x, inj = strain_2h
    bank = slide.local_bank(*BANK)
    n_total = x.size // N_S
    rows_mc, rows_c = srs_synth.slide_rows(srs_synth.log_templates(3e-2, 8e-2, 9), F_HI, T, bin_step=1.0)
    cands, m, _ = ctx.slide_search(x, BANK, rows_mc, rows_c, n_total, _params(), weighting=SRS_WEIGHT_AMPLITUDE)
    r, n = int(cands["template_idx"][0]), int(cands["bin"][0])
    assert abs(np.log(rows_mc[r] / inj[0]["mc"])) < 0.15 and abs((n + rows_c[r]) * T - inj[0]["t_start"]) <= T
    for r_, n_ in [(r, n), (3, 17), (len(rows_mc) - 1, n_total - 5)]:
        ref, tol, L = _track_nsigma(x, rows_mc[r_], rows_c[r_], n_, n_total, bank, weighting=1)
        assert abs(m[r_, n_] - ref) <= tol, (r_, n_, L, m[r_, n_], ref, tol)


def test_slide_search_under_a_cube_budget(ctx, strain_2h):
    """A device cube budget of 37 segments (7 chunks, partial sums carried)
    gives the one-chunk result."""
    x, _ = strain_2h
    xd = torch.from_numpy(x).cuda()
    rows_mc, rows_c = srs_synth.slide_rows(srs_synth.log_templates(1e-2, 9e-2, 6), F_HI, T, bin_step=2.0)
    p = _params()
    n_total = x.size // N_S
    one, r1 = ctx.slide_search(xd, BANK, rows_mc, rows_c, n_total, p)
    per_seg = 69 * N_B * 4
    many, r2 = ctx.slide_search(xd, BANK, rows_mc, rows_c, n_total, p, cube_budget_bytes=37 * per_seg)
    assert r1["n_items"] == 1 and r2["n_items"] == 7
    a, b = one["map"].cpu().numpy(), many["map"].cpu().numpy()
    assert np.allclose(a, b, rtol=1e-5, atol=2e-4)
    ca, cb = one["cands"].cpu().numpy(), many["cands"].cpu().numpy()
    assert np.array_equal(ca[:4, 1:], cb[:4, 1:])


def test_slide_argument_errors(ctx, strain_2h):
    x, _ = strain_2h
    p = _params()
    with pytest.raises(SrsError):
        ctx.slide_search(x, BANK, [1e-2], [1.0], 10, p)             # t0 fraction outside [0, 1)
    with pytest.raises(SrsError):
        ctx.slide_search(x, BANK, [1e-2], [0.0], 10, p, f0=30.0)    # f0 below the band
    with pytest.raises(SrsError):
        ctx.slide_search(x, (7e-4, 3e-8, 69), [1e-2], [0.0], 10, p)  # bank upside down
    with pytest.raises(SrsError):
        ctx.power_cube(x, BANK, 5, 5, p)                             # empty segment range
    with pytest.raises(SrsError):
        ctx.slide_search(x, BANK, [1e-2], [0.0], 10, p, weighting=2)  # unknown weighting
    with pytest.raises(SrsError):
        ctx.slide_search(x, BANK, [1e-2], [0.0], 10, p, s_eff=np.zeros((69, N_B), np.float32))  # PSD not positive
    with pytest.raises(SrsError):
        ctx.power_cube(x, BANK, 0, 1, Params(fs=FS, t_coh=T, f_lo=F_LO, f_hi=F_HI, eps=1e-9))  # below the mixed floor


def test_slide_edge_cases(ctx):
    """Degenerate sizes of the two-stage search against the oracle: a one-entry
    bank, a single t0 column, t0 columns past the data (empty tracks read 0),
    top_k larger than the map, f0 inside the band, and one-segment cube chunks."""
    x = srs_synth.strain_with_chirps(int(40 * T * FS), FS, 3, [])
    n_total = 40
    p = _params(top_k=64)
    # one-entry bank, f0 = 45 Hz, more t0 columns than segments
    bank1 = (2e-6, 2e-6, 1)
    rows_mc, rows_c = np.array([2e-3, 8e-2]), np.array([0.0, 0.5])
    cube, _ = ctx.power_cube(x, bank1, 0, n_total, p)
    cands, m, _ = ctx.stack_slide(cube, 0, n_total, bank1, rows_mc, rows_c, 50, p, f0=45.0)
    ref, L, absum = slide.stack_slide(cube.astype(np.float64), rows_mc, rows_c, 50, n_total,
                                      slide.local_bank(*bank1), 45.0, T, F_LO, N_B, with_abs=True)
    assert np.all(np.abs(m - ref) <= _slide_tol(L, absum, ref))
    assert np.all(m[:, n_total:] == 0.0) and np.all(L[:, n_total:] == 0)
    assert len(cands) == 64
    v, rr, nn = oracle.topk(m, 64)
    assert np.array_equal(cands["template_idx"], rr) and np.array_equal(cands["bin"], nn)
    # a single t0 column, the whole search in one-segment chunks
    rows_mc2, rows_c2 = srs_synth.slide_rows(srs_synth.log_templates(5e-3, 9e-2, 4), F_HI, T, bin_step=3.0)
    _, m_one, _ = ctx.slide_search(x, BANK, rows_mc2, rows_c2, 1, _params())
    per_seg = 69 * N_B * 4
    _, m_many, rep = ctx.slide_search(x, BANK, rows_mc2, rows_c2, 1, _params(), cube_budget_bytes=per_seg)
    assert rep["n_items"] == n_total and m_one.shape == (rows_mc2.size, 1)
    assert np.allclose(m_one, m_many, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("layout", ["128:global", "128:tma", "256:tma", "256:global"])
def test_power_cube_every_layout_against_oracle(monkeypatch, strain_2h, layout):
    """Every spreader layout the cube tuner can pick, on the bank's fastest
    chirps: 128-thread CTAs take an FP64 anchor per half-warp there, because a
    whole warp's span is too long for the anchor expansion at beta = 7e-4."""
    monkeypatch.setenv("SRS_MIXED_LAYOUT", layout)
    x, _ = strain_2h
    from paper_2609_12476_gb300 import srs_plan
    c = Context(0)
    try:
        cube, rep = c.power_cube(x, BANK, 40, 42, _params())
    finally:
        c.close()
    assert rep["cta_threads"] == int(layout.split(":")[0])
    bank = slide.local_bank(*BANK)
    ks = [0, 34, 66, 67, 68]
    F = oracle.spectra(x, FS, T, F_LO, N_B, bank, [(k, i) for k in ks for i in (40, 41)], local=True)
    F = F.reshape(len(ks), 2, N_B)
    P = oracle.power(F, N_S).transpose(0, 2, 1)
    tol = _p_bound(F, 1e-6).transpose(0, 2, 1) + 1e-6 * P + 1e-6
    err = np.abs(cube[ks] - P)
    assert np.all(err <= tol), (layout, float(np.max(err / tol)))


def test_cube_whitening_matches_oracle(ctx):
    """srs_cube_whiten on a seeded chi-square cube shaped by a PSD pattern,
    with the PSD estimated and with it given, against oracle.slide.whiten;
    then the stack-slide over the whitened cube with PSD weights."""
    bank = slide.local_bank(*BANK)
    n_seg = 120
    r = np.random.default_rng(12)
    S_true = r.uniform(0.5, 4.0, size=(69, N_B))
    host = (srs_synth.random_cube(69, N_B, n_seg, 13).astype(np.float64) * S_true[:, :, None])
    host[:, :, 5] *= 2.5                                       # one louder segment
    host = host.astype(np.float32)
    ref, S_ref, mu_ref, sg_ref = slide.whiten(host.astype(np.float64))
    cd = torch.from_numpy(host.copy()).cuda()
    S, mu, sg = ctx.cube_whiten(cd)
    assert np.allclose(S.cpu().numpy(), S_ref, rtol=2e-5)
    assert np.allclose(mu.cpu().numpy(), mu_ref, rtol=2e-5) and np.allclose(sg.cpu().numpy(), sg_ref, rtol=2e-5)
    out = cd.cpu().numpy()
    assert np.allclose(out, ref, rtol=1e-4, atol=2e-4), float(np.max(np.abs(out - ref)))
    # a given PSD table is used as is
    cd2 = torch.from_numpy(host.copy()).cuda()
    ctx.cube_whiten(cd2, s_eff=S_true.astype(np.float32))
    ref2, _, _, _ = slide.whiten(host.astype(np.float64), s_eff=S_true.astype(np.float32).astype(np.float64))
    assert np.allclose(cd2.cpu().numpy(), ref2, rtol=1e-4, atol=2e-4)
    # stack-slide over the whitened cube: amplitude weights over the estimated PSD, S in the weights alone
    rows_mc, rows_c = srs_synth.slide_rows(srs_synth.log_templates(2e-2, 1e-1, 5), F_HI, T, bin_step=4.0)
    S32 = S.cpu().numpy()
    _, m, _ = ctx.stack_slide(cd, 0, n_seg, BANK, rows_mc, rows_c, 100, _params(), weighting=SRS_WEIGHT_AMPLITUDE,
                              s_eff=S32, whiten=True)
    want, L, absum = slide.stack_slide(out.astype(np.float64), rows_mc, rows_c, 100, n_seg, bank, F_LO, T, F_LO, N_B,
                                       with_abs=True, weighting=1, s_eff=S32.astype(np.float64),
                                       s_eff_in_weights_only=True)
    assert np.all(np.abs(m.cpu().numpy() - want) <= _slide_tol(L, absum, want))


def test_whitened_search_in_coloured_noise(ctx):
    """Noise whose PSD falls by 2.5x across the band: unwhitened, the noise-only
    stack-slide statistic is far from N(0, 1); whitened (PSD estimated from the
    data, empirical per-segment moments), it is N(0, 1) to a few percent, and
    an entering chirp is found.  The search equals power cube + whitening +
    stack-slide called one by one."""
    # amplitude spectral density 1.5 at 40 Hz, 0.94 at 60 Hz, flat below 30 Hz
    asd = lambda f: 0.5 + (np.maximum(np.abs(f), 30.0) / 40.0) ** -2.0
    n = int(7200 * FS)
    mcs = srs_synth.log_templates(3e-2, 8e-2, 9)
    noise = srs_synth.coloured_noise(n, FS, 21, asd)
    rows_mc, rows_c = srs_synth.slide_rows(mcs, F_HI, T, bin_step=2.0)
    n_total = n // N_S
    p = _params()
    _, m_raw, _ = ctx.slide_search(noise, BANK, rows_mc, rows_c, n_total - 60, p)
    _, m_w, _ = ctx.slide_search(noise, BANK, rows_mc, rows_c, n_total - 60, p, whiten=True)
    assert abs(float(np.mean(m_w))) < 0.1 and 0.85 < float(np.std(m_w)) < 1.15
    assert abs(float(np.mean(m_raw))) > 0.3 or abs(float(np.std(m_raw)) - 1.0) > 0.3
    inj = [{"mc": float(mcs[4]), "f0": F_LO, "amp": 0.08, "t_start": 1500.0, "phi0": 1.0}]
    x = noise + srs_synth.strain_with_chirps(n, FS, 0, inj, noise=False)
    c, m, rep = ctx.slide_search(x, BANK, rows_mc, rows_c, n_total - 60, p, whiten=True)
    r, col = int(c["template_idx"][0]), int(c["bin"][0])
    assert abs(np.log(rows_mc[r] / inj[0]["mc"])) < 0.15 and abs((col + rows_c[r]) * T - 1500.0) <= T
    # the same through the three calls
    xd = torch.from_numpy(x).cuda()
    cube, _ = ctx.power_cube(xd, BANK, 0, n_total, p)
    ctx.cube_whiten(cube)
    _, m3, _ = ctx.stack_slide(cube, 0, n_total, BANK, rows_mc, rows_c, n_total - 60, p, whiten=True)
    assert np.allclose(m3.cpu().numpy(), m, rtol=1e-4, atol=1e-4)
