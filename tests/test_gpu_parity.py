"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: spectra within relative L2 <= 10 eps per spectrum (the NUFFT's
FINUFFT-sense tolerance, oracle = exact non-uniform DFT); the time map to
the phase accuracy each form is built for; n_sigma within the bound that the
per-spectrum error implies; top-k identical up to swaps inside that bound."""
import numpy as np
import pytest

import oracle
import srs_synth
from paper_2609_12476_gb300 import Context, Params, SrsError, SRS_MIXED, SRS_PLAIN_FP64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = Context(0)
    yield c
    c.close()


def rel_l2(a, b, axis=-1):
    return np.linalg.norm(a - b, axis=axis) / np.linalg.norm(b, axis=axis)


@pytest.fixture(scope="module")
def two_hours():
    return srs_synth.make_workload("semicoherent_2h")


def _oracle_phase(beta, i, n_s, fs, T, f_c):
    d = oracle.delta(beta, i * n_s / fs, np.arange(n_s) / fs)
    psi = d / T
    th = f_c * d
    return psi - np.floor(psi), th - np.floor(th)


def _cyc(a, b):
    d = np.abs(a - b)
    return np.minimum(d, 1.0 - d)


@pytest.mark.parametrize("precision,tol_psi,tol_th", [(SRS_MIXED, 1e-12, 2e-9), (SRS_PLAIN_FP64, 1e-12, 1e-11)])
def test_time_map_against_oracle(ctx, two_hours, precision, tol_psi, tol_th):
    w = two_hours
    p = Params(precision=precision)
    mc = w["mc"]
    _, beta, nseg = __import__("paper_2609_12476_gb300").srs_plan(p, mc, w["n_samples"])
    items = [(0, 0), (0, 239), (63, 0), (63, int(nseg[63]) - 1), (31, 57)]
    psi, th = ctx.time_map(mc, items, p, w["n_samples"])
    ep, et = 0.0, 0.0
    for k, (m, i) in enumerate(items):
        rp, rt = _oracle_phase(beta[m], i, 7680, 256.0, 30.0, 50.0)
        ep, et = max(ep, _cyc(psi[k], rp).max()), max(et, _cyc(th[k], rt).max())
        assert _cyc(psi[k], rp).max() < tol_psi, (m, i, _cyc(psi[k], rp).max())
        assert _cyc(th[k], rt).max() < tol_th, (m, i, _cyc(th[k], rt).max())
    print("time map (precision %d): max error %.3g periods (Psi), %.3g cycles (f_c delta)" % (precision, ep, et))


def test_time_map_with_a_fractional_demodulation_frequency(ctx, two_hours):
    """f_lo = 40.01 Hz makes k_c = f_c t_coh = 1500.3 non-integer: the mixed
    spreader then steps the demodulation phase as a second 64-bit map instead
    of deriving it from k_c Psi.  Same bars as the integer case."""
    w = two_hours
    p = Params(f_lo=40.01, f_hi=60.01, precision=SRS_MIXED)
    mc = w["mc"]
    _, beta, nseg = __import__("paper_2609_12476_gb300").srs_plan(p, mc, w["n_samples"])
    items = [(0, 0), (0, 239), (63, int(nseg[63]) - 1), (31, 57)]
    psi, th = ctx.time_map(mc, items, p, w["n_samples"])
    et = 0.0
    for k, (m, i) in enumerate(items):
        rp, rt = _oracle_phase(beta[m], i, 7680, 256.0, 30.0, 50.01)
        assert _cyc(psi[k], rp).max() < 1e-12, (m, i, _cyc(psi[k], rp).max())
        et = max(et, _cyc(th[k], rt).max())
    print("time map, k_c = 1500.3: max error %.3g cycles (f_c delta)" % et)
    assert et < 2e-9


def test_single_segment_full_band_plain_fp64(ctx):
    """Single segment, exact template, 3840 modes at eps = 1e-9 in FP64."""
    w = srs_synth.make_workload("single")
    p = Params(fs=128.0, f_lo=-64.0, f_hi=64.0, f_ref=50.0, eps=1e-9, precision=SRS_PLAIN_FP64)
    F, _ = ctx.segment_spectra(w["strain"], w["mc"], 0, 1, p)
    b = oracle.beta(1e-2, 50.0)
    R = oracle.spectra(w["strain"], 128.0, 30.0, -64.0, 3840, [b], [(0, 0)])
    assert rel_l2(F[0], R).max() <= 1e-8
    # the injected chirp sits in the 50 Hz bin
    assert np.argmax(np.abs(F[0, 0])) in (1920 + 1500, 1920 - 1500)


def test_single_segment_full_band_mixed(ctx):
    w = srs_synth.make_workload("single")
    p = Params(fs=128.0, f_lo=-64.0, f_hi=64.0, f_ref=50.0, eps=1e-6, precision=SRS_MIXED)
    F, _ = ctx.segment_spectra(w["strain"], w["mc"], 0, 1, p)
    R = oracle.spectra(w["strain"], 128.0, 30.0, -64.0, 3840, [oracle.beta(1e-2, 50.0)], [(0, 0)])
    assert rel_l2(F[0], R).max() <= 1e-5


@pytest.mark.parametrize("precision", [SRS_MIXED, SRS_PLAIN_FP64])
def test_spectra_two_hours_subset(ctx, two_hours, precision):
    w = two_hours
    p = Params(precision=precision, eps=1e-6)
    mc = w["mc"][[0, 31, 63]]
    segs = (0, 3)
    F, _ = ctx.segment_spectra(w["strain"], mc, segs[0], segs[1], p)
    betas = [oracle.beta(m, 40.0) for m in mc]
    items = [(m, i) for m in range(3) for i in range(*segs)]
    R = oracle.spectra(w["strain"], 256.0, 30.0, 40.0, 600, betas, items).reshape(3, 3, 600)
    err = rel_l2(F, R)
    assert err.max() <= 1e-5, err
    # last in-band segment of the heaviest template: its tau span exceeds one period (wrap)
    F2, _ = ctx.segment_spectra(w["strain"], mc[2:], 110, 112, p)
    R2 = oracle.spectra(w["strain"], 256.0, 30.0, 40.0, 600, betas[2:], [(0, 110), (0, 111)])
    assert rel_l2(F2[0], R2).max() <= 1e-5


@pytest.mark.parametrize("precision,eps", [(SRS_MIXED, 1e-2), (SRS_MIXED, 1e-3), (SRS_MIXED, 1e-4),
                                           (SRS_MIXED, 1e-5), (SRS_MIXED, 2e-7), (SRS_PLAIN_FP64, 1e-3),
                                           (SRS_PLAIN_FP64, 1e-7), (SRS_PLAIN_FP64, 1e-10)])
def test_eps_sweep(ctx, two_hours, precision, eps):
    w = two_hours
    mc = w["mc"][[5, 60]]
    p = Params(precision=precision, eps=eps)
    F, _ = ctx.segment_spectra(w["strain"], mc, 20, 22, p)
    betas = [oracle.beta(m, 40.0) for m in mc]
    R = oracle.spectra(w["strain"], 256.0, 30.0, 40.0, 600, betas,
                       [(0, 20), (0, 21), (1, 20), (1, 21)]).reshape(2, 2, 600)
    assert rel_l2(F, R).max() <= 10 * eps


def test_ragged_segment_and_noninteger_demodulation(ctx):
    """6000-sample segments (not a multiple of the 256-thread run layout) and a
    band whose centre is not a whole number of cycles per segment."""
    fs, T = 200.0, 30.0
    f_lo = 40.0 + 1.0 / 60.0
    p = Params(fs=fs, t_coh=T, f_lo=f_lo, f_hi=f_lo + 20.0, eps=1e-6)
    x = srs_synth.strain_with_chirps(4 * 6000, fs, 7, [{"mc": 5e-2, "f0": 47.0, "amp": 0.1}])
    mc = np.array([5e-2, 8e-3])
    F, _ = ctx.segment_spectra(x, mc, 1, 4, p)
    betas = [oracle.beta(m, 40.0) for m in mc]
    R = oracle.spectra(x, fs, T, f_lo, 600, betas, [(m, i) for m in range(2) for i in range(1, 4)]).reshape(2, 3, 600)
    assert rel_l2(F, R).max() <= 1e-5
    Fp, _ = ctx.segment_spectra(x, mc, 1, 4, Params(fs=fs, t_coh=T, f_lo=f_lo, f_hi=f_lo + 20.0, eps=1e-6,
                                                    precision=SRS_PLAIN_FP64))
    assert rel_l2(Fp, R).max() <= 1e-5


def _search_case():
    """40 segments, 6 templates; one chirp injected exactly on template 3 at bin
    120 (44 Hz): its beta at 44 Hz equals template 3's beta at f_ref = 40 Hz."""
    fs, T, nseg_tot = 256.0, 30.0, 40
    mc = srs_synth.log_templates(6e-2, 1e-1, 6)
    b3 = srs_synth.chirp_beta(mc[3], 40.0)
    inj = [{"mc": srs_synth.mc_for_beta(b3, 44.0), "f0": 44.0, "amp": 0.05}]
    x = srs_synth.strain_with_chirps(nseg_tot * 7680, fs, 21, inj)
    return x, mc


def _map_tolerance(P, items, nsegs, eps, n_s, shape):
    """Bound on |n_sigma_gpu - n_sigma_oracle| implied by rel-L2(F) <= 10 eps per
    spectrum: |dF_b| <= 10 eps ||F||, |dP_b| <= (4 |F_b| |dF_b| + 2 |dF_b|^2) / n_s."""
    tol = np.zeros(shape)
    e = 10 * eps
    for k, (m, _i) in enumerate(items):
        Fb = np.sqrt(P[k] * n_s / 2.0)
        Fn = np.sqrt(P[k].sum() * n_s / 2.0)
        tol[m] += (4 * Fb * e * Fn + 2 * (e * Fn) ** 2) / n_s
    return tol / (2.0 * np.sqrt(np.asarray(nsegs, dtype=float)).reshape(-1, 1))


@pytest.mark.parametrize("precision", [SRS_MIXED, SRS_PLAIN_FP64])
def test_search_against_oracle(ctx, precision):
    x, mc = _search_case()
    eps = 1e-6
    p = Params(precision=precision, eps=eps, top_k=32)
    cands, smap, rep = ctx.search(x, mc, p)
    betas = [oracle.beta(m, 40.0) for m in mc]
    nsegs = [oracle.nseg(b, 40.0, 60.0, 30.0, 40) for b in betas]
    items = [(m, i) for m in range(len(mc)) for i in range(nsegs[m])]
    F = oracle.spectra(x, 256.0, 30.0, 40.0, 600, betas, items)
    P = oracle.power(F, 7680)
    S = np.zeros((len(mc), 600))
    for k, (m, _i) in enumerate(items):
        S[m] += P[k]
    ns = oracle.n_sigma(S, nsegs)
    tol = _map_tolerance(P, items, nsegs, eps, 7680, ns.shape) + 1e-5 * np.abs(ns) + 1e-6
    assert np.all(np.abs(smap - ns) <= tol), np.max(np.abs(smap - ns) / tol)
    assert rep["n_spectra"] == sum(nsegs)
    # top-k: identical cells except swaps whose oracle values lie within tolerance
    ov, om, ob = oracle.topk(ns, 32)
    kth = ov[-1]
    for c in cands:
        m, b = int(c["template_idx"]), int(c["bin"])
        assert abs(c["value"] - ns[m, b]) <= tol[m, b]
        assert ns[m, b] >= kth - tol[m, b] - tol[om[-1], ob[-1]]
    for pos in range(32):
        gm, gb = int(cands[pos]["template_idx"]), int(cands[pos]["bin"])
        if (gm, gb) != (om[pos], ob[pos]):
            assert abs(ns[gm, gb] - ov[pos]) <= tol[gm, gb] + tol[om[pos], ob[pos]]
    # the injected chirp is the top candidate, in its own cell
    assert (int(cands[0]["template_idx"]), int(cands[0]["bin"])) == (3, 120)
    assert cands[0]["value"] > 20


def test_device_io_matches_host_io(ctx):
    torch = pytest.importorskip("torch")
    x, mc = _search_case()
    p = Params(eps=1e-6, top_k=16)
    c_host, m_host, _ = ctx.search(x, mc, p)
    xd = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()   # device inputs must be ready before the library's stream reads them
    out, _ = ctx.search(xd, mc, p)
    torch.cuda.synchronize()
    m_dev = out["map"].cpu().numpy()
    # shared-memory float atomics add in a run-dependent order: equal to rounding
    assert np.max(np.abs(m_dev - m_host)) < 1e-4
    cd = out["cands"].cpu().numpy()
    assert cd[0, 1] == c_host["template_idx"][0] and cd[0, 2] == c_host["bin"][0]
    # float32 strain through the same path
    c32, m32, _ = ctx.search(x.astype(np.float32), mc, p)
    assert np.max(np.abs(m32 - m_host)) < 1e-2


def test_errors_are_status_codes(ctx):
    x = np.zeros(7680 * 2)
    with pytest.raises(SrsError) as e:
        ctx.search(x, [1e-2], Params(fs=250.01))
    assert e.value.status == -1
    with pytest.raises(SrsError) as e:
        ctx.search(x[:100], [1e-2], Params())
    assert e.value.status == -1
    with pytest.raises(SrsError) as e:
        ctx.segment_spectra(x, [1e-2], 0, 1, Params(eps=1e-9, precision=SRS_MIXED))
    assert e.value.status == -5
    # the context is still usable afterwards
    c, m, _ = ctx.search(np.random.default_rng(0).standard_normal(7680 * 2), [1e-2], Params(top_k=4))
    assert len(c) == 4 and np.isfinite(m).all()


def test_binding_rejects_mismatched_buffers(ctx):
    """The binding checks caller-supplied tensors before any device work: the
    library writes exactly [templates, n_bins] float32 and [top_k, 3] int32 and
    reads the strain as one flat array on the context's device."""
    torch = pytest.importorskip("torch")
    from paper_2609_12476_gb300 import CAND_DTYPE
    mc = srs_synth.log_templates(2e-2, 5e-2, 2)
    p = Params(eps=1e-6, top_k=4)
    xh = srs_synth.white_noise(4 * 7680, 5)
    x = torch.from_numpy(xh).cuda()
    good = {"map": torch.empty((2, 600), dtype=torch.float32, device="cuda"),
            "cands": torch.empty((4, 3), dtype=torch.int32, device="cuda")}
    bad = [dict(good, map=torch.empty((2, 599), dtype=torch.float32, device="cuda")),
           dict(good, map=torch.empty((2, 600), dtype=torch.float64, device="cuda")),
           dict(good, map=torch.empty((600, 2), dtype=torch.float32, device="cuda").t()),
           dict(good, map=torch.empty((2, 600), dtype=torch.float32)),
           dict(good, cands=torch.empty((3, 3), dtype=torch.int32, device="cuda")),
           {"map": good["map"]}]
    for o in bad:
        with pytest.raises(ValueError):
            ctx.search(x, mc, p, out=o)
        with pytest.raises(ValueError):
            ctx.search_async(x, mc, p, o)
    xs = torch.from_numpy(np.repeat(xh, 2)).cuda()[::2]        # the same samples, strided
    with pytest.raises(ValueError):
        ctx.search(xs, mc, p)
    with pytest.raises(ValueError):
        ctx.segment_spectra(xs, mc, 0, 1, p)
    with pytest.raises(ValueError):
        ctx.search_async(xh, mc, p, {"map": np.empty((2, 599), np.float32), "cands": np.zeros(4, CAND_DTYPE)})
    with pytest.raises(ValueError):
        ctx.make_strain(100, 256.0, 1, out=torch.empty(99, dtype=torch.float32, device="cuda"))
    with pytest.raises(TypeError):
        ctx.score_map(torch.zeros((4, 600), dtype=torch.float64, device="cuda"), np.zeros(1, np.float32))
    # the right buffers still work, and give the map of a search with its own outputs
    out, _ = ctx.search(x, mc, p, out=good)
    ref, _ = ctx.search(x, mc, p)
    torch.cuda.synchronize()
    assert torch.allclose(out["map"], ref["map"], rtol=1e-5, atol=1e-5)


def test_bounded_wait_gives_up_with_a_status(ctx):
    """The spreader's staging wait, armed for a transfer that never comes,
    gives up after its cycle limit: the call returns SRS_ERR_TIMEOUT with the
    give-up recorded, nothing hangs, and the context keeps working."""
    import time
    t0 = time.perf_counter()
    with pytest.raises(SrsError) as ei:
        ctx.selftest_wait()
    assert ei.value.status == -4 and "gave up" in str(ei.value)
    assert time.perf_counter() - t0 < 30
    c, m, _ = ctx.search(srs_synth.white_noise(3 * 7680, 3), [3e-2], Params(top_k=4))
    assert len(c) == 4 and np.all(np.isfinite(m))


@pytest.mark.parametrize("chunk", [1, 2, 3, 16])
def test_chunked_items_and_many_items_per_cta(ctx, two_hours, chunk):
    """Work items of several segments, and more items than resident CTAs, give
    the same spectra and map as the oracle / as one segment per item."""
    w = two_hours
    mc = w["mc"][[0, 63]]
    p = Params(eps=1e-6, chunk=chunk)
    F, rep = ctx.segment_spectra(w["strain"], mc, 100, 112, p)
    assert rep["chunk"] == chunk
    betas = [oracle.beta(m, 40.0) for m in mc]
    sel = [(0, 100), (0, 105), (1, 111)]
    R = oracle.spectra(w["strain"], 256.0, 30.0, 40.0, 600, betas, sel)
    got = np.array([F[m, i - 100] for m, i in sel])
    assert rel_l2(got, R).max() <= 1e-5
    # a full 2 h search: thousands of items over a few hundred CTAs
    c1, m1, r1 = ctx.search(w["strain"], w["mc"], Params(eps=1e-6, chunk=chunk))
    assert r1["chunk"] == chunk and r1["n_items"] > 600
    if chunk == 1:
        test_chunked_items_and_many_items_per_cta.ref = m1
    elif hasattr(test_chunked_items_and_many_items_per_cta, "ref"):
        assert np.max(np.abs(m1 - test_chunked_items_and_many_items_per_cta.ref)) < 1e-4


@pytest.mark.parametrize("k", [1, 32, 1000])
def test_topk_is_exact_on_the_returned_map(ctx, two_hours, k):
    """The candidates are exactly the k largest cells of the map the call
    returns, ordered by (value desc, template asc, bin asc): index work, so
    bit-exact, across the multi-level tile reduction."""
    w = two_hours
    cands, smap, _ = ctx.search(w["strain"], w["mc"], Params(eps=1e-6, top_k=k))
    v, m, b = oracle.topk(smap, k)
    assert np.array_equal(cands["template_idx"], m) and np.array_equal(cands["bin"], b)
    assert np.array_equal(cands["value"], v.astype(np.float32))


def test_graph_replay_and_interleaved_calls(ctx, two_hours):
    """Repeated searches replay a captured CUDA graph; calls of another kind in
    between (which regrow the device tables) must not leave a stale graph."""
    w = two_hours
    p = Params(eps=1e-6, top_k=16)
    c0, m0, r0 = ctx.search(w["strain"], w["mc"], p)
    c1, m1, r1 = ctx.search(w["strain"], w["mc"], p)
    assert r1["kernel_launches"] == r0["kernel_launches"]
    # a spectra call with a wider band and more templates regrows corr / tw / items
    wide = Params(fs=256.0, f_lo=20.0, f_hi=100.0, eps=1e-6)
    ctx.segment_spectra(w["strain"], srs_synth.log_templates(2e-2, 5e-2, 80), 0, 3, wide)
    ctx.time_map(w["mc"], [(0, 0), (5, 3)], p, w["n_samples"])
    c2, m2, r2 = ctx.search(w["strain"], w["mc"], p)
    for m in (m1, m2):
        assert np.max(np.abs(m - m0)) < 1e-4
    assert (c2["template_idx"][0], c2["bin"][0]) == (c0["template_idx"][0], c0["bin"][0])
    # autotuned chunk stays fixed for this shape
    assert r2["chunk"] == r0["chunk"]


@pytest.mark.parametrize("layout", ["256:tma", "256:global", "128:tma", "128:global"])
def test_every_spreader_layout_against_oracle(monkeypatch, layout):
    """Each CTA size / sample-staging layout the tuner may pick gives the same
    map as the FP64 oracle within the spectrum-error bound."""
    monkeypatch.setenv("SRS_MIXED_LAYOUT", layout)
    # lighter templates than _search_case, so that the degree-5 anchor expansion
    # also holds over the 128-thread layout's doubled warp span
    fs, T, nseg_tot = 256.0, 30.0, 40
    mc = srs_synth.log_templates(2e-2, 5e-2, 6)
    b3 = srs_synth.chirp_beta(mc[3], 40.0)
    inj = [{"mc": srs_synth.mc_for_beta(b3, 44.0), "f0": 44.0, "amp": 0.05}]
    x = srs_synth.strain_with_chirps(nseg_tot * 7680, fs, 23, inj)
    eps = 1e-6
    c = Context(0)
    try:
        cands, smap, rep = c.search(x.astype(np.float32), mc, Params(precision=SRS_MIXED, eps=eps, top_k=8))
    finally:
        c.close()
    threads, staging = layout.split(":")
    assert rep["cta_threads"] == int(threads)
    assert rep["staging"] == (1 if staging == "tma" else 0)
    betas = [oracle.beta(m, 40.0) for m in mc]
    nsegs = [oracle.nseg(b, 40.0, 60.0, 30.0, 40) for b in betas]
    items = [(m, i) for m in range(len(mc)) for i in range(nsegs[m])]
    F = oracle.spectra(x.astype(np.float32).astype(np.float64), 256.0, 30.0, 40.0, 600, betas, items)
    P = oracle.power(F, 7680)
    S = np.zeros((len(mc), 600))
    for k, (m, _i) in enumerate(items):
        S[m] += P[k]
    ns = oracle.n_sigma(S, nsegs)
    tol = _map_tolerance(P, items, nsegs, eps, 7680, ns.shape) + 1e-5 * np.abs(ns) + 1e-6
    assert np.all(np.abs(smap - ns) <= tol), np.max(np.abs(smap - ns) / tol)
    assert (int(cands[0]["template_idx"]), int(cands[0]["bin"])) == (3, 120)


def test_async_searches_match_synchronous(ctx):
    """srs_search_async queued back to back on different strains (and past the
    256 event slots) equals srs_search on each, within the map tolerance of
    run-to-run float summation order; srs_sync reports averaged timing."""
    torch = pytest.importorskip("torch")
    fs, nseg_tot = 256.0, 12
    mc = srs_synth.log_templates(2e-2, 5e-2, 4)
    p = Params(eps=1e-6, top_k=8)
    xs = [torch.from_numpy(srs_synth.white_noise(nseg_tot * 7680, 100 + k)).cuda() for k in range(3)]
    ref = [ctx.search(x, mc, p)[0]["map"].clone() for x in xs]
    outs = [{"map": torch.empty_like(ref[0]), "cands": torch.empty((8, 3), dtype=torch.int32, device="cuda")}
            for _ in xs]
    for rep in range(2):
        for x, o in zip(xs, outs):
            assert ctx.search_async(x, mc, p, o) == 8
    r = ctx.sync()
    from paper_2609_12476_gb300 import srs_plan
    info, _, _ = srs_plan(p, mc, nseg_tot * 7680)
    assert r["device_ms"] > 0 and r["spread_ms"] > 0 and r["n_spectra"] == info["n_spectra"]
    for a, b in zip(outs, ref):
        assert torch.allclose(a["map"], b, rtol=1e-5, atol=1e-5)
    # more calls than event slots: the oldest are settled inside, the rest at sync
    for k in range(300):
        ctx.search_async(xs[k % 3], mc, p, outs[k % 3])
    ctx.sync()
    for a, b in zip(outs, ref):
        assert torch.allclose(a["map"], b, rtol=1e-5, atol=1e-5)
    # host buffers (pinned strain, numpy outputs): uploads overlap the previous
    # search through two staging buffers; each call sees its own strain
    from paper_2609_12476_gb300 import CAND_DTYPE
    hs = [x.cpu().pin_memory().numpy() for x in xs]
    hout = [{"map": np.empty(tuple(ref[0].shape), np.float32), "cands": np.zeros(8, CAND_DTYPE)} for _ in range(7)]
    for k in range(7):
        ctx.search_async(hs[k % 3], mc, p, hout[k])
    ctx.sync()
    for k in range(7):
        assert np.allclose(hout[k]["map"], ref[k % 3].cpu().numpy(), rtol=1e-5, atol=1e-5)
        c_ref, _, _ = ctx.search(hs[k % 3], mc, p, stat_map=False)
        assert np.array_equal(hout[k]["cands"][["template_idx", "bin"]], c_ref[["template_idx", "bin"]])
    with pytest.raises(ValueError):
        ctx.search_async(hs[0], mc, p, {"map": None, "cands": np.zeros(3, CAND_DTYPE)})   # too few candidates


def test_search_degenerate_sizes(ctx):
    """One segment of data; a template that leaves the band inside its first
    segment (N_seg = 1, FP64 form: the mixed form refuses chirps that fast);
    top_k at its maximum, 1024."""
    fs = 256.0
    x1 = srs_synth.strain_with_chirps(7680, fs, 31, [{"mc": 3e-2, "f0": 50.0, "amp": 0.1}])
    c, m, rep = ctx.search(x1, [3e-2], Params(eps=1e-6, top_k=4))
    assert rep["n_spectra"] == 1
    F = oracle.spectra(x1, fs, 30.0, 40.0, 600, [oracle.beta(3e-2, 40.0)], [(0, 0)])
    ref = oracle.n_sigma(oracle.power(F, 7680), [1])
    assert np.max(np.abs(m - ref)) < 1e-3
    # N_seg = 1 next to a light template, FP64 form
    x = srs_synth.strain_with_chirps(8 * 7680, fs, 32, [])
    mc = np.array([0.62, 3e-2])
    betas = [oracle.beta(v, 40.0) for v in mc]
    nsegs = [oracle.nseg(b, 40.0, 60.0, 30.0, 8) for b in betas]
    assert nsegs[0] == 1
    c, m, rep = ctx.search(x, mc, Params(eps=1e-9, precision=SRS_PLAIN_FP64, top_k=8))
    assert rep["n_spectra"] == sum(nsegs)
    items = [(k, i) for k in range(2) for i in range(nsegs[k])]
    P = oracle.power(oracle.spectra(x, fs, 30.0, 40.0, 600, betas, items), 7680)
    S = np.zeros((2, 600))
    for q, (k, _i) in enumerate(items):
        S[k] += P[q]
    assert np.max(np.abs(m - oracle.n_sigma(S, nsegs))) < 1e-4
    # the largest top-k
    w = srs_synth.make_workload("semicoherent_2h")
    cands, smap, _ = ctx.search(w["strain"], w["mc"], Params(eps=1e-6, top_k=1024))
    v, mm, bb = oracle.topk(smap, 1024)
    assert len(cands) == 1024
    assert np.array_equal(cands["template_idx"], mm) and np.array_equal(cands["bin"], bb)


def test_cufft_comparison_path_matches_oracle_and_fused(ctx, two_hours):
    """srs_segment_spectra_cufft (spread grids in HBM, cuFFT C2C, separate
    deconvolution) computes the same spectra as the fused kernel: both within
    10 eps of the oracle, and within FP32 rounding of each other."""
    w = two_hours
    p = Params(precision=SRS_MIXED, eps=1e-6)
    mc = w["mc"][[0, 31, 63]]
    F, _ = ctx.segment_spectra(w["strain"], mc, 0, 3, p)
    Fc, rep = ctx.segment_spectra(w["strain"], mc, 0, 3, p, via_cufft=True)
    betas = [oracle.beta(m, 40.0) for m in mc]
    items = [(m, i) for m in range(3) for i in range(3)]
    R = oracle.spectra(w["strain"], 256.0, 30.0, 40.0, 600, betas, items).reshape(3, 3, 600)
    assert rel_l2(Fc, R).max() <= 1e-5
    assert rel_l2(Fc, F).max() <= 2e-6
    assert rep["kernel_launches"] >= 3 and rep["fft_ms"] > 0 and rep["spread_ms"] > 0
    # device-resident strain, a larger batch that re-plans cuFFT, then the first size again
    torch = pytest.importorskip("torch")
    xd = torch.from_numpy(np.ascontiguousarray(w["strain"])).cuda()
    mcb = w["mc"][:16]
    Fd, _ = ctx.segment_spectra(xd, mcb, 10, 30, p)
    Fdc, _ = ctx.segment_spectra(xd, mcb, 10, 30, p, via_cufft=True)
    assert rel_l2(Fdc.cpu().numpy(), Fd.cpu().numpy()).max() <= 2e-6
    Fc2, _ = ctx.segment_spectra(w["strain"], mc, 0, 3, p, via_cufft=True)
    # shared-memory atomics in the spreader sum in no fixed order: equal up to FP32 rounding
    assert rel_l2(Fc2, Fc).max() <= 1e-6
    with pytest.raises(SrsError):
        ctx.segment_spectra(w["strain"], mc, 0, 1, Params(precision=SRS_PLAIN_FP64, eps=1e-6), via_cufft=True)


_OOM_SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle, srs_synth
from paper_2609_12476_gb300 import Context, Params, SrsError
w = srs_synth.make_workload("semicoherent_2h")
ctx = Context(0)
try:
    ctx.search(w["strain"], w["mc"], Params(eps=1e-6))
    print("NO-ERROR")
except SrsError as e:
    print("STATUS", e.status, str(e).replace("\n", " "))
x = srs_synth.strain_with_chirps(4 * 7680, 256.0, 3, [{"mc": 8e-2, "f0": 50.0, "amp": 0.05}])
c, m, rep = ctx.search(x, [8e-2], Params(eps=1e-6, top_k=4))
b = oracle.beta(8e-2, 40.0)
n = oracle.nseg(b, 40.0, 60.0, 30.0, 4)
ref = oracle.n_sigma(oracle.power(oracle.spectra(x, 256.0, 30.0, 40.0, 600, [b], [(0, i) for i in range(n)]),
                                  7680).sum(axis=0, keepdims=True), [n])
print("AFTER", rep["n_spectra"], float(np.max(np.abs(m - ref))))
ctx.close()
"""


def test_out_of_memory_is_a_status_and_the_context_recovers(tmp_path):
    """An allocation the device cannot satisfy comes back as SRS_ERR_OOM with a
    message, and the same context then runs a search that fits.  The failure
    is made on the host: SRS_ALLOC_LIMIT_BYTES caps every device allocation
    (here 4 MB, below the 2 h search's 7 MB float32 strain copy), so no GPU
    memory is exhausted."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "oom.py"
    script.write_text(_OOM_SCRIPT)
    env = dict(os.environ, SRS_ALLOC_LIMIT_BYTES=str(4 << 20))
    r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split("\n")
    status = [l for l in lines if l.startswith("STATUS")]
    assert status and status[0].split()[1] == "-2", r.stdout          # SRS_ERR_OOM
    after = [l for l in lines if l.startswith("AFTER")][0].split()
    assert int(after[1]) >= 1 and float(after[2]) < 1e-3
