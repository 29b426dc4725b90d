"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (device-resident strain, autotuned layout, graph replay): the whole map
of the 2 h, 6 h and 24 h searches comes from the GPU; the FP64 oracle recomputes
whole rows of it (every segment of a sampled template) one spectrum at a time,
and the rows must agree within the bound the spectra tolerance implies."""
import numpy as np
import pytest

import oracle
import srs_synth
from paper_2609_12476_gb300 import Context, Params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _row_bound(P, nseg, eps, n_s):
    """|n_sigma_gpu - n_sigma_oracle| per bin of one template row implied by
    rel-L2(F) <= 10 eps per spectrum: |dF_b| <= 10 eps ||F||,
    |dP_b| <= (4 |F_b| |dF_b| + 2 |dF_b|^2) / n_s, summed over segments."""
    e = 10 * eps
    tol = np.zeros(P.shape[1])
    for Pi in P:
        Fb = np.sqrt(Pi * n_s / 2.0)
        Fn = np.sqrt(Pi.sum() * n_s / 2.0)
        tol += (4 * Fb * e * Fn + 2 * (e * Fn) ** 2) / n_s
    return tol / (2.0 * np.sqrt(nseg))


def _check_rows(name, rows):
    w = srs_synth.make_workload(name)
    p = Params(fs=w["fs"], t_coh=w["t_coh"], f_lo=w["f_lo"], f_hi=w["f_hi"], f_ref=w["f_ref"], eps=w["eps"],
               top_k=32)
    ctx = Context(0)
    try:
        xd = torch.from_numpy(np.ascontiguousarray(w["strain"])).cuda()
        torch.cuda.synchronize()
        out = None
        for _ in range(2):                       # the second call replays the captured graph
            out, rep = ctx.search(xd, w["mc"], p, out=out)
        torch.cuda.synchronize()
        smap = out["map"].cpu().numpy()
        cands = out["cands"].cpu().numpy()
    finally:
        ctx.close()
    n_s = int(round(w["t_coh"] * w["fs"]))
    n_b = smap.shape[1]
    n_tot = w["n_samples"] // n_s
    x64 = np.asarray(w["strain"], dtype=np.float64)
    for m in rows:
        b = oracle.beta(w["mc"][m], w["f_ref"])
        ns_m = oracle.nseg(b, w["f_ref"], w["f_hi"], w["t_coh"], n_tot)
        F = oracle.spectra(x64, w["fs"], w["t_coh"], w["f_lo"], n_b, [b], [(0, i) for i in range(ns_m)])
        P = oracle.power(F, n_s)
        ref = oracle.n_sigma(P.sum(axis=0, keepdims=True), [ns_m])[0]
        tol = _row_bound(P, ns_m, w["eps"], n_s) + 1e-5 * np.abs(ref) + 1e-6
        err = np.abs(smap[m] - ref)
        assert np.all(err <= tol), (name, m, float(np.max(err / tol)))
    # the candidates are the largest cells of the returned map, in order
    v, mm, bb = oracle.topk(smap, 32)
    assert np.array_equal(cands[:, 1], mm) and np.array_equal(cands[:, 2], bb)
    return smap


def test_two_hour_search_rows_match_oracle():
    """The 2 h / 64-template search: the lightest and heaviest templates
    (240 and 112 segments) and the template of the injected chirp."""
    w = srs_synth.WORKLOADS["semicoherent_2h"]
    mc = srs_synth.log_templates(2e-2, 5e-2, 64)
    inj = w["injections"][0]
    m_inj = int(np.argmin(np.abs(np.log(mc) - np.log(inj["mc"] * (inj["f0"] / 40.0) ** 1.6))))
    smap = _check_rows("semicoherent_2h", [0, 63, m_inj])
    # the injection is the loudest cell, in (or next to) its own row and bin
    m, b = np.unravel_index(np.argmax(smap), smap.shape)
    assert abs(m - m_inj) <= 1 and abs(b - int(round((inj["f0"] - 40.0) * 30.0))) <= 1


def test_six_hour_batched_search_rows_match_oracle():
    """The 6 h / 1024-template search with uneven segment counts (35 to 720
    segments per template): three rows across the bank."""
    _check_rows("batched_6h", [0, 511, 1023])


def test_large_24h_search_rows_match_oracle():
    """The 24 h / 4096-template search on float32 strain (7.2 M spectra, 64
    injections): the heaviest template (35 segments), a middle one (374) and
    the lightest, which spans all 2880 segments."""
    _check_rows("large_24h", [4095, 3000, 0])


def test_two_stage_24h_sampled_templates_match_oracle():
    """The 24 h two-stage search in the configuration bench.py times (float32
    strain on the device, 69-entry bank, 1270 x 2880 {Mc, t0} templates, one
    cube chunk): sampled templates recomputed by the oracle from their
    tracks' spectra, the heaviest rows (short tracks) and a light row cut by
    the end of the data, within the bound the spectra tolerance implies."""
    from oracle import slide
    w = srs_synth.make_slide_workload("stackslide_24h")
    p = Params(fs=w["fs"], t_coh=w["t_coh"], f_lo=w["f_lo"], f_hi=w["f_hi"], eps=w["eps"], top_k=32)
    ctx = Context(0)
    try:
        xd = torch.from_numpy(np.ascontiguousarray(w["strain"])).cuda()
        out, rep = ctx.slide_search(xd, w["bank"], w["rows_mc"], w["rows_c"], w["n_total"], p)
        torch.cuda.synchronize()
        m = out["map"].cpu().numpy()
        cands = out["cands"].cpu().numpy()
    finally:
        ctx.close()
    n_total, n_s, n_b = w["n_total"], 7680, 600
    bank = slide.local_bank(*w["bank"])
    x64 = np.asarray(w["strain"], dtype=np.float64)
    R = w["rows_mc"].size
    picks = [(R - 1, 100), (R - 1, 2000), (R - 20, 1234), (0, n_total - 25), (R // 2, n_total - 40)]
    for r, n in picks:
        mc, c = w["rows_mc"][r], w["rows_c"][r]
        k, j = slide.track(mc, c, w["f_lo"], w["t_coh"], w["f_lo"], n_b, bank, n_total)
        first = slide.first_segment(n, c)
        L = max(0, min(len(k), n_total - first))
        assert 0 < L <= 60, (r, n, L)
        F = oracle.spectra(x64, w["fs"], w["t_coh"], w["f_lo"], n_b, bank,
                           [(int(k[s]), first + s) for s in range(L)], local=True)
        P = oracle.power(F[np.arange(L), j[:L]], n_s)
        ref = slide.n_sigma_track(P)
        d = 10 * w["eps"] * np.linalg.norm(F, axis=1)
        dP = (4 * np.abs(F[np.arange(L), j[:L]]) * d + 2 * d ** 2) / n_s
        tol = np.sum(dP) / (2 * np.sqrt(L)) + L * 2.0 ** -24 * np.sum(np.abs(P - 2) / 2) / np.sqrt(L) + 1e-5
        assert abs(m[r, n] - ref) <= tol, (r, n, L, float(m[r, n]), ref, tol)
    v, rr, nn = oracle.topk(m, 32)
    assert np.array_equal(cands[:, 1], rr) and np.array_equal(cands[:, 2], nn)
    assert rep["slide_reads"] > 0 and rep["n_items"] == 1
