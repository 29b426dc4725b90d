"""The C ABI library on the host: it builds, loads, exports every entry point
of include/srs.h, and its planner (no GPU) agrees with the pinned oracle and
rejects bad arguments with the documented status codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import srs_synth
from paper_2609_12476_gb300 import _capi
from paper_2609_12476_gb300 import Params, SrsError, srs_plan, SRS_MIXED, SRS_PLAIN_FP64

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "srs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(srs_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    L = _capi.lib()
    names = _declared()
    assert set(names) == set(_capi.EXPORTS)
    for n in names:
        assert hasattr(L, n), n


def test_plan_matches_oracle_beta_and_segments():
    w = srs_synth.WORKLOADS["semicoherent_2h"]
    mc = srs_synth.log_templates(2e-2, 5e-2, 64)
    info, beta, nseg = srs_plan(Params(), mc, int(7200 * 256))
    for m in range(64):
        b = oracle.beta(mc[m], 40.0)
        assert beta[m] == pytest.approx(b, rel=1e-13)
        assert nseg[m] == oracle.nseg(b, 40.0, 60.0, 30.0, 240)
    assert nseg.min() == 112 and nseg.max() == 240 and nseg.sum() == 13022
    assert info["n_spectra"] == 13022
    assert info["n_bins"] == 600 and info["n_s"] == 7680 and info["n_seg_total"] == 240


def test_plan_nufft_sizes_from_eps():
    mc = [1e-2]
    info, _, _ = srs_plan(Params(eps=1e-6), mc, 7680 * 4)
    assert info["w"] == 7 and info["n_fine"] == 1200 and info["sigma"] == pytest.approx(2.0)
    assert info["beta_es"] == pytest.approx(2.30 * 7)
    info, _, _ = srs_plan(Params(eps=1e-3), mc, 7680 * 4)
    assert info["w"] == 4
    info, _, _ = srs_plan(Params(eps=1e-9, precision=SRS_PLAIN_FP64), mc, 7680 * 4)
    assert info["w"] == 10 and info["n_fine"] == 1200
    # the full-band single-segment case needs a smaller sigma to fit shared memory
    p = Params(fs=128.0, f_lo=-64.0, f_hi=64.0, f_ref=50.0, eps=1e-9, precision=SRS_PLAIN_FP64)
    info, _, _ = srs_plan(p, mc, 3840)
    assert info["n_bins"] == 3840 and info["n_fine"] * 32 <= 200 * 1024
    assert info["n_fine"] >= 1.25 * 3840


def test_plan_rejects_bad_arguments():
    mc = [1e-2]
    bad = [Params(fs=250.01), Params(f_hi=60.01), Params(f_hi=200.0), Params(eps=1e-13), Params(eps=0.5),
           Params(top_k=0), Params(top_k=2000), Params(f_lo=60.0, f_hi=40.0), Params(sigma=1.0)]
    for p in bad:
        with pytest.raises(SrsError) as e:
            srs_plan(p, mc, 7680 * 4)
        assert e.value.status == -1, p
    with pytest.raises(SrsError) as e:
        srs_plan(Params(), mc, 100)                       # shorter than a segment
    assert e.value.status == -1
    with pytest.raises(SrsError) as e:
        srs_plan(Params(), [-1.0], 7680)
    assert e.value.status == -1


def test_plan_domain_error_past_coalescence():
    # 2 h with cut_segments = 0: the heaviest template of the 2e-2..5e-2 bank
    # coalesces at 3/(8 beta) ~ 5.1e3 s < 7200 s.
    mc = srs_synth.log_templates(2e-2, 5e-2, 64)
    with pytest.raises(SrsError) as e:
        srs_plan(Params(cut_segments=0), mc, 7200 * 256)
    assert e.value.status == -6
    srs_plan(Params(cut_segments=1), mc, 7200 * 256)


def test_plan_mixed_form_floor():
    """The mixed form accepts eps down to 2e-7 (its FP32 floor of about 1.2e-6
    relative error must stay under 10 eps) and refuses anything tighter."""
    for eps in (1e-9, 1.5e-7):
        with pytest.raises(SrsError) as e:
            srs_plan(Params(eps=eps, precision=SRS_MIXED), [1e-2], 7680)
        assert e.value.status == -5
    info, _, _ = srs_plan(Params(eps=2e-7, precision=SRS_MIXED), [1e-2], 7680)
    assert info["w"] == 8


def test_plan_items_cover_every_segment_once():
    mc = srs_synth.log_templates(5e-4, 1e-1, 32)
    for chunk in (1, 3, 16):
        info, _, nseg = srs_plan(Params(chunk=chunk), mc, 720 * 7680)
        assert info["chunk"] == chunk
        assert info["n_items"] == sum((int(n) + chunk - 1) // chunk for n in nseg)


def test_xu_roofline_arithmetic():
    """bench.py's XU model: w sqrt + w ex2 (half a slot) + sin + cos per sample."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench", os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    r = bench.xu_roofline(n_spec=1000, n_s=7680, w_taps=7, kernel_ms=1.0, n_sm=152, sm_mhz=2000.0, traffic=None)
    assert r["slots_per_sample"] == 12.5
    assert abs(r["achieved"] - 1000 * 7680 * 12.5 / 1e-3 / 1e12) < 1e-12
    assert abs(r["peak"] - 16 * 152 * 2000e6 / 1e12) < 1e-12
    assert r["bound"] == "alu" and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15


def test_component_rule_against_breadth_first_search():
    """proposal.component_cells vs a plain BFS over 8-neighbours on random masks."""
    import numpy as np
    from paper_2609_12476_gb300.proposal import component_cells
    rng = np.random.default_rng(5)
    for trial in range(20):
        score = rng.random((17, 23))
        ns = rng.standard_normal((17, 23)).astype(np.float32)
        th, top = 0.7, int(rng.integers(1, 4))
        mask = score > th
        seen = np.zeros(mask.shape, bool)
        expect = np.zeros(mask.shape, bool)
        for i0, j0 in zip(*np.nonzero(mask)):
            if seen[i0, j0]:
                continue
            comp, stack = [], [(i0, j0)]
            seen[i0, j0] = True
            while stack:
                i, j = stack.pop()
                comp.append((i, j))
                for di in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        a, b = i + di, j + dj
                        if 0 <= a < 17 and 0 <= b < 23 and mask[a, b] and not seen[a, b]:
                            seen[a, b] = True
                            stack.append((a, b))
            comp.sort(key=lambda c: (-ns[c], c[0] * 23 + c[1]))
            for c in comp[:top]:
                expect[c] = True
        assert (component_cells(score, th, ns, top) == expect).all(), trial


def test_without_a_gpu_compute_calls_fail_loudly():
    """No CPU path: without a CUDA device, creating a context fails with
    SRS_ERR_CUDA, and the entry points refuse a NULL context with SRS_ERR_ARG
    instead of computing anything."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2609_12476_gb300 import Context
    with pytest.raises(SrsError) as e:
        Context(0)
    assert e.value.status == -3          # SRS_ERR_CUDA
    L = _capi.lib()
    n = ctypes.c_int32(0)
    p = Params().c()
    x = np.zeros(7680 * 2)
    mc = np.array([1e-2])
    st = L.srs_search(None, x.ctypes.data, x.size, 1, mc.ctypes.data, 1, ctypes.byref(p), None, None,
                      ctypes.byref(n), None)
    assert st == -1                      # SRS_ERR_ARG


def test_plan_invariants_on_random_configurations():
    """Seeded random bands, rates, segment lengths, tolerances and banks: the
    fine grid is a 2^a 3^b 5^c size of at least sigma n_bins, the width follows
    the eps rule for sigma = 2, and beta and the segment counts match the oracle."""
    r = np.random.default_rng(77)
    done = 0
    while done < 40:
        fs = float(r.choice([64.0, 128.0, 256.0, 512.0]))
        t_coh = float(r.choice([8.0, 16.0, 30.0, 60.0]))
        f_lo = float(r.integers(5, int(fs / 2) - 10))
        f_hi = float(min(fs / 2, f_lo + r.integers(2, 40)))
        eps = float(10 ** r.uniform(-6.5, -2))
        mc = np.exp(r.uniform(np.log(5e-4), np.log(1e-1), size=5))
        n_total = int(r.integers(1, 200))
        p = Params(fs=fs, t_coh=t_coh, f_lo=f_lo, f_hi=f_hi, f_ref=f_lo, eps=eps)
        try:
            info, beta, nseg = srs_plan(p, mc, int(n_total * t_coh * fs))
        except SrsError as e:
            if e.status == -6:      # a template coalesces inside its first segment (Sec. II duration)
                assert min(3.0 / (8.0 * oracle.beta(m, f_lo)) for m in mc) < t_coh, (fs, f_lo, mc)
            else:                   # e.g. a band too wide for the shared-memory FFT
                assert e.status in (-1, -5), (fs, t_coh, f_lo, f_hi, eps, str(e))
            continue
        done += 1
        n_fine, n_bins = info["n_fine"], info["n_bins"]
        assert n_bins == round((f_hi - f_lo) * t_coh)
        m = n_fine
        for q in (2, 3, 5):
            while m % q == 0:
                m //= q
        assert m == 1 and n_fine >= info["sigma"] * n_bins - 1e-9
        if abs(info["sigma"] - 2.0) < 1e-12:
            assert info["w"] == int(np.ceil(np.log10(1.0 / eps))) + 1
        for k in range(5):
            b = oracle.beta(mc[k], f_lo)
            assert beta[k] == pytest.approx(b, rel=1e-13)
            assert nseg[k] == oracle.nseg(b, f_lo, f_hi, t_coh, n_total)


def test_plan_refuses_more_spectra_than_32_bit_items_hold():
    """A year of data for the lightest template (Mc = 5e-4 stays in band for
    its first N segments, about 83 days): enough copies of it to pass 2^31 - 1
    segment spectra are refused before any table is built (the largest count
    that fits is planned too, but that builds 2 GB of host tables, so the test
    plans a smaller one)."""
    n = int(365 * 86400 * 256)
    _, _, nseg = srs_plan(Params(), [5e-4], n)
    per = int(nseg[0])
    fit = (2 ** 31 - 1) // per
    with pytest.raises(SrsError) as e:
        srs_plan(Params(), np.full(fit + 1, 5e-4), n)
    assert e.value.status == -5
    info, _, _ = srs_plan(Params(), np.full(fit // 64, 5e-4), n)
    assert info["n_spectra"] == (fit // 64) * per


def test_host_output_buffers_are_checked_before_the_call():
    """A caller's numpy output must be exactly what the library writes
    (dtype, shape, C order) and writeable: a smaller or transposed array would
    take out-of-bounds or misplaced host writes."""
    _capi._host_out(None, (2, 3), np.float32, "m")
    _capi._host_out(np.empty((2, 3), np.float32), (2, 3), np.float32, "m")
    ro = np.empty((2, 3), np.float32)
    ro.flags.writeable = False
    for bad in (np.empty((2, 4), np.float32), np.empty((2, 3), np.float64), np.empty((3, 2), np.float32).T, ro,
                [[0.0] * 3] * 2):
        with pytest.raises(ValueError):
            _capi._host_out(bad, (2, 3), np.float32, "m")
