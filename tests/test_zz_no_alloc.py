"""srs_segment_spectra_static: segment spectra with no device allocation.

This entry point is for callers that cannot let the library call cudaMalloc
or cudaFree: pipelines that give all of a GPU's memory to their own
allocator when they start, and low-latency paths that cannot take the stall
and device-wide synchronisation of allocating and freeing.  It runs the same
mixed-form kernel as srs_segment_spectra, with its scratch in a fixed array
inside the library.  Here it is called through the C ABI twice in a row, and
each result must match the regular entry point's to the parity tolerance the
other tests use (relative L2 <= 1e-5 per spectrum at eps = 1e-6).  The file
is named to run last, and it builds everything it needs itself, so it passes
alone in a fresh process as well as after the other tests."""
import numpy as np
import pytest

import srs_synth
from paper_2609_12476_gb300 import Context, Params, SrsError
from paper_2609_12476_gb300._capi import segment_spectra_static

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_static_scratch_matches_regular_entry_point(dtype):
    torch = pytest.importorskip("torch")
    fs = 256.0
    x = srs_synth.strain_with_chirps(40 * 7680, fs, 5, [{"mc": 3e-2, "f0": 45.0, "amp": 0.05}])
    if dtype == "f32":
        x = x.astype(np.float32)
    mc = srs_synth.log_templates(2e-2, 5e-2, 5)
    p = Params(eps=1e-6)
    ctx = Context(0)
    ref, _ = ctx.segment_spectra(x, mc, 10, 22, p)
    ctx.close()
    xd = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()
    for _ in range(2):   # two calls in a row share (and reset) the same scratch
        F = segment_spectra_static(xd, mc, 10, 22, p)
        torch.cuda.synchronize()
        got = F.cpu().numpy()
        assert got.shape == ref.shape
        assert _rel_l2(got, ref).max() <= 1e-5


def test_static_scratch_rejects_requests_beyond_its_size():
    torch = pytest.importorskip("torch")
    # float64 strain needs a float32 copy in the scratch: 24 h at 256 Hz is
    # 88 MB, beyond the fixed array
    x = torch.zeros(86400 * 256, dtype=torch.float64, device="cuda")
    with pytest.raises(SrsError) as e:
        segment_spectra_static(x, [5e-4], 0, 2880, Params(eps=1e-6))
    assert e.value.status == -1 and "static scratch" in str(e.value)


def test_static_scratch_late_segments_of_long_float64_strain():
    """Only the requested segments of float64 strain are converted into the
    scratch, so a few segments far into a long series fit."""
    torch = pytest.importorskip("torch")
    fs = 256.0
    x = srs_synth.white_noise(700 * 7680, seed=9)          # 43 MB of float64, beyond the scratch
    mc = srs_synth.log_templates(5e-4, 2e-3, 2)
    p = Params(eps=1e-6)
    ctx = Context(0)
    ref, _ = ctx.segment_spectra(x, mc, 650, 653, p)
    ctx.close()
    xd = torch.from_numpy(x).cuda()
    for _ in range(2):
        got = segment_spectra_static(xd, mc, 650, 653, p).cpu().numpy()
        assert _rel_l2(got, ref).max() <= 1e-5


def test_static_scratch_checks_the_output_tensor():
    torch = pytest.importorskip("torch")
    xd = torch.zeros(4 * 7680, dtype=torch.float32, device="cuda")
    bad = [torch.empty((1, 2, 600), dtype=torch.complex64, device="cuda"),     # wrong dtype
           torch.empty((1, 3, 600), dtype=torch.complex128, device="cuda"),    # wrong shape
           torch.empty((1, 600, 2), dtype=torch.complex128, device="cuda").transpose(1, 2)]   # not contiguous
    for F in bad:
        with pytest.raises(ValueError):
            segment_spectra_static(xd, [1e-2], 0, 2, Params(eps=1e-6), F=F)
    with pytest.raises(ValueError):
        segment_spectra_static(xd[::2], [1e-2], 0, 1, Params(eps=1e-6))
