"""The XU (special-function) rates behind the spreader's roofline.

bench.py scores k_mixed against the special-function unit: per sample the
mixed spreader issues w sqrt.approx, w ex2.approx and one sin + one cos, and
the peak it divides by assumes 16 such operations per clock per SM, with
ex2.approx counted as half an operation because it runs at twice that rate.
This test measures those rates on the GPU (tests/probes/xu_rates.cu) and
checks that the constants in bench.py hold."""
import json
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_xu_rates_match_the_roofline_constants(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "xu_rates")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "probes", "xu_rates.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    r = json.loads(out.strip().splitlines()[-1])
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(HERE, "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    slot = bench.XU_SLOTS_PER_CLK_SM
    # sqrt and sin/cos at the slot rate, ex2 at twice it; FMA far above (not the bound)
    assert 0.85 * slot <= r["sqrt_per_clk_sm"] <= 1.15 * slot, r
    assert 0.85 * slot <= r["sincos_per_clk_sm"] <= 1.15 * slot, r
    assert 0.85 * slot / bench.XU_EX2_SLOT <= r["ex2_per_clk_sm"] <= 1.15 * slot / bench.XU_EX2_SLOT, r
    assert r["ffma_per_clk_sm"] > 4 * slot, r
