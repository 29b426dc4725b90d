"""The Python binding's ctypes structures match the C header's layout: for
every struct of include/srs.h that the binding passes across the ABI, a small
C program built with the host compiler prints sizeof and the offset of each
field, and the ctypes mirror must agree field by field.  CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2609_12476_gb300 import _capi  # noqa: E402

PAIRS = [
    ("srs_params", _capi._Params),
    ("srs_plan_info", _capi._PlanInfo),
    ("srs_candidate", _capi.Candidate),
    ("srs_report", _capi._Report),
    ("srs_bank", _capi._Bank),
    ("srs_slide_grid", _capi._SlideGrid),
    ("srs_injection", _capi._Injection),
    ("srs_train_cfg", _capi._TrainCfg),
    ("srs_proposal_params", _capi._ProposalParams),
    ("srs_proposal_report", _capi._ProposalReport),
]


def test_ctypes_structures_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "srs.h"', "int main(void) {"]
    for cname, py in PAIRS:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            name, field, val = line.split()
            got[(name, field)] = int(val)
    for cname, py in PAIRS:
        assert got[(cname, "sizeof")] == _ctypes_sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def _ctypes_sizeof(t):
    import ctypes
    return ctypes.sizeof(t)
