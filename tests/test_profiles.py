"""The committed ncu summaries match the kernel sources that are built now, so
bench.py's traffic and instruction figures are the current kernels' (a
kernel edit without a new capture would make them null).  Each summary names
the command that produced it.  CPU only."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2609_12476_gb300", "csrc")

# (summary, kernel source files it was taken on, keys bench.py reads)
SUMMARIES = [
    ("k_mixed_semicoherent_2h.md", ("srs_kernels.cu", "srs_device.cuh"),
     ("traffic_bytes_per_launch", "inst_executed_per_launch")),
    ("k_mixed_large_24h.md", ("srs_kernels.cu", "srs_device.cuh"),
     ("traffic_bytes_per_launch", "inst_executed_per_launch")),
    ("two_stage_24h.md", ("srs_kernels.cu", "srs_device.cuh"), ("k_mixed cube traffic_bytes_per_launch",)),
    ("two_stage_24h.md", ("srs_slide.cu", "srs_device.cuh"), ("k_stack_slide traffic_bytes_per_launch",)),
    ("k_score_tc_proposal_score.md", ("srs_score_tc.cu",), ()),
]


def _hash(files):
    return hashlib.sha256(b"".join(open(os.path.join(CSRC, f), "rb").read() for f in files)).hexdigest()[:16]


def test_summaries_were_taken_on_the_current_kernel_sources():
    for name, files, keys in SUMMARIES:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        assert _hash(files) in txt, (name, files)
        for key in keys:
            v = bench.profile_traffic(name, files, key)
            assert v is not None and v > 0, (name, key)


def test_summaries_name_their_commands():
    for name in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        txt = open(os.path.join(ROOT, "profiles", name)).read()
        assert "ncu " in txt and "--clock-control none" in txt, name
