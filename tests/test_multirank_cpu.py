"""bench.py's multi-rank path on CPU with the gloo backend, world size 2: the
barrier and the max over ranks that time a weak-scaling run (each rank
searches an independent problem; no collective touches the data), and the
reference arm reporting from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import json, os, sys
sys.path.insert(0, %(root)r)
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
t = 1.5 + rank          # per-rank timed seconds
bench.barrier(world)
m = bench.max_over_ranks(t, world)
n_spec, steps = 1000, 4
value = world * n_spec * steps / m
print(json.dumps({"rank": rank, "max": m, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _run_two(code, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_over_ranks_and_weak_scaling_value():
    outs = _run_two(WORKER % {"root": ROOT})
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert all(r["max"] == 2.5 for r in res)
    assert all(r["value"] == pytest.approx(2 * 1000 * 4 / 2.5) for r in res)


def test_reference_arm_reports_from_rank_zero_only():
    code = r"""
import sys
sys.path.insert(0, %(root)r)
import bench
class A: pass
a = A(); a.gpus = 2; a.steps = 1; a.warmup = 0; a.workload = "semicoherent_2h"
import os
if os.environ["RANK"] != "0":
    bench.run_reference(a)     # must return at once, printing nothing
    print("DONE")
""" % {"root": ROOT}
    outs = _run_two(code)
    assert outs[1].strip() == "DONE"
