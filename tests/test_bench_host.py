"""Host logic of bench.py: replica aggregation across ranks (gloo, CPU)."""
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
import os, sys, json
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
r = dist.get_rank()
mx, tot = bench.aggregate(dist, 100.0 + 50.0 * r, 3 + r)
print(json.dumps({"rank": r, "max": mx, "total": tot}))
dist.destroy_process_group()
"""


def test_aggregate_two_ranks_gloo():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER % ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for r in res:
        assert r["max"] == 150.0 and r["total"] == 7


def test_flop_counts():
    sys.path.insert(0, ROOT)
    import bench
    fv, ff = bench.flops_per_jvp(60, 6)
    assert fv == 6 * 3600 * 36 * 165 and ff == 12 * 3600 * 6 * 112


def test_reference_arm_runs_on_cpu():
    """--impl reference times the oracle on the host (small bounded sample)."""
    sys.path.insert(0, ROOT)
    env = dict(os.environ)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--workload", "small_ne4_p3"], capture_output=True, text=True,
                         timeout=600, env=env)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
