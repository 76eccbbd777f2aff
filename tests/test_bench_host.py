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


def test_orth_bytes_fused():
    """Both passes in one launch move each vector once: z and the window vectors
    read, V_{j+1} written (and its FP32 copy in the complex64-bulk form)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.orth_bytes_per_unknown(2, 1, True) == 8 * (1 + 2 + 1)
    assert bench.orth_bytes_per_unknown(3, 1, True) == 8 * (1 + 3 + 1)
    assert bench.orth_bytes_per_unknown(3, 2, True) == 8 * (1 + 3 + 1) + 4
    assert bench.orth_bytes_per_unknown(2, 1) == 56 and bench.orth_bytes_per_unknown(3, 2) == 60


def test_kernel_rooflines_arithmetic():
    """Per-kernel figures of a profiled EPI step: algorithmic flops and bytes per
    launch (the volume kernel: v and Jv, the window vectors, 4 b-columns, 11
    coefficients and the face fluxes per node, FP32 copies of the tables in the
    complex64-bulk form; the vector passes 8 (2 window + 3) B per unknown),
    divided by the average event time, against the given peaks."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2101_05617_gb300 import synth
    wl = synth.WORKLOADS["ne60_p5"]
    nodes = 6 * 60 * 60 * 36
    prof = {k: {"ms": 0.0, "count": 0} for k in ("volume_jvp", "face_jvp", "orthogonalisation", "expm", "linearize")}
    prof["volume_jvp"] = {"ms": 2.0, "count": 10}       # 0.2 ms per launch
    prof["face_jvp"] = {"ms": 0.5, "count": 10}
    prof["orthogonalisation"] = {"ms": 1.0, "count": 20}  # two passes per iteration: 0.1 ms per iteration
    for mode, iop, coef in ((1, 2, 8), (1, 3, 8), (2, 3, 4)):
        r = bench.kernel_rooflines(prof, wl, mode, iop, 10.0, 1.25)
        window = 24 * iop if mode == 1 else 0        # the complex64-bulk volume kernel reads no window vectors
        vb = nodes * (3 * coef + 24 + window + 12 * coef + 11 * coef + 2 * coef)   # EPI5: 4 b-columns; N_s = 6
        assert r["volume"]["bytes"] == vb
        assert abs(r["volume"]["gbs"] - vb / 2e-4 / 1e9) < 1e-9 * r["volume"]["gbs"]
        ob = (8.0 * (2 * iop + 3) if mode == 1 else 8.0 * (iop + 2) + 20.0) * (wl.n_unknowns + 4)
        assert r["orthogonalisation"]["bytes_per_iteration"] == ob
        assert abs(r["orthogonalisation"]["gbs"] - ob / 1e-4 / 1e9) < 1e-9 * ob
        fv = bench.flops_per_jvp(60, 6)[0] + 6 * nodes * (iop - 2)
        if mode == 1:
            assert abs(r["volume"]["fp64_frac"] - fv / 2e-4 / 1e12 / 1.25) < 1e-12
        else:
            assert "fp64_frac" not in r["volume"] and "fp32_tflops" in r["volume"]
        assert r["share_of_step"]["volume_jvp"] == 0.2 and "expm" not in r


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
    assert line["projected"] is True and "PROJECTED" in line["cpu_baseline"]["sample"]


def test_oracle_step_projection_arithmetic():
    """The projected oracle step: Krylov iterations x their cost + one expm per
    substep attempt + one combination per accepted substep + P remainder JVPs +
    one RHS."""
    sys.path.insert(0, ROOT)
    import bench
    s = {"t_iter": 0.5, "t_expm": 0.1, "t_combine_128": 0.2, "t_jvp": 0.4, "t_rhs": 0.3}
    assert abs(bench.project_oracle_step(s, 100, 5, 3, 3) - (50.0 + 0.5 + 0.6 + 1.2 + 0.3)) < 1e-12


def test_oracle_full_step_runs_on_cpu():
    """--oracle-full-step: one complete oracle EPI step (measured, with its own
    KIOPS counts) on the small workload."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-full-step", "--workload",
                          "small_ne4_p3"], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    r = json.loads(out.stdout.strip().splitlines()[-1])["oracle_full_step"]
    assert r["finite"] and r["krylov_iters"] > 0 and r["attempts"] >= r["substeps"] >= 1 and r["seconds"] > 0


def test_headline_keys():
    """The compact comparison at the end of the line reads the n_e = 60 form."""
    sys.path.insert(0, ROOT)
    import bench
    out = {"value": 10.0, "e2e": {"value": 9.5}, "forms": {"complex64_bulk_ne60_p5": {
        "steps": 48, "time_discretisation_err_rel_l2": [1e-5, 2e-4, 1e-4],
        "fp64": {"steps_per_s": 9.0},
        "complex64_bulk_window3": {"steps_per_s": 20.0, "speedup_vs_fp64": 20 / 9, "err_vs_fp64_rel_l2": [1e-7, 5e-7, 2e-7],
                                   "finite": True},
        "complex64_bulk_window3_learned": {"error": "SWError: non-finite value"}}}}
    h = bench.headline(out)
    assert h["fp64_steps_per_s"] == 10.0 and h["time_disc_err"] == 2e-4 and h["steps"] == 48
    assert h["plain_c64"]["err_vs_fp64"] == 5e-7 and h["plain_c64"]["finite"]
    assert "non-finite" in h["learned_c64"]["error"]
