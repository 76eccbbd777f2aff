"""The bounds-checked build (libswepi_check.so, compiled with -DSW_CHECK) on
the GPU: the face kernels test every interface line's element and edge
numbers, the staged complex64-bulk volume kernel its copy ranges, the ensemble
kernel its decoded tasks.  With valid tables no check fires and every result
equals the default build's (the checks only guard accesses); a planted
out-of-range interface line is caught (status 1) with the access skipped, and
the context works again once the line is restored.  compute-sanitizer is not
available here, so this is the bounds check the tests rely on."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked_library():
    from paper_2101_05617_gb300 import build as b
    return b.build(checked=True)


def _run(tmp_path, checked, inject=False):
    env = dict(os.environ)
    env.pop("SWEPI_CHECKED", None)
    if checked:
        env["SWEPI_CHECKED"] = "1"
    out = str(tmp_path / ("checked.npz" if checked else "default.npz"))
    cmd = [sys.executable, "-m", "tests.checked_build_worker", out] + (["--inject"] if inject else [])
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    return np.load(out)


def test_checked_build_agrees_and_catches_a_planted_index(tmp_path, checked_library):
    assert os.path.exists(checked_library)
    d = _run(tmp_path, checked=False)
    c = _run(tmp_path, checked=True, inject=True)
    assert not bool(d["checked"]) and bool(c["checked"])
    assert list(d["codes"]) == [0, 0, 0]
    # single-context calls, EPI steps, ensemble run: no check fired; then the
    # planted line (code 1, interface line), then the restored table (0)
    assert list(c["codes"]) == [0, 0, 0, 1, 0], list(c["codes"])
    for k in d.files:
        if k in ("checked", "codes"):
            continue
        if k.startswith("ens"):   # batched reductions: compared to the order of floating-point sums
            rel = np.linalg.norm(c[k] - d[k]) / np.linalg.norm(d[k])
            assert rel < 1e-12, (k, rel)
        else:
            assert np.array_equal(c[k], d[k]), k
    assert np.array_equal(c["rhs_after"], d["rhs"])
