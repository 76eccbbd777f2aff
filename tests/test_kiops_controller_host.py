"""Host logic of the phi-function solver: the library's controller
(csrc/kiops_ctl.h, the substep size / Krylov size / accept-reject rule of the
KIOPS reading in oracle/kiops.py) replayed on the oracle's own attempts.

The oracle runs KIOPS on small dense operators and records, per attempt, the
controller's inputs (happy breakdown, j, beta, h_{j+1,j}, F[j-1][j]) and its
decisions.  A small C++ driver feeds the same inputs to KiopsController; every
decision (accept, next m, next tau, omega) and the call's statistics must
agree: m and accept exactly, tau and omega to rounding."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import kiops as okiops

HERE = os.path.dirname(os.path.abspath(__file__))


def _cuda_include():
    for root in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if root and os.path.exists(os.path.join(root, "include", "cuda_runtime.h")):
            return os.path.join(root, "include")
    return None


@pytest.fixture(scope="module")
def replay_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs a C++ compiler and the CUDA runtime headers")
    exe = str(tmp_path_factory.mktemp("kiops_ctl") / "replay")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, os.path.join(HERE, "kiops_ctl_replay.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


def _advection_diffusion(n, c, nu, seed):
    """Periodic 1-D upwind advection plus diffusion (stiff, non-normal), with a
    seeded diagonal perturbation so that the spectrum is not symmetric."""
    I = np.eye(n)
    D1 = (I - np.roll(I, 1, axis=1)) * n
    D2 = (np.roll(I, 1, axis=1) - 2 * I + np.roll(I, -1, axis=1)) * n * n
    rng = np.random.default_rng(seed)
    return -c * D1 + nu * D2 - np.diag(rng.uniform(0.0, 5.0, n))


CASES = [
    # (n, c, nu, nb, tol, m_init, m_max, tau_init, seed)
    (64, 8.0, 0.02, 2, 1e-10, 10, 24, 0.0, 0),     # substepping at a capped Krylov size
    (64, 20.0, 0.05, 4, 1e-12, 10, 128, 0.0, 1),   # three phi-vectors, m grows
    (96, 3.0, 0.002, 3, 1e-8, 40, 60, 0.0, 2),     # large initial m
    (64, 1.0, 0.002, 2, 1e-10, 100, 128, 0.5, 4),  # half-interval first substep: the last one shrinks m
    (32, 0.0, 0.01, 1, 1e-10, 10, 128, 0.0, 3),    # symmetric, two modes: happy breakdown
]


def _case(n, c, nu, nb, seed):
    A = _advection_diffusion(n, c, nu, seed) if c > 0 else _diffusion(n, nu)
    rng = np.random.default_rng(100 + seed)
    x = np.linspace(0, 1, n, endpoint=False)
    if c > 0:
        b = [np.sin(2 * np.pi * x) + 0.1 * rng.standard_normal(n)]
        b += [rng.standard_normal(n) * 10.0 ** -k for k in range(nb - 1)]
    else:
        # two eigenvectors of the symmetric operator and b_1 = 0: the augmented
        # operator is symmetric, the window-two basis is exact, and the Krylov
        # space closes after three vectors
        b = [np.sin(2 * np.pi * x) + 0.5 * np.cos(6 * np.pi * x)]
    return A, b


def _diffusion(n, nu):
    I = np.eye(n)
    return nu * (np.roll(I, 1, axis=1) - 2 * I + np.roll(I, -1, axis=1)) * n * n


@pytest.mark.parametrize("case", CASES)
def test_controller_replays_oracle_decisions(replay_exe, case):
    n, c, nu, nb, tol, m_init, m_max, tau_init, seed = case
    A, b = _case(n, c, nu, nb, seed)
    tr = []
    _, st = okiops.kiops(1.0, lambda v: A @ v, b, tol=tol, m_init=m_init, m_max=m_max,
                         tau_init=tau_init or None, trace=tr)
    assert tr

    # the controller's initial state as the drivers set it, and beta_0 of the call
    bb = list(b) if len(b) > 1 else list(b) + [np.zeros(n)]
    p = len(bb) - 1
    norm_b = max(np.sum(np.abs(v)) for v in bb[1:])
    mu = 2.0 ** np.ceil(np.log2(norm_b)) if norm_b > 0 else 1.0
    x0 = np.concatenate([bb[0], np.zeros(p)])
    x0[n + p - 1] = mu
    beta0 = float(np.linalg.norm(x0))
    m0 = min(max(m_init, 10), m_max)
    tau0 = min(tau_init, 1.0) if tau_init > 0 else 1.0
    lines = [f"{1.0!r} {tol!r} {beta0!r} 10 {m_max} {tau0!r} {m0}"]
    for t in tr:
        lines.append(f"{int(t['happy'])} {t['j']} {float(t['beta'])!r} {float(t['hsub'])!r} {float(t['Fjj'])!r}")
    out = subprocess.run([replay_exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    rows = out.stdout.strip().splitlines()
    assert len(rows) == len(tr) + 1, out.stdout

    for t, row in zip(tr, rows[:-1]):
        m, tau, acc, m_new, tau_new, omega, _ = row.split()
        assert int(m) == t["m"] and int(acc) == int(t["accept"]) and int(m_new) == t["m_new"], (row, t)
        assert float(tau) == pytest.approx(t["tau"], rel=1e-14, abs=0.0), (row, t)
        assert float(tau_new) == pytest.approx(t["tau_new"], rel=1e-12, abs=0.0), (row, t)
        assert float(omega) == pytest.approx(t["omega"], rel=1e-12, abs=1e-300), (row, t)
    krylov, substeps, rejects, m_final, status = map(int, rows[-1].split())
    assert status == 0
    assert (krylov, substeps, rejects, m_final) == (st["krylov_iters"], st["substeps"], st["rejects"],
                                                    st["m_final"])


def test_cases_exercise_every_branch():
    """The cases above reach rejections, substepping, m changes in both
    directions and a happy breakdown (so the replay covers each decision)."""
    seen = {"reject": False, "substeps": False, "m_up": False, "m_down": False, "happy": False}
    for n, c, nu, nb, tol, m_init, m_max, tau_init, seed in CASES:
        A, b = _case(n, c, nu, nb, seed)
        tr = []
        _, st = okiops.kiops(1.0, lambda v: A @ v, b, tol=tol, m_init=m_init, m_max=m_max,
                             tau_init=tau_init or None, trace=tr)
        seen["reject"] |= st["rejects"] > 0
        seen["substeps"] |= st["substeps"] > 1
        seen["m_up"] |= any(t["m_new"] > t["m"] for t in tr)
        seen["m_down"] |= any(t["m_new"] < t["m"] for t in tr)
        seen["happy"] |= any(t["happy"] for t in tr)
    assert all(seen.values()), seen
