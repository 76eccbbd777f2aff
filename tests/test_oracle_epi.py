"""Pins of the EPI coefficients (Eq. 30, 36-38) and of the integrator's order."""
from fractions import Fraction as Fr
from math import factorial

import numpy as np
import pytest

from oracle import epi
from oracle.testpdes import AdvectionDiffusionReaction, Burgers, SemilinearParabolic


def order_condition_residuals(A, upto):
    """Residuals of sum_m sum_i a_mi (-i)^k / (k! (m+j)!) = 1/(k+1+j)! for k >= 2,
    j >= 0, k+1+j <= upto (Taylor expansion of the remainder integral of Eq. 24
    against the ansatz Eq. 34-35).  Exact rational arithmetic."""
    res = {}
    for k in range(2, upto):
        for j in range(0, upto - k):
            lhs = sum(A[m][i] * Fr((-(i + 1)) ** k, factorial(k)) / factorial(m + 1 + j)
                      for m in range(len(A)) for i in range(len(A[0])))
            res[(k, j)] = lhs - Fr(1, factorial(k + 1 + j))
    return res


@pytest.mark.parametrize("order", [3, 4, 5, 6])
def test_order_conditions_exact(order):
    A = epi.COEFFS[order]
    assert all(v == 0 for v in order_condition_residuals(A, order).values())
    nxt = order_condition_residuals(A, order + 1)
    assert any(v != 0 for (k, j), v in nxt.items() if k + 1 + j == order + 1)


@pytest.mark.slow
@pytest.mark.parametrize("order", [4, 5, 6])
def test_empirical_order_semilinear_parabolic(order):
    """EPI4/5/6 reach their order on the semilinear parabolic PDE of Sec. 5.1
    (history seeded with the exact solution; t in [0, 1])."""
    prob = SemilinearParabolic(40)
    errs = []
    dts = [1 / 8, 1 / 16, 1 / 32] if order < 6 else [1 / 6, 1 / 12, 1 / 24]
    for dt in dts:
        P = epi.history_length(order)
        it = epi.EPI(prob.rhs, prob.jvp, order, tol=1e-14)
        # seed q_{-1..-P} with the exact solution at t = -dt, .., -P dt
        it.history = [(prob.exact(-i * dt), prob.rhs(prob.exact(-i * dt))) for i in range(1, P + 1)]
        y = prob.exact(0.0)
        nsteps = int(round(1.0 / dt))
        for _ in range(nsteps):
            y = it.step(y, dt)
        errs.append(np.linalg.norm(y - prob.exact(1.0)) / np.linalg.norm(prob.exact(1.0)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > order - 0.6, (errs, rates)


def test_startup_epi2_converges():
    """EPI2 (Eq. 25) is second order; the start-up path runs without history."""
    prob = SemilinearParabolic(30)
    errs = []
    for dt in (1 / 4, 1 / 8):
        it = epi.EPI(prob.rhs, prob.jvp, 2, tol=1e-13)
        y = prob.exact(0.0)
        for _ in range(int(round(1 / dt))):
            y = it.step(y, dt)
        errs.append(np.linalg.norm(y - prob.exact(1.0)))
    assert np.log2(errs[0] / errs[1]) > 1.6


# ---- the two nonlinear problems of Sec. 5.1 against an independent stiff solver
# The paper's reference is a stiff implicit integrator at tolerance 1e-14; here
# scipy's Radau IIA at 1e-13 (a library routine, no code shared with the oracle's
# exponential path).  The multistep history is seeded from that reference at
# t = 0, dt, .., (P - 1) dt: the paper's start-up (EPI2 with eight substeps per
# interval) has an O(dt^3) error that would hide the orders above three.  The
# step counts lie where the explicit multistep schemes are stable on these
# problems (EPI4 diverges on Burgers at 64 steps, EPI6 at 128).
STEPS = {"burgers": {3: (128, 256), 4: (256, 512), 5: (256, 512), 6: (512, 1024)},
         "adr": {3: (64, 128), 4: (64, 128), 5: (64, 128), 6: (64, 128)}}


def _problem(name):
    return Burgers() if name == "burgers" else AdvectionDiffusionReaction()


@pytest.fixture(scope="module")
def nonlinear_references():
    from scipy.integrate import solve_ivp
    out = {}
    for name, table in STEPS.items():
        pb = _problem(name)
        keys = {(N, k) for Ns in table.values() for N in Ns for k in range(5)}
        times = sorted({k * pb.T / N for N, k in keys} | {pb.T})
        sol = solve_ivp(lambda t, u: pb.rhs(u), (0.0, pb.T), pb.u0, method="Radau",
                        jac=lambda t, u: pb.jacobian(u), rtol=1e-13, atol=1e-13, t_eval=times)
        assert sol.status == 0
        at = {round(t, 12): sol.y[:, i] for i, t in enumerate(sol.t)}
        out[name] = (pb, at)
    return out


@pytest.mark.parametrize("name", ["adr", "burgers"])
def test_nonlinear_problem_jacobians(name):
    """The hand-written JVP equals the complex step of the right-hand side (exact
    for these polynomial right-hand sides) and the assembled sparse Jacobian."""
    pb = _problem(name)
    rng = np.random.default_rng(3)
    u = pb.u0 + 0.05 * rng.standard_normal(pb.u0.size)
    v = rng.standard_normal(u.size)
    Jv = pb.jvp(u, v)
    cs = pb.rhs(u + 1e-30j * v).imag / 1e-30
    assert np.max(np.abs(Jv - cs)) <= 1e-13 * np.max(np.abs(Jv))
    assert np.max(np.abs(Jv - pb.jacobian(u) @ v)) <= 1e-13 * np.max(np.abs(Jv))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["adr", "burgers"])
@pytest.mark.parametrize("order", [3, 4, 5, 6])
def test_empirical_order_nonlinear_problems(nonlinear_references, name, order):
    """EPI3-6 reach their order on the advection-diffusion-reaction PDE and on
    Burgers' equation of Sec. 5.1 (KIOPS tolerance 1e-14 as in the paper; error
    in the discrete 2-norm at the final time)."""
    pb, ref = nonlinear_references[name]
    P = epi.history_length(order)
    errs = []
    for N in STEPS[name][order]:
        dt = pb.T / N
        it = epi.EPI(pb.rhs, pb.jvp, order, tol=1e-14)
        it.history = [(ref[round((P - 1 - i) * dt, 12)], pb.rhs(ref[round((P - 1 - i) * dt, 12)])) for i in range(P)]
        y = ref[round(P * dt, 12)].copy()
        for _ in range(N - P):
            y = it.step(y, dt)
        errs.append(np.linalg.norm(y - ref[round(pb.T, 12)]))
    rate = np.log2(errs[0] / errs[1])
    assert rate > order - 0.3, (errs, rate)
