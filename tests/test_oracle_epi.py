"""Pins of the EPI coefficients (Eq. 30, 36-38) and of the integrator's order."""
from fractions import Fraction as Fr
from math import factorial

import numpy as np
import pytest

from oracle import epi
from oracle.testpdes import SemilinearParabolic


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
