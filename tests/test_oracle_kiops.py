"""Pins of the oracle's phi-function combination (Eq. 26, 29)."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle.kiops import kiops


def phi_scalar(k, z):
    """phi_k(z) by the integral of Eq. (26) (Gauss-Legendre quadrature, exact to
    round-off for the moderate |z| used here) -- independent of any recursion."""
    if k == 0:
        return np.exp(z)
    x, w = np.polynomial.legendre.leggauss(60)
    s = 0.5 * (x + 1)
    return 0.5 * np.sum(w[None] * np.exp(np.outer(z, 1 - s)) * s[None] ** (k - 1), axis=1) / math.factorial(k - 1)


def test_zero_matrix():
    """A = 0: sum_k tau^k phi_k(0) b_k = sum_k tau^k b_k / k!."""
    rng = np.random.default_rng(0)
    b = [rng.standard_normal(30) for _ in range(5)]
    for tau in (1.0, 0.37):
        w, st = kiops(tau, lambda x: 0 * x, b, tol=1e-13)
        ref = sum(tau ** k * b[k] / math.factorial(k) for k in range(5))
        np.testing.assert_allclose(w, ref, rtol=1e-11, atol=1e-12 * np.max(np.abs(ref)))


def test_diagonal_matrix_closed_form():
    """Diagonal A: each component is a scalar sum of phi_k(lambda_i) b_k,i (Eq. 26)."""
    rng = np.random.default_rng(1)
    lam = -np.geomspace(1e-2, 40.0, 60) + 1j * 0
    lam = lam.real
    b = [rng.standard_normal(60) for _ in range(4)]
    w, st = kiops(1.0, lambda x: lam * x, b, tol=1e-12)
    ref = sum(phi_scalar(k, lam) * b[k] for k in range(4))
    np.testing.assert_allclose(w, ref, rtol=1e-9, atol=1e-10 * np.max(np.abs(ref)))


@pytest.mark.parametrize("p", [1, 2, 4])
def test_dense_augmented_exponential(p):
    """Against the exponential of the (n+p)^2 augmented matrix (scipy expm)."""
    rng = np.random.default_rng(p)
    n = 60
    B = rng.standard_normal((n, n))
    A = -(B @ B.T) / n * 8 + 2.0 * (B - B.T) / np.sqrt(n)
    b = [rng.standard_normal(n) for _ in range(p + 1)]
    aug = np.zeros((n + p, n + p))
    aug[:n, :n] = A
    for l in range(p):
        aug[:n, n + l] = b[p - l]
    for l in range(p - 1):
        aug[n + l, n + l + 1] = 1.0
    x0 = np.zeros(n + p)
    x0[:n] = b[0]
    x0[-1] = 1.0
    ref = (scipy.linalg.expm(aug) @ x0)[:n]
    for tol in (1e-8, 1e-12):
        w, st = kiops(1.0, lambda x: A @ x, b, tol=tol, m_min=5)
        assert np.linalg.norm(w - ref) <= 50 * tol * np.linalg.norm(ref) + 1e-14
    # a symmetric case checked independently by eigen-decomposition
    S = -(B @ B.T) / n * 8
    lam, Q = np.linalg.eigh(S)
    ref2 = sum(Q @ (phi_scalar(k, lam) * (Q.T @ b[k])) for k in range(p + 1))
    w2, _ = kiops(1.0, lambda x: S @ x, b, tol=1e-12, m_min=5)
    np.testing.assert_allclose(w2, ref2, rtol=1e-9, atol=1e-10 * np.max(np.abs(ref2)))


def test_happy_breakdown():
    """b inside a 3-dimensional invariant subspace: Arnoldi breaks down after 3
    vectors and the projection is exact."""
    rng = np.random.default_rng(3)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = np.diag(np.concatenate([[-1.0, -2.0, -3.0], -rng.uniform(1, 5, n - 3)]))
    A = Q @ D @ Q.T
    b0 = Q[:, :3] @ rng.standard_normal(3)
    b1 = np.zeros(n)
    w, st = kiops(1.0, lambda x: A @ x, [b0, b1], tol=1e-10, m_min=10)
    np.testing.assert_allclose(w, scipy.linalg.expm(A) @ b0, rtol=1e-12, atol=1e-13)
    assert st['krylov_iters'] <= 5 and st['rejects'] == 0


def test_substepping_on_stiff_operator():
    """A stiff operator forces several substeps and rejections; the result still
    meets the tolerance."""
    n = 200
    h = 1.0 / (n + 1)
    main = -2 * np.ones(n) / h ** 2
    off = np.ones(n - 1) / h ** 2
    A = np.diag(main) + np.diag(off, 1) + np.diag(off, -1)
    x = np.arange(1, n + 1) * h
    b = [np.sin(np.pi * x) + x * (1 - x), np.ones(n)]
    lam, Q = np.linalg.eigh(A * 0.01)
    ref = Q @ (phi_scalar(0, lam) * (Q.T @ b[0])) + Q @ (phi_scalar(1, lam) * (Q.T @ b[1]))
    w, st = kiops(1.0, lambda v: 0.01 * (A @ v), b, tol=1e-10, m_max=40)
    assert st['substeps'] > 1
    assert np.linalg.norm(w - ref) < 1e-8 * np.linalg.norm(ref)


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_non_finite_error_estimate_stops_the_solve():
    """An operator that produces a non-finite value ends the solve with an error
    at the first attempt (the library returns SW_ENONFINITE there) instead of
    rejecting substeps until the limit."""
    n = 20
    calls = []

    def matvec(x):
        calls.append(1)
        y = -x.copy()
        y[3] = np.inf
        return y
    from oracle.kiops import KiopsError
    with pytest.raises(KiopsError, match="non-finite"):
        kiops(1.0, matvec, [np.zeros(n), np.ones(n)], max_rejects=50)
    assert len(calls) <= 10
