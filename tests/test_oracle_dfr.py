"""Pins of the DFR operators (Sec. 3.1, Eq. 7-14)."""
import numpy as np
import pytest

from oracle import dfr


@pytest.mark.parametrize("ns", [1, 2, 3, 4, 5, 6, 7, 8])
def test_derivative_exact_on_extended_polynomials(ns):
    """F'_j of Eq. (12) is exact for polynomials of degree <= N_s + 1 sampled on
    the extended nodes (Eq. 11 interpolates them exactly)."""
    D = dfr.flux_derivative_matrix(ns)
    xe = dfr.extended_nodes(ns)
    xi, _ = dfr.gauss_legendre(ns)
    for deg in range(ns + 2):
        np.testing.assert_allclose(D @ xe ** deg, deg * xi ** max(deg - 1, 0) if deg else 0 * xi, atol=1e-11)
    np.testing.assert_allclose(D.sum(axis=1), 0, atol=1e-12)


@pytest.mark.parametrize("ns", [1, 2, 3, 4, 5, 6, 7])
def test_radau_mass_property(ns):
    """sum_k w_k ell~'_n(xi_k) = ell~_n(1) - ell~_n(-1): Gauss-Legendre quadrature
    of F' is exact (degree N_s <= 2 N_s - 1), the discrete mass budget telescopes
    to the interface fluxes (Sec. 3.1 equivalence with the weak NDG form)."""
    D = dfr.flux_derivative_matrix(ns)
    _, w = dfr.gauss_legendre(ns)
    expect = np.zeros(ns + 2)
    expect[0], expect[-1] = -1.0, 1.0
    np.testing.assert_allclose(w @ D, expect, atol=1e-12)


@pytest.mark.parametrize("ns", [2, 3, 4, 6])
def test_gauss_legendre_exactness(ns):
    xi, w = dfr.gauss_legendre(ns)
    for deg in range(2 * ns):
        exact = (1 - (-1) ** (deg + 1)) / (deg + 1)
        assert abs(np.sum(w * xi ** deg) - exact) < 1e-13


@pytest.mark.parametrize("ns", [2, 3, 5])
def test_traces_and_collocation(ns):
    xi, _ = dfr.gauss_legendre(ns)
    lm, lp = dfr.trace_rows(ns)
    Dg = dfr.collocation_derivative_matrix(ns)
    for deg in range(ns):
        assert abs(lm @ xi ** deg - (-1.0) ** deg) < 1e-12
        assert abs(lp @ xi ** deg - 1.0) < 1e-12
        np.testing.assert_allclose(Dg @ xi ** deg, deg * xi ** max(deg - 1, 0) if deg else 0 * xi, atol=1e-11)


def test_dfr_1d_advection_matches_upwind_ndg():
    """1-D DFR with upwind interface fluxes on periodic f(q) = q: the semi-discrete
    derivative of a polynomial of degree <= N_s - 1 that is continuous across
    elements (so every interface flux equals the trace) is exact."""
    ns, ne = 4, 5
    D = dfr.flux_derivative_matrix(ns)
    xi, _ = dfr.gauss_legendre(ns)
    lm, lp = dfr.trace_rows(ns)
    dx = 1.0 / ne
    x = (np.arange(ne)[:, None] + 0.5) * dx + xi[None] * dx / 2
    q = 3 * x ** 3 - x ** 2 + 2 * x        # degree 3 = N_s - 1, continuous
    right = q @ lp                           # trace at xi = +1 of each element
    left_face = np.concatenate([[0.0], right[:-1]])   # upwind flux at the left face
    left_face[0] = q[0] @ lm                 # boundary: use own trace
    ext = np.concatenate([left_face[:, None], q, right[:, None]], axis=1)
    dqdx = (2 / dx) * ext @ D.T
    np.testing.assert_allclose(dqdx, 9 * x ** 2 - 2 * x + 2, rtol=1e-11)
