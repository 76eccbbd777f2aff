"""Direct flux reconstruction operators (paper Sec. 3.1), plain numpy FP64.

Test infrastructure only (see ``oracle/__init__.py``).
"""
import numpy as np


def gauss_legendre(ns):
    """N_s Gauss-Legendre points and weights on [-1, 1] (Sec. 3.1: the solution
    points are the roots of the Legendre polynomial).  numpy's leggauss is used
    as a library primitive."""
    xi, w = np.polynomial.legendre.leggauss(ns)
    return xi, w


def lagrange_values(nodes, x):
    """ell_k(x) of Eq. (8) for every node k at the points x: returns [len(x), N]."""
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(nodes)
    out = np.ones((len(x), n))
    for k in range(n):
        for l in range(n):
            if l != k:
                out[:, k] *= (x - nodes[l]) / (nodes[k] - nodes[l])
    return out


def lagrange_derivatives(nodes, x):
    """ell'_n(x) written out as Eq. (13): sum over i != n of 1/(xi_n - xi_i)
    times the product over m != i, n of (x - xi_m)/(xi_n - xi_m).
    Returns [len(x), N]."""
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(nodes)
    out = np.zeros((len(x), n))
    for j in range(n):          # the basis function index ("n" in Eq. 13)
        for i in range(n):
            if i == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[i]))
            for m in range(n):
                if m != i and m != j:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            out[:, j] += term
    return out


def extended_nodes(ns):
    """{xi_0 = -1, xi_1..xi_Ns (Gauss-Legendre), xi_{Ns+1} = +1} (Sec. 3.1)."""
    xi, _ = gauss_legendre(ns)
    return np.concatenate(([-1.0], xi, [1.0]))


def flux_derivative_matrix(ns):
    """D[k, n] = ell~'_n(xi_k): derivative at solution point k of the Lagrange
    polynomial of extended node n (Eq. 12-13), shape [N_s, N_s + 2]."""
    xi, _ = gauss_legendre(ns)
    return lagrange_derivatives(extended_nodes(ns), xi)


def trace_rows(ns):
    """ell_k(-1) and ell_k(+1) (Eq. 7-8 evaluated at the element ends)."""
    xi, _ = gauss_legendre(ns)
    v = lagrange_values(xi, [-1.0, 1.0])
    return v[0], v[1]


def collocation_derivative_matrix(ns):
    """Dg[k, l] = ell'_l(xi_k) on the Gauss-Legendre points alone (Sec. 3.1 basis; used for the
    bottom-topography gradient, which the paper does not specify)."""
    xi, _ = gauss_legendre(ns)
    return lagrange_derivatives(xi, xi)
