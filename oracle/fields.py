"""State q from physical fields at the nodes (test infrastructure only).

Given the free-surface height h, the bottom height h_B and the wind as a
Cartesian 3-vector V (m/s) at every node, the state of Eq. (1)-(2) is
q^0 = sqrt(g) H with H = h - h_B, and q^i = sqrt(g) H u^i with the
contravariant components u^i = h^{ij} (V . t_j), t_j = d(a r)/dx^j.
"""
import numpy as np

from . import geometry as geo


def state_from_fields(grid, h, hB, V):
    """q of Eq. (1)-(2) (q^0 = sqrt(g) H, q^i = q^0 u^i, App. D) from h, h_B and the
    Cartesian wind at the nodes, u^i = h^{ij} (V . t_j) with Eq. (67)-(69)."""
    shp = grid.x1.shape
    h = np.asarray(h, dtype=float).reshape(shp)
    hB = np.asarray(hB, dtype=float).reshape(shp)
    V = np.asarray(V, dtype=float).reshape((3,) + shp)
    H = h - hB
    u1 = np.empty(shp)
    u2 = np.empty(shp)
    for p in range(6):
        t1, t2 = geo.tangent_vectors(grid.x1[p], grid.x2[p], grid.frames[p], grid.a)
        c1 = np.einsum('k...,k...->...', V[:, p], t1)      # covariant u_1
        c2 = np.einsum('k...,k...->...', V[:, p], t2)
        m = grid.m
        u1[p] = m['h11'][p] * c1 + m['h12'][p] * c2
        u2[p] = m['h12'][p] * c1 + m['h22'][p] * c2
    sg = grid.m['sqrtg']
    return np.stack([sg * H, sg * H * u1, sg * H * u2])


def wind_from_state(grid, q):
    """Inverse map of state_from_fields (diagnostics of Sec. 5): Cartesian wind and H from q."""
    shp = grid.x1.shape
    q = np.asarray(q).reshape((3,) + shp)
    H = q[0] / grid.m['sqrtg']
    u1, u2 = q[1] / q[0], q[2] / q[0]
    V = np.empty((3,) + shp)
    for p in range(6):
        t1, t2 = geo.tangent_vectors(grid.x1[p], grid.x2[p], grid.frames[p], grid.a)
        V[:, p] = t1 * u1[p] + t2 * u2[p]
    return H, V
