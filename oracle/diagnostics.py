"""Diagnostics of Sec. 5 (test infrastructure only): the Gauss-Legendre global
integral Eq. (42), the error norms Eq. (39)-(41), relative vorticity Eq. (43),
the Coriolis parameter Eq. (45)-(46), and the integrands of mass, total energy
and potential enstrophy whose normalised drift Eq. (44) the paper monitors.

Reading: the paper does not say how the derivative in Eq. (43) is discretised;
it is the element-local collocation derivative of the covariant velocity
u_j = g_jk u^k (as for the bottom gradient).  Eq. (42) is written without the
element Jacobian (dx/2)^2, which is the same for every element; it is kept out
here too, so integrals are in units of the angular coordinates."""
import numpy as np

from . import geometry as geo


def integral(grid, psi):
    """Eq. (42): sum of Psi sqrt(g) w_m w_n over all nodes."""
    w2 = grid.w[:, None] * grid.w[None, :]
    return float(np.sum(np.asarray(psi).reshape(grid.x1.shape) * grid.m['sqrtg'] * w2))


def primitives(grid, q):
    """H = q^0 / sqrt(g) and u^i = q^i / q^0 (the state of Eq. 1-2, App. D)."""
    q = np.asarray(q).reshape((3,) + grid.x1.shape)
    H = q[0] / grid.m['sqrtg']
    u1, u2 = q[1] / q[0], q[2] / q[0]
    return H, u1, u2


def coriolis_parameter(grid):
    """Eq. (46): f = 2 Omega s / delta with s the bracket of Eq. (71)-(74)."""
    f = np.empty(grid.x1.shape)
    X, Y = np.tan(grid.x1), np.tan(grid.x2)
    for p in range(6):
        _, php, alp = grid.angles[p]
        d = np.sqrt(1 + X[p] ** 2 + Y[p] ** 2)
        f[p] = 2 * grid.omega / d * geo.coriolis_bracket(X[p], Y[p], php, alp)
    return f


def relative_vorticity(grid, q):
    """Eq. (43): (d_1 u_2 - d_2 u_1) / sqrt(g), u_j = g_jk u^k."""
    H, u1, u2 = primitives(grid, q)
    m = grid.m
    c1 = m['g11'] * u1 + m['g12'] * u2
    c2 = m['g12'] * u1 + m['g22'] * u2
    s = 2.0 / grid.dx
    d1c2 = s * np.einsum('kl,pefjl->pefjk', grid.Dg, c2)     # d/dx^1 along k1
    d2c1 = s * np.einsum('kl,pefli->pefki', grid.Dg, c1)     # d/dx^2 along k2
    return (d1c2 - d2c1) / m['sqrtg']


def invariants(grid, q):
    """(mass, total energy, potential enstrophy) integrals (Sec. 5.4, Eq. 44)."""
    H, u1, u2 = primitives(grid, q)
    m = grid.m
    hB = grid.hB
    uu = m['g11'] * u1 * u1 + 2 * m['g12'] * u1 * u2 + m['g22'] * u2 * u2
    energy = 0.5 * (H * uu + grid.gr * ((H + hB) ** 2 - hB ** 2))
    zeta = relative_vorticity(grid, q)
    f = coriolis_parameter(grid)
    enstrophy = (zeta + f) ** 2 / (2 * H)
    return integral(grid, H), integral(grid, energy), integral(grid, enstrophy)


def error_norms(grid, H, HT):
    """Eq. (39)-(41): L1, L2, Linf of H against a reference H_T."""
    H = np.asarray(H).reshape(grid.x1.shape)
    HT = np.asarray(HT).reshape(grid.x1.shape)
    l1 = integral(grid, np.abs(H - HT)) / integral(grid, HT)
    l2 = np.sqrt(integral(grid, (H - HT) ** 2) / integral(grid, HT ** 2))
    linf = np.max(np.abs(H - HT)) / np.max(np.abs(HT))
    return l1, l2, linf
