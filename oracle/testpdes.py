"""The three test problems of Sec. 5.1, discretised (test infrastructure
only): the semilinear parabolic PDE, the advection-diffusion-reaction PDE and
Burgers' equation.

Semilinear parabolic PDE:
u_t = u_xx + int_0^1 u(s, t) ds + phi(x, t) on (0, 1), u = 0 at both ends.
Readings: the garbled integral is a spatial integral of u; u_xx is the
second-order central difference on n interior points x_i = i/(n+1) and the
integral the trapezoidal rule; phi is built from the discrete operators so that
u_i(t) = x_i (1 - x_i) e^t solves the semi-discrete system exactly, which
isolates the temporal error.  Time is appended as an extra unknown (dt/dt = 1)
to make the system autonomous as Eq. (21) requires.
"""
import numpy as np


class SemilinearParabolic:
    """The semilinear parabolic problem of Sec. 5.1 (readings in the module docstring)."""
    def __init__(self, n=50):
        self.n = n
        self.h = 1.0 / (n + 1)
        self.x = np.arange(1, n + 1) * self.h
        s0 = self.x * (1 - self.x)
        self.s0 = s0
        self.T0 = self.h * np.sum(s0)                   # trapezoid of x(1-x) (end values 0)
        self.L0 = self._lap(s0)

    def _lap(self, u):
        up = np.concatenate([[0.0], u, [0.0]])
        return (up[:-2] - 2 * up[1:-1] + up[2:]) / self.h ** 2

    def _int(self, u):
        return self.h * np.sum(u)

    def phi(self, t):
        """The forcing of the semilinear problem of Sec. 5.1 (built from the discrete operators)."""
        return np.exp(t) * (self.s0 - self.L0 - self.T0)

    def exact(self, t):
        """The exact solution x (1 - x) e^t of Sec. 5.1 (and t)."""
        return np.concatenate([self.s0 * np.exp(t), [t]])

    def rhs(self, y):
        """Right-hand side of the semi-discrete problem (Sec. 5.1)."""
        u, t = y[:-1], y[-1]
        return np.concatenate([self._lap(u) + self._int(u) + self.phi(t), [1.0]])

    def jvp(self, y, v):
        """Exact Jacobian times v (Sec. 5.1 uses the exact Jacobian)."""
        vu, vt = v[:-1], v[-1]
        t = y[-1]
        return np.concatenate([self._lap(vu) + self._int(vu) + self.phi(t) * vt, [0.0]])


class AdvectionDiffusionReaction:
    """u_t + alpha (u_x + u_y) = eps (u_xx + u_yy) + gamma u (u - 1/2) (1 - u) on
    [0, 1]^2 with homogeneous Neumann boundaries, eps = 1/100, alpha = -10,
    gamma = 100, u_0 = 256 (x y (1 - x) (1 - y))^2 + 0.3, t in [0, 0.1]
    (Sec. 5.1).  Readings: the n = 1600 grid points are the 40 x 40 cell centres
    (i + 1/2)/40; both derivatives are second-order central differences; the
    Neumann condition is a reflection (the ghost value equals the adjacent
    interior value)."""

    T = 0.1

    def __init__(self, m=40, eps=0.01, alpha=-10.0, gamma=100.0):
        self.m, self.eps, self.alpha, self.gamma = m, eps, alpha, gamma
        self.h = 1.0 / m
        x = (np.arange(m) + 0.5) * self.h
        X, Y = np.meshgrid(x, x, indexing="ij")
        self.u0 = (256.0 * (X * Y * (1 - X) * (1 - Y)) ** 2 + 0.3).ravel()

    def _lin(self, v):
        """eps (v_xx + v_yy) - alpha (v_x + v_y), second-order, reflected ghosts."""
        V = v.reshape(self.m, self.m)
        P = np.pad(V, 1, mode="edge")
        lap = (P[2:, 1:-1] + P[:-2, 1:-1] + P[1:-1, 2:] + P[1:-1, :-2] - 4.0 * V) / self.h ** 2
        adv = (P[2:, 1:-1] - P[:-2, 1:-1] + P[1:-1, 2:] - P[1:-1, :-2]) / (2.0 * self.h)
        return (self.eps * lap - self.alpha * adv).ravel()

    def rhs(self, u):
        """Right-hand side of the semi-discrete problem (Sec. 5.1)."""
        return self._lin(u) + self.gamma * u * (u - 0.5) * (1.0 - u)

    def jvp(self, u, v):
        """Exact Jacobian times v (Sec. 5.1 uses the exact Jacobian)."""
        return self._lin(v) + self.gamma * (-3.0 * u * u + 3.0 * u - 0.5) * v

    def jacobian(self, u):
        """The Jacobian as a sparse matrix, assembled from the 1-D stencils
        (for an implicit reference solver as in Sec. 5.1; equal to jvp)."""
        import scipy.sparse as sps
        m, h = self.m, self.h
        e = np.ones(m)
        d2 = sps.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], format="lil")
        d2[0, 0] = d2[m - 1, m - 1] = -1.0                  # reflected ghosts
        d1 = sps.diags([-e[:-1], e[:-1]], [-1, 1], format="lil")
        d1[0, 0], d1[m - 1, m - 1] = -1.0, 1.0
        d2, d1 = d2.tocsr() / h ** 2, d1.tocsr() / (2.0 * h)
        I = sps.identity(m, format="csr")
        L = self.eps * (sps.kron(d2, I) + sps.kron(I, d2)) - self.alpha * (sps.kron(d1, I) + sps.kron(I, d1))
        return (L + sps.diags(self.gamma * (-3.0 * u * u + 3.0 * u - 0.5))).tocsr()


class Burgers:
    """u_t + (u^2 / 2)_x = eps u_xx on [0, 1] with homogeneous Dirichlet
    boundaries, eps = 1e-3, u_0 = exp(-(x - 0.3)^2 / (2 0.05^2)), t in [0, 1]
    (Sec. 5.1).  Readings: the n = 1024 grid points are interior,
    x_i = i / 1025; both derivatives are second-order central differences, the
    convective term differencing u^2 / 2."""

    T = 1.0

    def __init__(self, n=1024, eps=1e-3, mu=0.3, sigma=0.05):
        self.n, self.eps = n, eps
        self.h = 1.0 / (n + 1)
        x = np.arange(1, n + 1) * self.h
        self.u0 = np.exp(-(x - mu) ** 2 / (2.0 * sigma ** 2))

    def _d2(self, v):
        P = np.pad(v, 1)
        return (P[2:] - 2.0 * v + P[:-2]) / self.h ** 2

    def _d1(self, v):
        P = np.pad(v, 1)
        return (P[2:] - P[:-2]) / (2.0 * self.h)

    def rhs(self, u):
        """Right-hand side of the semi-discrete problem (Sec. 5.1)."""
        return self.eps * self._d2(u) - 0.5 * self._d1(u * u)

    def jvp(self, u, v):
        """Exact Jacobian times v (Sec. 5.1 uses the exact Jacobian)."""
        return self.eps * self._d2(v) - self._d1(u * v)

    def jacobian(self, u):
        """The Jacobian as a sparse matrix (for an implicit reference solver as in
        Sec. 5.1; equal to jvp)."""
        import scipy.sparse as sps
        n, h = self.n, self.h
        e = np.ones(n)
        d2 = sps.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], format="csr") / h ** 2
        d1 = sps.diags([-e[:-1], e[:-1]], [-1, 1], format="csr") / (2.0 * h)
        return (self.eps * d2 - d1 @ sps.diags(u)).tocsr()
