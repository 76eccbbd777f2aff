"""The semilinear parabolic test problem of Sec. 5.1, discretised (test
infrastructure only).

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
        return np.exp(t) * (self.s0 - self.L0 - self.T0)

    def exact(self, t):
        return np.concatenate([self.s0 * np.exp(t), [t]])

    def rhs(self, y):
        u, t = y[:-1], y[-1]
        return np.concatenate([self._lap(u) + self._int(u) + self.phi(t), [1.0]])

    def jvp(self, y, v):
        vu, vt = v[:-1], v[-1]
        t = y[-1]
        return np.concatenate([self._lap(vu) + self._int(vu) + self.phi(t) * vt, [0.0]])
