"""Multistep exponential propagation iterative (EPI) methods, Eq. (25), (30),
(34)-(38), with EPI2 start-up (Sec. 4).  Plain numpy FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Readings: v_m carries the factor Delta t as in Eq. (35) (the step list after
Eq. 38 writes it without Delta t and multiplies w_n by Delta t instead, which
is the same update); the first P steps use N_sub = 8 EPI2 substeps of
Delta t / N_sub each (the paper fixes only that the start-up steps are
shorter, not by how much).
"""
from fractions import Fraction as Fr

import numpy as np

from .kiops import kiops

# Rows m = 1..M (phi_m), columns i = 1..P (q_{n-i}); Eq. (30) and (36)-(38).
COEFFS = {
    3: [[Fr(0)], [Fr(2, 3)]],
    4: [[Fr(0), Fr(0)], [Fr(-3, 10), Fr(3, 40)], [Fr(32, 5), Fr(-11, 10)]],
    5: [[Fr(0), Fr(0), Fr(0)], [Fr(-4, 5), Fr(2, 5), Fr(-4, 45)], [Fr(12), Fr(-9, 2), Fr(8, 9)],
        [Fr(3), Fr(0), Fr(-1, 3)]],
    6: [[Fr(0), Fr(0), Fr(0), Fr(0)],
        [Fr(-49, 60), Fr(351, 560), Fr(-359, 1260), Fr(367, 6720)],
        [Fr(92, 7), Fr(-99, 14), Fr(176, 63), Fr(-1, 2)],
        [Fr(485, 21), Fr(-151, 14), Fr(23, 9), Fr(-31, 168)]],
}

N_SUB_STARTUP = 8


def history_length(order):
    """P, the number of past states q_{n-1} .. q_{n-P} the scheme of Eq. (34)-(38) uses."""
    return 0 if order == 2 else len(COEFFS[order][0])


class EPI:
    """State of a multistep EPI integration of dq/dt = F(q) (Eq. 21).

    rhs(q) -> F(q); jvp(q, v) -> J(q) v.  The history holds (q_{n-i}, F(q_{n-i}))
    for i = 1..P, most recent first."""

    def __init__(self, rhs, jvp, order, tol=1e-10, m_init=10, m_min=10, m_max=128, iop=2,
                 n_sub=N_SUB_STARTUP):
        self.rhs, self.jvp, self.order = rhs, jvp, order
        self.kopts = dict(tol=tol, m_min=m_min, m_max=m_max, iop=iop)
        self.m_init = m_init
        self.n_sub = n_sub
        self.history = []
        self.stats = []

    def _phi(self, q, dt, b):
        w, st = kiops(1.0, lambda x: dt * self.jvp(q, x), b, m_init=self.m_init, **self.kopts)
        self.m_init = st['m_final']
        self.stats.append(st)
        return w

    def epi2(self, q, dt):
        """Exponential Euler, Eq. (25)."""
        F = self.rhs(q)
        return q + self._phi(q, dt, [np.zeros_like(q), dt * F]), F

    def step(self, q, dt):
        """q_{n+1} by Eq. (34)-(35) with the remainders of Eq. (33) (EPI2 substeps of
        Eq. 25 while the history is short: the start-up of Sec. 4)."""
        q = np.asarray(q, dtype=float)
        P = history_length(self.order)
        if len(self.history) < P:
            Fn = self.rhs(q)
            qs = q
            h = dt / self.n_sub
            for _ in range(self.n_sub):
                qs, _ = self.epi2(qs, h)
            self.history.insert(0, (q, Fn))
            return qs
        if self.order == 2:
            out, _ = self.epi2(q, dt)
            return out
        A = COEFFS[self.order]
        M = len(A)
        Fn = self.rhs(q)
        R = []
        for i in range(1, P + 1):                      # Eq. (33) / remainder R(q_{n-i})
            qi, Fi = self.history[i - 1]
            R.append(Fi - Fn - self.jvp(q, qi - q))
        v = []
        for mrow in range(M):                          # Eq. (35)
            vm = np.zeros_like(q)
            for i in range(P):
                vm = vm + float(A[mrow][i]) * dt * R[i]
            v.append(vm)
        b = [np.zeros_like(q), dt * Fn + v[0]] + v[1:]  # Eq. (34) with b_0 = 0
        w = self._phi(q, dt, b)
        self.history.insert(0, (q, Fn))
        del self.history[P:]
        return q + w
