"""Readers of the fixtures under tests/golden/ (values printed in the paper)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def golden_app_c():
    """App. C, Eq. (100)-(135): per interface p, q, Z and the symbolic 2 x 2
    contravariant (M) and covariant (C) matrices."""
    out = []
    for t in _rows("app_c_relations.txt"):
        out.append({"p": int(t[0]), "q": int(t[1]), "Z": t[2], "M": t[3:7], "C": t[7:11], "eq": t[11]})
    return out


def entries(sym, s):
    """2 x 2 (x len(s)) array from symbolic entries 0, 1, -1, s, -s."""
    s = np.asarray(s, dtype=float)
    val = {"0": 0.0 * s, "1": 1.0 + 0.0 * s, "-1": -1.0 + 0.0 * s, "s": s, "-s": -s}
    return np.array([[val[sym[0]], val[sym[1]]], [val[sym[2]], val[sym[3]]]])


def golden_epi_coefficients():
    """Eq. (30), (36)-(38): {order: A as nested lists of Fractions}."""
    A = {}
    for order, row, col, v in _rows("epi_coefficients.txt"):
        order, row, col = int(order), int(row), int(col)
        A.setdefault(order, {})[(row, col)] = Fraction(v)
    out = {}
    for order, d in A.items():
        M = max(r for r, _ in d)
        P = max(c for _, c in d)
        out[order] = [[d[(r, c)] for c in range(1, P + 1)] for r in range(1, M + 1)]
    return out


def golden_dfr_orders():
    """Table 1: {N_s: (L1, L2, Linf) order of accuracy}."""
    return {int(t[0]): tuple(float(x) for x in t[1:4]) for t in _rows("dfr_orders_table1.txt")}
