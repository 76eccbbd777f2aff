"""Shared helpers of the GPU parity tests: seeded inputs built by the oracle
(oracle geometry + seeded fields) so that both sides see identical arrays."""
import numpy as np

from oracle import fields as ofields
from oracle import shallow_water as osw
from paper_2101_05617_gb300 import synth


def oracle_case(ne, ns, workload="small_ne4_p3", seed=0, bottom_amp=0.0):
    f = synth.make_fields(workload, seed)
    g = osw.Grid(ne, ns, f.rotation)
    h, hB, V = f.evaluate(g.node_xyz())
    if bottom_amp > 0:
        bf = synth.make_fields("ne90_p6", seed + 11).bottom
        hB = bottom_amp * bf(g.node_xyz().reshape(3, -1)).reshape(h.shape)
    g.set_bottom(hB)
    q = ofields.state_from_fields(g, h, hB, V)
    return f, g, q, hB


def scaled_direction(q, seed):
    """A seeded direction with each variable scaled like the state."""
    v = synth.random_perturbation(q.size, seed).reshape(q.shape)
    for var in range(3):
        v[var] *= np.abs(q[var]).mean()
    return v


def rel_err_per_var(a, b):
    a = np.asarray(a).reshape(3, -1)
    b = np.asarray(b).reshape(3, -1)
    return [float(np.max(np.abs(a[k] - b[k])) / np.max(np.abs(b[k]))) for k in range(3)]


def rel_l2_per_var(a, b):
    a = np.asarray(a).reshape(3, -1)
    b = np.asarray(b).reshape(3, -1)
    return [float(np.linalg.norm(a[k] - b[k]) / np.linalg.norm(b[k])) for k in range(3)]


def term_scale(g, q, v=None, eps=1e-30):
    """Per-variable magnitude of the terms the DFR sums: (2/dx) max_k sum_n |D_kn|
    times the largest nodal flux of that variable (its tangent for a JVP), plus
    the largest source.  Rounding errors of any evaluation order scale with it;
    the tendency itself can be a small residual of these terms (balanced flow)."""
    z = np.asarray(q, dtype=complex).reshape((3,) + g.x1.shape)
    if v is not None:
        z = z + 1j * eps * np.asarray(v).reshape(z.shape)
    m = g.m
    pre = g.gr * z[0] ** 2 / (2 * m['sqrtg'])
    hij = [[m['h11'], m['h12']], [m['h12'], m['h22']]]
    part = (lambda x: np.abs(np.imag(x)) / eps) if v is not None else (lambda x: np.abs(np.real(x)))
    fl = [max(np.max(part(z[1])), np.max(part(z[2])))]
    for i in range(2):
        fl.append(max(np.max(part(z[i + 1] * z[j + 1] / z[0] + pre * hij[i][j])) for j in range(2)))
    dsum = np.max(np.sum(np.abs(g.D), axis=1)) * 2.0 / g.dx
    return [dsum * f for f in fl]


def scaled_err_per_var(a, b, scale):
    a = np.asarray(a).reshape(3, -1)
    b = np.asarray(b).reshape(3, -1)
    return [float(np.max(np.abs(a[k] - b[k])) / scale[k]) for k in range(3)]
