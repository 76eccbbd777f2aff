"""Pins of the oracle's right-hand side F(q) and complex-step JVP."""
import numpy as np
import pytest

from oracle import fields, geometry as geo, shallow_water as sw
from paper_2101_05617_gb300 import synth


def _state(ne, ns, seed=0, workload="small_ne4_p3", bottom=False):
    f = synth.make_fields(workload, seed)
    g = sw.Grid(ne, ns, f.rotation)
    h, hB, V = f.evaluate(g.node_xyz())
    if bottom:
        hB = 1500.0 * synth.make_fields("ne90_p6", seed + 7).bottom(g.node_xyz().reshape(3, -1)).reshape(h.shape)
        g.set_bottom(hB)
    return g, fields.state_from_fields(g, h, hB, V)


@pytest.mark.parametrize("ne,ns,seed,bottom", [(2, 3, 0, False), (3, 4, 1, True), (4, 5, 2, False)])
def test_mass_conserved_to_roundoff(ne, ns, seed, bottom):
    """Mass (Eq. 42 with Psi = H) is conserved to machine precision (Sec. 5.4.2):
    sum of w_m w_n dq^0/dt vanishes up to round-off."""
    g, q = _state(ne, ns, seed, bottom=bottom)
    F = sw.rhs_real(g, q)
    w2 = g.w[:, None] * g.w[None, :]
    assert abs(np.sum(F[0] * w2)) < 1e-13 * np.sum(np.abs(F[0]) * w2)


def _rest_state(ne, ns, rot=(0.3, 0.5, -1.0)):
    g = sw.Grid(ne, ns, rot)
    shp = g.x1.shape
    q = fields.state_from_fields(g, np.full(shp, 8000.0), np.zeros(shp), np.zeros((3,) + shp))
    return g, q


def test_rest_state():
    """A flat fluid at rest: the continuity tendency is exactly zero; the
    momentum tendency (pressure-gradient / metric-term imbalance, which the paper
    says is not exactly balanced, Sec. 5.4.2) converges to zero under refinement."""
    errs = []
    for ne in (4, 8, 16):
        g, q = _rest_state(ne, 4)
        F = sw.rhs_real(g, q)
        assert np.max(np.abs(F[0])) == 0.0
        errs.append(np.max(np.abs(F[1:] / q[0])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    # max-norm tendency error of a degree N_s - 1 interpolant: order ~ N_s - 1 = 3
    assert np.all(rates > 2.5), (errs, rates)


def _continuous_rhs(g, f, p, x1, x2, h=1e-5):
    """Exact tendency of Eq. (1)-(2) at points of panel p, with the flux
    divergence by central differences in (x^1, x^2) of the analytic fields."""
    fr = g.frames[p]
    _, php, alp = g.angles[p]

    def qfun(u, v):
        r = geo.unit_position(u, v, fr)
        hh, hB, V = f.evaluate(r)
        t1, t2 = geo.tangent_vectors(u, v, fr)
        m = geo.metric(np.tan(u), np.tan(v))
        c1, c2 = np.sum(V * t1, axis=0), np.sum(V * t2, axis=0)
        u1 = m['h11'] * c1 + m['h12'] * c2
        u2 = m['h12'] * c1 + m['h22'] * c2
        H = hh - hB
        q0 = m['sqrtg'] * H
        return [q0, q0 * u1, q0 * u2], m

    def flux(u, v, j):
        qq, m = qfun(u, v)
        hij = [[m['h11'], m['h12']], [m['h12'], m['h22']]]
        pre = g.gr * qq[0] ** 2 / (2 * m['sqrtg'])
        return [qq[j + 1]] + [qq[i + 1] * qq[j + 1] / qq[0] + pre * hij[i][j] for i in range(2)]

    f1p, f1m = flux(x1 + h, x2, 0), flux(x1 - h, x2, 0)
    f2p, f2m = flux(x1, x2 + h, 1), flux(x1, x2 - h, 1)
    qq, m = qfun(x1, x2)
    X, Y = np.tan(x1), np.tan(x2)
    Gt = geo.christoffel_time(X, Y, php, alp)
    Gs = geo.christoffel_space(X, Y)
    out = []
    for mu in range(3):
        div = (f1p[mu] - f1m[mu]) / (2 * h) + (f2p[mu] - f2m[mu]) / (2 * h)
        s = 0.0
        if mu > 0:
            i = mu - 1
            for j in range(2):
                s = s - 2 * Gt[i][j] * qq[j + 1]
                for k in range(2):
                    s = s - Gs[i][j][k] * qq[j + 1] * qq[k + 1] / qq[0]
        out.append(-div + s)
    return np.array(out)


@pytest.mark.slow
@pytest.mark.parametrize("ns", [3, 4])
def test_h_convergence_of_rhs(ns):
    """On a smooth field the DFR tendency converges to the exact tendency of
    Eq. (1)-(2) as n_e grows, at roughly the formal order N_s (Table 1)."""
    f = synth.make_fields("small_ne4_p3", 3)
    errs = []
    for ne in (4, 8, 16):
        g = sw.Grid(ne, ns, f.rotation)
        h, hB, V = f.evaluate(g.node_xyz())
        q = fields.state_from_fields(g, h, hB, V)
        F = sw.rhs_real(g, q)
        err = 0.0
        scale = 0.0
        for p in range(6):
            ex = _continuous_rhs(g, f, p, g.x1[p].ravel(), g.x2[p].ravel())
            for mu in range(3):
                err = max(err, np.max(np.abs(F[mu, p].ravel() - ex[mu])) / np.max(np.abs(ex[mu])))
        errs.append(err)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > ns - 1.6, (errs, rates)


def test_ausm_consistency_and_mirror_symmetry():
    """AUSM with equal states returns the physical flux of Eq. (136); mirroring
    the normal (swap sides, flip normal velocity) flips the flux."""
    rng = np.random.default_rng(5)
    n = 50
    sqrtg = rng.uniform(2e13, 4e13, n)
    hdd = rng.uniform(2e-14, 4e-14, n)
    h1d, h2d = hdd, rng.uniform(-1e-14, 1e-14, n)
    H = rng.uniform(7000, 9000, n)
    u1 = rng.uniform(-0.3, 0.3, n) * np.sqrt(hdd * 9.80616 * H)
    u2 = rng.uniform(-0.3, 0.3, n) * np.sqrt(hdd * 9.80616 * H)
    q = [sqrtg * H, sqrtg * H * u1, sqrtg * H * u2]
    fl = sw.ausm_flux(q, q, 1, sqrtg, hdd, h1d, h2d, 9.80616)
    phys = [q[1], q[1] * q[1] / q[0] + 9.80616 * q[0] ** 2 / (2 * sqrtg) * h1d,
            q[2] * q[1] / q[0] + 9.80616 * q[0] ** 2 / (2 * sqrtg) * h2d]
    for a, b in zip(fl, phys):
        np.testing.assert_allclose(np.real(a), b, rtol=1e-13)
    H2 = rng.uniform(7000, 9000, n)
    v1 = rng.uniform(-0.3, 0.3, n) * np.sqrt(hdd * 9.80616 * H2)
    r = [sqrtg * H2, sqrtg * H2 * v1, sqrtg * H2 * u2]
    f_lr = sw.ausm_flux(q, r, 1, sqrtg, hdd, h1d, h2d, 9.80616)
    # mirror x^1 -> -x^1: q^1 -> -q^1, h^12 -> -h^12; left and right swap
    qm = [q[0], -q[1], q[2]]
    rm = [r[0], -r[1], r[2]]
    f_m = sw.ausm_flux(rm, qm, 1, sqrtg, hdd, -h1d * 0 + h1d, -h2d, 9.80616)
    np.testing.assert_allclose(np.real(f_m[0]), -np.real(f_lr[0]), rtol=1e-12)
    np.testing.assert_allclose(np.real(f_m[1]), np.real(f_lr[1]), rtol=1e-12)
    np.testing.assert_allclose(np.real(f_m[2]), -np.real(f_lr[2]), rtol=1e-12, atol=1e-12 * np.abs(f_lr[2]).max())


def test_ausm_supersonic_states_take_the_upwind_flux():
    """With both sides supersonic in the same normal direction (|M| > 1, the
    branches the subsonic workloads never reach) the split flux is the upwind
    side's physical flux of Eq. (136): the left one for M > 1, the right one for
    M < -1; and the Mach and pressure splittings are continuous at |M| = 1."""
    rng = np.random.default_rng(8)
    n = 40
    g = 9.80616
    sqrtg = rng.uniform(2e13, 4e13, n)
    hdd = rng.uniform(2e-14, 4e-14, n)
    h1d, h2d = hdd, rng.uniform(-1e-14, 1e-14, n)

    def state(H, mach, tang):
        a = np.sqrt(hdd * g * H)
        return [sqrtg * H, sqrtg * H * mach * a, sqrtg * H * tang * a]

    def phys(q):
        return [q[1], q[1] * q[1] / q[0] + g * q[0] ** 2 / (2 * sqrtg) * h1d,
                q[2] * q[1] / q[0] + g * q[0] ** 2 / (2 * sqrtg) * h2d]
    HL, HR = rng.uniform(7000, 9000, n), rng.uniform(7000, 9000, n)
    for sgn in (1.0, -1.0):
        qL = state(HL, sgn * rng.uniform(1.1, 3.0, n), rng.uniform(-0.5, 0.5, n))
        qR = state(HR, sgn * rng.uniform(1.1, 3.0, n), rng.uniform(-0.5, 0.5, n))
        f = sw.ausm_flux(qL, qR, 1, sqrtg, hdd, h1d, h2d, g)
        ref = phys(qL if sgn > 0 else qR)
        for a, b in zip(f, ref):
            np.testing.assert_allclose(np.real(a), b, rtol=1e-13, atol=1e-13 * np.max(np.abs(b)))
    for m in (-1.0, 1.0):
        for eps in (1e-12, -1e-12):
            lo, hi = np.array(sw.split_mach(m + eps)), np.array(sw.split_mach(m - eps))
            assert np.max(np.abs(lo - hi)) < 1e-10
            lo, hi = np.array(sw.split_pressure(m + eps)), np.array(sw.split_pressure(m - eps))
            assert np.max(np.abs(lo - hi)) < 1e-10


def test_flux_jacobian_eigenvalues():
    """The complex-step Jacobian of the physical flux sqrt(g) T^{mu 1}(q) is
    Eq. (146) with eigenvalues u^1, u^1 +- sqrt(h^11 g_r H) (Eq. 147)."""
    rng = np.random.default_rng(2)
    sqrtg, h11, h12 = 3e13, 3e-14, 4e-15
    H, u1, u2 = 8123.0, 1.1e-6, -0.7e-6
    q = np.array([sqrtg * H, sqrtg * H * u1, sqrtg * H * u2])

    def phys(qq):
        pre = 9.80616 * qq[0] ** 2 / (2 * sqrtg)
        return np.array([qq[1], qq[1] * qq[1] / qq[0] + pre * h11, qq[2] * qq[1] / qq[0] + pre * h12])

    J = np.empty((3, 3))
    for a in range(3):
        e = np.zeros(3, complex)
        e[a] = 1e-30j * abs(q[a])
        J[:, a] = np.imag(phys(q + e)) / (1e-30 * abs(q[a]))
    gH = 9.80616 * H
    expect = np.array([[0, 1, 0], [gH * h11 - u1 * u1, 2 * u1, 0], [gH * h12 - u1 * u2, u2, u1]])
    np.testing.assert_allclose(J, expect, rtol=1e-12, atol=1e-25)
    ev = np.sort(np.linalg.eigvals(J).real)
    a1 = np.sqrt(h11 * gH)
    np.testing.assert_allclose(ev, np.sort([u1 - a1, u1, u1 + a1]), rtol=1e-9)


@pytest.mark.parametrize("ne,ns", [(1, 2), (1, 3), (2, 2)])
def test_jvp_matches_dense_fd_jacobian(ne, ns):
    """Eq. (28) agrees with a dense Jacobian built column by column from central
    differences (Eq. 27 made second order) on a tiny grid."""
    g, q = _state(ne, ns, 4)
    n = q.size
    qf = q.reshape(-1)
    scale = np.repeat(np.abs(q.reshape(3, -1)).mean(axis=1), n // 3)
    J = np.empty((n, n))
    for c in range(n):
        hstep = 1e-6 * scale[c]
        e = np.zeros(n)
        e[c] = hstep
        J[:, c] = (sw.rhs_real(g, qf + e).reshape(-1) - sw.rhs_real(g, qf - e).reshape(-1)) / (2 * hstep)
    v = synth.random_perturbation(n, 9) * scale
    jv = sw.jvp(g, q, v).reshape(-1)
    assert np.linalg.norm(jv - J @ v) < 1e-7 * np.linalg.norm(jv)


def test_jvp_linear_and_eps_independent():
    g, q = _state(2, 4, 6)
    n = q.size
    s = np.repeat(np.abs(q.reshape(3, -1)).mean(axis=1), n // 3)
    v = synth.random_perturbation(n, 1) * s
    w = synth.random_perturbation(n, 2) * s
    a, b = sw.jvp(g, q, v), sw.jvp(g, q, w)
    c = sw.jvp(g, q, 2 * v + 3 * w)
    assert np.linalg.norm(c - 2 * a - 3 * b) < 1e-14 * np.linalg.norm(c)
    # the paper's eps ~ 1.5e-8 relative to the state (Sec. 5) gives the same JVP
    d = sw.jvp(g, q, v / np.linalg.norm(v) * np.linalg.norm(q), eps=1.5e-8) * np.linalg.norm(v) / np.linalg.norm(q)
    assert np.linalg.norm(d - a) < 1e-12 * np.linalg.norm(a)
