"""Pins of the oracle's geometry (App. B, App. C) against the 3-D embedding."""
import numpy as np
import pytest

from oracle import geometry as geo
from tests.golden_tables import entries, golden_app_c

ROTATIONS = [(0.0, 0.0, 0.0), (0.0, np.pi / 4, 0.0), (0.7, -0.4, 1.9), (-2.5, 0.9, -0.3)]


def _pts(n=64, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi / 4, np.pi / 4, n), rng.uniform(-np.pi / 4, np.pi / 4, n)


def test_metric_matches_embedding():
    """g_ij of Eq. (64)-(66) equal t_i . t_j of the embedded surface; h^ij of
    Eq. (67)-(69) is their inverse; sqrt(g) of Eq. (70) is sqrt(det g)."""
    x1, x2 = _pts()
    fr = geo.panel_frame(*geo.panel_angles(0.3, 0.2, 0.1)[2])
    t1, t2 = geo.tangent_vectors(x1, x2, fr)
    m = geo.metric(np.tan(x1), np.tan(x2))
    for a, b, key in ((t1, t1, 'g11'), (t1, t2, 'g12'), (t2, t2, 'g22')):
        np.testing.assert_allclose(np.sum(a * b, axis=0), m[key], rtol=1e-12, atol=1e-13 * geo.RADIUS ** 2)
    det = m['g11'] * m['g22'] - m['g12'] ** 2
    np.testing.assert_allclose(m['sqrtg'], np.sqrt(det), rtol=1e-13)
    np.testing.assert_allclose(m['h11'] * m['g11'] + m['h12'] * m['g12'], 1, rtol=1e-13)
    np.testing.assert_allclose(m['h11'] * m['g12'] + m['h12'] * m['g22'], 0, atol=1e-13)
    np.testing.assert_allclose(m['h12'] * m['g12'] + m['h22'] * m['g22'], 1, rtol=1e-13)


def _num_deriv(f, x1, x2, h=1e-6):
    return ((f(x1 + h, x2) - f(x1 - h, x2)) / (2 * h), (f(x1, x2 + h) - f(x1, x2 - h)) / (2 * h))


def test_spatial_christoffel_is_levi_civita():
    """Eq. (75)-(80) equal the Levi-Civita connection of g_ij (Eq. 50)."""
    x1, x2 = _pts(32, 1)
    a = geo.RADIUS

    def g(i, j):
        key = 'g' + str(min(i, j) + 1) + str(max(i, j) + 1)
        return lambda u, v: geo.metric(np.tan(u), np.tan(v))[key] / a ** 2

    dg = {(i, j): _num_deriv(g(i, j), x1, x2) for i in range(2) for j in range(2)}
    m = geo.metric(np.tan(x1), np.tan(x2))
    hinv = [[m['h11'] * a * a, m['h12'] * a * a], [m['h12'] * a * a, m['h22'] * a * a]]
    G = geo.christoffel_space(np.tan(x1), np.tan(x2))
    for i in range(2):
        for j in range(2):
            for k in range(2):
                lc = sum(0.5 * hinv[i][l] * (dg[(l, j)][k] + dg[(l, k)][j] - dg[(j, k)][l]) for l in range(2))
                np.testing.assert_allclose(G[i][j][k], lc, atol=1e-8)


def test_contraction_vanishes():
    """h^jk Gamma^i_jk = 0 on the cubed sphere (App. B, after Eq. 80) and
    d(sqrt(g) h^ij)/dx^j = 0 (App. A identity)."""
    x1, x2 = _pts()
    X, Y = np.tan(x1), np.tan(x2)
    m = geo.metric(X, Y)
    G = geo.christoffel_space(X, Y)
    h = [[m['h11'], m['h12']], [m['h12'], m['h22']]]
    for i in range(2):
        c = sum(h[j][k] * G[i][j][k] for j in range(2) for k in range(2))
        assert np.max(np.abs(c * geo.RADIUS ** 2)) < 1e-13
        f = lambda u, v, i=i, j=0: (geo.metric(np.tan(u), np.tan(v))['sqrtg'] * (
            geo.metric(np.tan(u), np.tan(v))['h11' if i == 0 else 'h12']))
        f2 = lambda u, v, i=i: (geo.metric(np.tan(u), np.tan(v))['sqrtg'] * (
            geo.metric(np.tan(u), np.tan(v))['h12' if i == 0 else 'h22']))
        div = _num_deriv(f, x1, x2)[0] + _num_deriv(f2, x1, x2)[1]
        assert np.max(np.abs(div)) < 1e-7


@pytest.mark.parametrize("rot", ROTATIONS)
def test_coriolis_christoffel_from_spacetime_metric(rot):
    """Eq. (71)-(74) equal (1/2) h^ik (d_j g_k0 - d_k g_0j) built from Eq. (62)-(63),
    and g_0j of Eq. (62)-(63) equals the rotating-frame velocity Omega z x (a r)
    dotted with the covariant basis vector t_j."""
    x1, x2 = _pts(32, 2)
    for p, ang in enumerate(geo.panel_angles(*rot)):
        _, php, alp = ang
        fr = geo.panel_frame(*ang)
        g0 = lambda u, v, k: geo.spacetime_metric_g0(np.tan(u), np.tan(v), php, alp)[k]
        r = geo.unit_position(x1, x2, fr)
        t1, t2 = geo.tangent_vectors(x1, x2, fr)
        vel = geo.OMEGA * geo.RADIUS * np.stack([-r[1], r[0], np.zeros_like(r[0])])
        np.testing.assert_allclose(g0(x1, x2, 1), np.sum(vel * t1, axis=0), rtol=1e-12, atol=1e-3)
        np.testing.assert_allclose(g0(x1, x2, 2), np.sum(vel * t2, axis=0), rtol=1e-12, atol=1e-3)
        d = {k: _num_deriv(lambda u, v: g0(u, v, k), x1, x2, 1e-5) for k in (1, 2)}
        m = geo.metric(np.tan(x1), np.tan(x2))
        h = [[m['h11'], m['h12']], [m['h12'], m['h22']]]
        G = geo.christoffel_time(np.tan(x1), np.tan(x2), php, alp)
        for i in range(2):
            for j in range(2):
                val = sum(0.5 * h[i][k] * (d[k + 1][j] - d[j + 1][k]) for k in range(2))
                np.testing.assert_allclose(G[i][j], val, atol=1e-12)


@pytest.mark.parametrize("rot", ROTATIONS)
def test_coriolis_parameter(rot):
    """f of Eq. (46) equals 2 Omega sin(latitude) (Eq. 45)."""
    x1, x2 = _pts()
    for ang in geo.panel_angles(*rot):
        fr = geo.panel_frame(*ang)
        r = geo.unit_position(x1, x2, fr)
        X, Y = np.tan(x1), np.tan(x2)
        f = 2 * geo.OMEGA / np.sqrt(1 + X * X + Y * Y) * geo.coriolis_bracket(X, Y, ang[1], ang[2])
        np.testing.assert_allclose(f, 2 * geo.OMEGA * r[2], atol=1e-18)


@pytest.mark.parametrize("rot", ROTATIONS)
def test_panel_frames_are_cube_faces(rot):
    """The frames of Eq. (81)-(95) (atan2 branches) are the six faces of a cube:
    relative to panel 0's (c, e1, e2): p1 = (e1, -c, e2), p2 = (-c, -e1, e2),
    p3 = (-e1, c, e2), p4 = (e2, e1, -c), p5 = (-e2, e1, c)."""
    frames = [geo.panel_frame(*a) for a in geo.panel_angles(*rot)]
    c, e1, e2 = frames[0]
    expect = [(c, e1, e2), (e1, -c, e2), (-c, -e1, e2), (-e1, c, e2), (e2, e1, -c), (-e2, e1, c)]
    for got, exp in zip(frames, expect):
        for g, e in zip(got, exp):
            np.testing.assert_allclose(g, e, atol=1e-14)


@pytest.mark.parametrize("rot", ROTATIONS[1:])
def test_eq59_60_inverts_frames(rot):
    """Eq. (59)-(60) applied to the longitude/latitude of r(X, Y) give back X, Y."""
    x1, x2 = _pts()
    for ang in geo.panel_angles(*rot):
        r = geo.unit_position(x1, x2, geo.panel_frame(*ang))
        lam, phi = np.arctan2(r[1], r[0]), np.arcsin(r[2])
        X, Y = geo.xy_from_lonlat(lam, phi, *ang)
        np.testing.assert_allclose(X, np.tan(x1), atol=1e-11)
        np.testing.assert_allclose(Y, np.tan(x2), atol=1e-11)


@pytest.mark.parametrize("rot", ROTATIONS)
def test_interfaces_coincide(rot):
    frames = [geo.panel_frame(*a) for a in geo.panel_angles(*rot)]
    t = np.linspace(-np.pi / 4, np.pi / 4, 17)
    for pa, ea, pb, eb, rev in geo.INTERFACES:
        ra = geo.unit_position(*geo.edge_coords(ea, t), frames[pa])
        rb = geo.unit_position(*geo.edge_coords(eb, t[::-1] if rev else t), frames[pb])
        np.testing.assert_allclose(ra, rb, atol=1e-15)


def _appc(pa, pb, s):
    """The printed App. C contravariant relations A_(p) = T A_(q), Eq. (100)-(135),
    read from tests/golden/app_c_relations.txt for the interface {pa, pb};
    s = 2Z/(1+Z^2) with Z the tan-coordinate named by the paper.  Returns (p, q, T)."""
    for row in golden_app_c():
        if {row["p"], row["q"]} == {pa, pb}:
            return row["p"], row["q"], entries(row["M"], s)
    raise KeyError((pa, pb))


@pytest.mark.parametrize("rot", ROTATIONS[:2])
def test_app_c_relations(rot):
    """The oracle's geometric interface Jacobians equal the printed Eq. (100)-(135)."""
    frames = [geo.panel_frame(*a) for a in geo.panel_angles(*rot)]
    t = np.linspace(-np.pi / 4, np.pi / 4, 13)
    edge_of = {}
    for pa, ea, pb, eb, rev in geo.INTERFACES:
        edge_of[(pa, pb)] = (ea, eb, rev)
        edge_of[(pb, pa)] = (eb, ea, rev)
    for pa, ea, pb, eb, rev in geo.INTERFACES:
        p, q, _ = _appc(pa, pb, np.zeros(1))
        eq_, ep_, rev_ = edge_of[(q, p)]
        x1q, x2q = geo.edge_coords(eq_, t)
        Z = np.tan(t)                     # along-edge tan coordinate of panel q
        _, _, T = _appc(pa, pb, 2 * Z / (1 + Z * Z))
        J = geo.contravariant_jacobian(x1q, x2q, frames[q], frames[p])
        np.testing.assert_allclose(J, T, atol=1e-12)
