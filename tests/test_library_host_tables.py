"""The library's host-built tables, checked without a GPU: the EPI coefficient
matrices sw_epi_step uses equal the values printed in Eq. 30 and 36-38
exactly, and the DFR operators sw_init builds (Gauss-Legendre points and
weights, the Eq. 13 derivative matrix on the extended nodes, the Eq. 8 trace
rows; the library's own Newton iteration and barycentric formulas) equal the
oracle's (numpy's leggauss and the product formulas) to rounding."""
import numpy as np
import pytest

from oracle import dfr as odfr
from tests.golden_tables import golden_epi_coefficients


def test_library_epi_coefficients_equal_printed_values():
    from paper_2101_05617_gb300 import swepi
    golden = golden_epi_coefficients()
    for order in (3, 4, 5, 6):
        A = swepi.sw_epi_coefficients(order)
        ref = np.array([[float(v) for v in row] for row in golden[order]])
        assert A.shape == ref.shape and np.array_equal(A, ref), (order, A, ref)
    for bad in (2, 7):
        with pytest.raises(swepi.SWError):
            swepi.sw_epi_coefficients(bad)


@pytest.mark.parametrize("p", range(8))
def test_library_dfr_operators_equal_oracle(p):
    from paper_2101_05617_gb300 import swepi
    ns = p + 1
    xi, w, D, lm, lp = swepi.sw_dfr_operators(p)
    oxi, ow = odfr.gauss_legendre(ns)
    np.testing.assert_allclose(xi, oxi, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, ow, rtol=0, atol=1e-15)
    oD = odfr.flux_derivative_matrix(ns)
    np.testing.assert_allclose(D, oD, rtol=0, atol=1e-13 * np.max(np.abs(oD)))
    olm, olp = odfr.trace_rows(ns)
    np.testing.assert_allclose(lm, olm, rtol=0, atol=1e-13)
    np.testing.assert_allclose(lp, olp, rtol=0, atol=1e-13)


def test_library_dfr_operators_reject_bad_degree():
    from paper_2101_05617_gb300 import swepi
    for bad in (-1, 8):
        with pytest.raises(swepi.SWError):
            swepi.sw_dfr_operators(bad)


ROTATIONS = [(0.3, 0.5, -1.0), (-2.1, 0.9, 0.4), (0.0, np.pi / 4, 0.0), (0.7, 0.0, 0.0)]


@pytest.mark.parametrize("rot", ROTATIONS)
def test_library_node_coefficients_equal_oracle_metric(rot):
    """The metric, Coriolis and Christoffel coefficients the library tabulates
    (its panel frames from cube symmetry) equal the oracle's Eq. 67-80 (its
    frames from the printed angles of Eq. 81-95) at random points of every panel."""
    from oracle import geometry as geo
    from paper_2101_05617_gb300 import swepi
    rng = np.random.default_rng(21)
    X, Y = rng.uniform(-1.0, 1.0, 200), rng.uniform(-1.0, 1.0, 200)
    gr, om = 9.80616, 7.292e-5
    angles = geo.panel_angles(*rot)
    for p in range(6):
        out = swepi.sw_node_coefficients(rot, p, X, Y, gravity=gr, omega=om)
        m = geo.metric(X, Y)
        Gt = geo.christoffel_time(X, Y, angles[p][1], angles[p][2], om)
        Gs = geo.christoffel_space(X, Y)
        ref = [0.5 * gr * m["h11"] / m["sqrtg"], 0.5 * gr * m["h12"] / m["sqrtg"], 0.5 * gr * m["h22"] / m["sqrtg"],
               -2 * Gt[0][0], -2 * Gt[0][1], -2 * Gt[1][0], -2 * Gt[1][1],
               Gs[0][0][0], 2 * Gs[0][0][1], 2 * Gs[1][0][1], Gs[1][1][1], 0 * X, 0 * X]
        for k, r in enumerate(ref):
            scale = max(np.max(np.abs(r)), 1e-300)
            assert np.max(np.abs(out[k] - r)) <= 1e-13 * scale, (p, k)


def test_library_interface_transforms_equal_oracle_jacobians():
    """The twelve interfaces the library connects are the oracle's (panels, edges,
    orientation), and its App. C transforms equal the oracle's Jacobians of the
    coordinate change, built from the panel frames, along every edge."""
    from oracle import geometry as geo
    from oracle import shallow_water as sw
    from paper_2101_05617_gb300 import swepi
    edge = "WESN"
    g = sw.Grid(2, 3, (0.3, 0.5, -1.0))
    t = np.linspace(-np.pi / 4, np.pi / 4, 9)[1:-1]
    libs = []
    for k in range(12):
        (pa, ea, pb, eb, rev), _ = swepi.sw_interface_transform(k, 0.0)
        libs.append((pa, edge[ea], pb, edge[eb], bool(rev)))
        x1b, x2b = geo.edge_coords(edge[eb], -t if rev else t)
        J = geo.contravariant_jacobian(x1b, x2b, g.frames[pb], g.frames[pa], g.a)   # d x_(a) / d x_(b)
        for i, ti in enumerate(t):
            _, T = swepi.sw_interface_transform(k, ti)
            np.testing.assert_allclose(T, J[:, :, i], rtol=0, atol=1e-12)
    assert sorted(libs) == sorted(geo.INTERFACES)
