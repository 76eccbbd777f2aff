"""Pins of the diagnostics (Sec. 5, Eq. 39-46)."""
import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import fields, geometry as geo, shallow_water as sw


def _solid_body(grid, w0, H0=8000.0):
    """Solid-body rotation about the z axis: V = w0 z x (a r)."""
    r = grid.node_xyz()
    V = w0 * grid.a * np.stack([-r[1], r[0], np.zeros_like(r[0])])
    shp = grid.x1.shape
    return fields.state_from_fields(grid, np.full(shp, H0), np.zeros(shp), V), r


def test_sphere_area_and_mass():
    """Eq. (42) of H = 1 is the sphere's area in angular units (the element
    Jacobian (dx/2)^2 left out): 4 pi a^2 / (dx/2)^2 / ... checked against the
    exact area of the cube panels, and mass = sum q^0 w w."""
    g = sw.Grid(4, 5, (0.2, 0.3, 0.4))
    area = dg.integral(g, np.ones(g.x1.shape)) * (g.dx / 2) ** 2
    assert abs(area - 4 * np.pi * g.a ** 2) < 1e-9 * 4 * np.pi * g.a ** 2
    q, _ = _solid_body(g, 0.0)
    assert abs(dg.invariants(g, q)[0] - sw.mass_integral(g, q)) < 1e-12 * sw.mass_integral(g, q)


@pytest.mark.parametrize("ne", [4, 8])
def test_vorticity_of_solid_body_rotation(ne):
    """Relative vorticity of V = w0 z x r is 2 w0 sin(latitude) (exact for the
    continuous field; converges spectrally in the degree)."""
    g = sw.Grid(ne, 6, (0.5, -0.4, 1.1))
    w0 = 1e-5
    q, r = _solid_body(g, w0)
    zeta = dg.relative_vorticity(g, q)
    assert np.max(np.abs(zeta - 2 * w0 * r[2])) < 1e-4 * 2 * w0


def test_coriolis_parameter_and_rest_energy():
    g = sw.Grid(3, 4, (0.1, 0.7, -0.3))
    r = g.node_xyz()
    np.testing.assert_allclose(dg.coriolis_parameter(g), 2 * geo.OMEGA * r[2], atol=1e-18)
    q, _ = _solid_body(g, 0.0, 8000.0)
    mass, energy, ens = dg.invariants(g, q)
    # at rest on a flat bottom: E = g_r H^2 / 2 * area, enstrophy = f^2/(2H) integrated
    assert abs(energy - 0.5 * g.gr * 8000.0 ** 2 * dg.integral(g, np.ones(g.x1.shape))) < 1e-12 * energy
    assert abs(ens - dg.integral(g, dg.coriolis_parameter(g) ** 2 / (2 * 8000.0))) < 1e-12 * ens


def test_error_norms():
    g = sw.Grid(2, 3)
    HT = np.full(g.x1.shape, 2.0)
    H = HT * 1.01
    l1, l2, linf = dg.error_norms(g, H, HT)
    assert abs(l1 - 0.01) < 1e-14 and abs(l2 - 0.01) < 1e-14 and abs(linf - 0.01) < 1e-14
