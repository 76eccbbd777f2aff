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
