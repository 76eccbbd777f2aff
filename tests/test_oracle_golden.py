"""The oracle against values the paper prints (fixtures under tests/golden/)."""
import numpy as np
import pytest

from oracle import epi
from tests.golden_tables import entries, golden_app_c, golden_epi_coefficients


def test_epi_coefficients_as_printed():
    """The oracle's EPI coefficient matrices equal Eq. (30) and (36)-(38) exactly."""
    gold = golden_epi_coefficients()
    assert sorted(gold) == [3, 4, 5, 6]
    for order, A in gold.items():
        assert epi.COEFFS[order] == A, order


def test_app_c_table_is_complete_and_consistent():
    """Every interface of the cube appears once, and the printed covariant
    relations are the inverse transpose of the printed contravariant ones (the
    tensor transformation law): a transcription check of the fixture."""
    rows = golden_app_c()
    pairs = {frozenset((r["p"], r["q"])) for r in rows}
    assert len(rows) == 12 and len(pairs) == 12
    s = np.linspace(-1.0, 1.0, 9)
    for r in rows:
        M = np.moveaxis(entries(r["M"], s), -1, 0)
        C = np.moveaxis(entries(r["C"], s), -1, 0)
        np.testing.assert_allclose(C, np.transpose(np.linalg.inv(M), (0, 2, 1)), atol=1e-15)
        np.testing.assert_allclose(np.linalg.det(M), 1.0, atol=1e-15)
