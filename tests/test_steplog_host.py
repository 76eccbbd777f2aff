"""The per-step JSON-lines record of an EPI integration (steplog.integrate),
driven by a stand-in context on the CPU: one record per step with the solver's
statistics, the simulated time and, on the chosen steps, the invariants with
their drifts from the initial state."""
import io
import json

import pytest

from paper_2101_05617_gb300 import steplog


class FakeCtx:
    """Stand-in for SWContext: each step adds 1 to q[0], the 'mass' follows it."""

    def __init__(self):
        self.calls = 0

    def epi_step(self, order, dt, q, **opts):
        self.calls += 1
        q[0] += 1.0
        return {"substeps": 2, "rejects": self.calls % 2, "krylov_iters": 10 * self.calls, "m_final": 12,
                "tau_final": 0.5, "err_last": 1e-3, "extra": "ignored"}

    def diagnostics(self, q):
        return [100.0 + q[0], 50.0, 0.0, 7.0]


def test_records_and_lines():
    q = [0.0]
    buf = io.StringIO()
    recs = steplog.integrate(FakeCtx(), 5, 1800.0, q, 3, log=steplog.StepLog(buf), t0=3600.0, tol=1e-10)
    assert [r["step"] for r in recs] == [1, 2, 3]
    assert [r["time_s"] for r in recs] == [5400.0, 7200.0, 9000.0]
    assert [r["krylov_iters"] for r in recs] == [10, 20, 30] and [r["rejects"] for r in recs] == [1, 0, 1]
    assert "extra" not in recs[0] and recs[0]["order"] == 5
    assert recs[2]["mass"] == 103.0 and recs[2]["mass_drift"] == pytest.approx(0.03)
    assert recs[2]["energy_drift"] == 0.0 and recs[2]["enstrophy_drift"] is None   # zero reference
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert lines == recs


def test_diagnostics_every_and_path(tmp_path):
    q = [0.0]
    path = str(tmp_path / "run.jsonl")
    recs = steplog.integrate(FakeCtx(), 4, 900.0, q, 4, log=path, diagnostics_every=2)
    assert ["mass" in r for r in recs] == [False, True, False, True]
    assert len(open(path).read().splitlines()) == 4
    recs = steplog.integrate(FakeCtx(), 4, 900.0, [0.0], 2, diagnostics_every=0)
    assert all("mass" not in r for r in recs)
    with pytest.raises(ValueError):
        steplog.integrate(FakeCtx(), 4, 900.0, [0.0], -1)
