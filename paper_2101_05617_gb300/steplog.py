"""Per-step record of an EPI integration as JSON lines.

`integrate` advances a state with `sw_epi_step` and writes one JSON object
per step: the step index and simulated time, the phi-function solver's
statistics for that step (substeps, rejected attempts, Krylov iterations,
final Krylov size, last substep fraction and error estimate), the host wall
time of the step (the call returns after its stream has drained), and, every
`diagnostics_every` steps, the invariants of Sec. 5 (mass and total energy,
Eq. 44; potential enstrophy; max |zeta|, Eq. 43) from `sw_diagnostics` with
their drifts relative to the initial state.  The same records feed the
training data of the learned Krylov controller and a run's post-mortem."""
import json
import time

FIELDS = ("substeps", "rejects", "krylov_iters", "m_final", "tau_final", "err_last")


class StepLog:
    """JSON-lines sink: a path (opened for append) or an object with write()."""

    def __init__(self, target):
        self._own = isinstance(target, str)
        self._f = open(target, "a") if self._own else target

    def write(self, record):
        self._f.write(json.dumps(record, sort_keys=True) + "\n")
        if hasattr(self._f, "flush"):
            self._f.flush()

    def close(self):
        if self._own:
            self._f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _invariants(d):
    return {"mass": float(d[0]), "energy": float(d[1]), "enstrophy": float(d[2]), "max_abs_zeta": float(d[3])}


def integrate(ctx, order, dt, q, steps, log=None, diagnostics_every=1, t0=0.0, **opts):
    """Advance q (device state of ctx's grid) by `steps` EPI steps of order
    `order` and size dt; returns the list of records (also written to `log`,
    a StepLog, a path or None).  diagnostics_every = 0 skips the invariants."""
    if steps < 0 or diagnostics_every < 0:
        raise ValueError("steps and diagnostics_every must be >= 0")
    sink = StepLog(log) if isinstance(log, str) else log
    records = []
    ref = _invariants(ctx.diagnostics(q)) if diagnostics_every else None
    try:
        for k in range(1, steps + 1):
            w0 = time.perf_counter()
            st = ctx.epi_step(order, dt, q, **opts)
            rec = {"step": k, "time_s": t0 + k * dt, "order": order, "dt": dt,
                   "wall_ms": (time.perf_counter() - w0) * 1e3}
            rec.update({f: st[f] for f in FIELDS})
            if diagnostics_every and k % diagnostics_every == 0:
                inv = _invariants(ctx.diagnostics(q))
                rec.update(inv)
                for key in ("mass", "energy", "enstrophy"):
                    rec[key + "_drift"] = (inv[key] - ref[key]) / ref[key] if ref[key] != 0 else None
            records.append(rec)
            if sink is not None:
                sink.write(rec)
    finally:
        if isinstance(log, str):
            sink.close()
    return records
