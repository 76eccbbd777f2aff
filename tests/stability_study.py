"""Stability of the oracle's multistep EPI on a synthetic workload's fields:
max |zeta| (relative vorticity, Eq. 43) and the mass and energy drifts (Eq. 44)
after every step, FP64 throughout.  A growing localized vorticity mode with
mass still conserved to round-off is the order-6 instability of the unfiltered
scheme (the paper uses no filter, Sec. 5).

Not a test (it takes minutes): run as
    python -m tests.stability_study WORKLOAD N_E P ORDER DT STEPS
e.g. `python -m tests.stability_study ne90_p6 30 6 6 1200 16` (the 6x90x90
workload's fields, EPI6, 1200 s steps, on a 6x30x30, p = 6 grid).  Uses the
oracle only."""
import sys
import time

import numpy as np


def main():
    from oracle import diagnostics as od
    from oracle import epi as oepi
    from oracle import fields
    from oracle import shallow_water as sw
    from paper_2101_05617_gb300 import synth
    name, ne, p, order, dt, steps = sys.argv[1], int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), \
        float(sys.argv[5]), int(sys.argv[6])
    wl = synth.WORKLOADS[name]
    f = synth.make_fields(wl, 0)
    g = sw.Grid(ne, p + 1, f.rotation)
    h, hB, V = f.evaluate(g.node_xyz())
    g.set_bottom(hB)
    q = fields.state_from_fields(g, h, hB, V)
    it = oepi.EPI(lambda x: sw.rhs_real(g, x.reshape(q.shape)).reshape(-1),
                  lambda x, v: sw.jvp(g, x.reshape(q.shape), v.reshape(q.shape)).reshape(-1), order, tol=wl.tol)
    y = q.reshape(-1).copy()
    inv0 = od.invariants(g, q)
    t0 = time.time()
    for k in range(steps):
        y = it.step(y, dt)
        qq = y.reshape(q.shape)
        inv = od.invariants(g, qq)
        print(f"step {k + 1:3d}  max|zeta| {np.max(np.abs(od.relative_vorticity(g, qq))):.3e}  "
              f"mass drift {(inv[0] - inv0[0]) / inv0[0]:+.1e}  energy drift {(inv[1] - inv0[1]) / inv0[1]:+.2e}  "
              f"Krylov {sum(s['krylov_iters'] for s in it.stats)}  ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main()
