"""Spatial convergence of the oracle's whole method on an exact steady solution
(the zonal flow of tests/test_oracle_steady.py on a rotated grid), set beside
the DFR orders the paper prints in Table 1 (Sec. 5.3): EPI6 with one-hour
steps and KIOPS tolerance 1e-10, the error norms of Eq. 39-41 of H after a
given time against the exact (initial) state, and the observed orders between
consecutive N_e for N_s = 3..6.

Not a test (it takes minutes): run as
    python -m tests.convergence_study [hours] [n_e list]
e.g. `python -m tests.convergence_study 24 10,20`, or for the p-refinement of
Fig. 3a (N_e = 10, N_s = 3..8)
    python -m tests.convergence_study [hours] p
One spawned process per (N_e, N_s); uses the oracle only."""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROTATION = (0.3, 0.5, -1.0)


def _run(args):
    ne, ns, order, dt, hours = args
    from oracle import diagnostics as od
    from oracle import epi as oepi
    from oracle import shallow_water as sw
    from tests.test_oracle_steady import _steady
    g, q = _steady(ne, ns, ROTATION)
    it = oepi.EPI(lambda x: sw.rhs_real(g, x.reshape(q.shape)).reshape(-1),
                  lambda x, v: sw.jvp(g, x.reshape(q.shape), v.reshape(q.shape)).reshape(-1), order, tol=1e-10)
    y = q.reshape(-1).copy()
    t0 = time.time()
    for _ in range(int(round(hours * 3600.0 / dt))):
        y = it.step(y, dt)
    H = y.reshape(q.shape)[0] / g.m['sqrtg']
    HT = q[0] / g.m['sqrtg']
    return ne, ns, [float(e) for e in od.error_norms(g, H, HT)], time.time() - t0


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def run_jobs(jobs):
    """Run the (N_e, N_s, order, dt, hours) jobs in spawned processes, one BLAS
    thread each (the children inherit the environment at spawn)."""
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    os.environ.update({k: "1" for k in _THREAD_VARS})
    try:
        with mp.get_context("spawn").Pool(min(len(jobs), mp.cpu_count())) as pool:
            return pool.map(_run, jobs, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def main():
    hours = float(sys.argv[1]) if len(sys.argv) > 1 else 24.0
    if len(sys.argv) > 2 and sys.argv[2] == "p":
        res = run_jobs([(10, ns, 6, 3600.0, hours) for ns in range(3, 9)])
        for ne, ns, e, sec in res:
            print(f"N_e={ne:3d} N_s={ns}  L1 {e[0]:.3e}  L2 {e[1]:.3e}  Linf {e[2]:.3e}  ({sec:.0f} s)")
        return
    nes = [int(x) for x in sys.argv[2].split(",")] if len(sys.argv) > 2 else [5, 10]
    jobs = [(ne, ns, 6, 3600.0, hours) for ns in (3, 4, 5, 6) for ne in nes]
    res = run_jobs(jobs)
    err = {(ne, ns): np.array(e) for ne, ns, e, _ in res}
    for ne, ns, e, sec in res:
        print(f"N_e={ne:3d} N_s={ns}  L1 {e[0]:.3e}  L2 {e[1]:.3e}  Linf {e[2]:.3e}  ({sec:.0f} s)")
    for ns in (3, 4, 5, 6):
        for a, b in zip(nes[:-1], nes[1:]):
            o = np.log(err[(a, ns)] / err[(b, ns)]) / np.log(b / a)
            print(f"N_s={ns}  N_e {a}->{b}  order L1 {o[0]:.2f}  L2 {o[1]:.2f}  Linf {o[2]:.2f}")


if __name__ == "__main__":
    main()
