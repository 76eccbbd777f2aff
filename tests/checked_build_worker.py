"""A fixed set of library calls on small grids, run in a process of its own
by test_gpu_checked_build.py: once with the default library and once with the
bounds-checked one (SWEPI_CHECKED=1).  It saves every result and the check
status after each group of calls, and with --inject also the status after a
planted out-of-range interface line (the checks must catch it)."""
import sys

import numpy as np
import torch

from tests.gpu_common import oracle_case, scaled_direction


def main(out_path, inject):
    from paper_2101_05617_gb300 import ensemble, swepi, synth
    res, codes = {}, []

    def status():
        code, checked = swepi.sw_check_status()
        codes.append(code)
        return checked

    _, g, q, _ = oracle_case(4, 4, seed=0)
    ctx = swepi.SWContext(4, 3, g.rotation)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    vd = torch.tensor(scaled_direction(q, 5).reshape(-1), device="cuda")
    res["rhs"] = ctx.rhs(qd).cpu().numpy()                   # face_flux_kernel<double>
    res["jvp"] = ctx.jvp(qd, vd).cpu().numpy()               # face_flux_kernel<cs>
    ctx.linearize(qd)                                          # lin_face_kernel
    res["jvp_split"] = ctx.jvp_linearized(vd).cpu().numpy()   # face_tangent_kernel<double>
    ctx.set_jvp_mode(2)
    ctx.linearize(qd)
    res["jvp_c64"] = ctx.jvp_linearized(vd).cpu().numpy()    # FP32 face and staged tile kernels
    status()
    for mode in (1, 2):                                        # EPI steps (start-up and multistep)
        c = swepi.SWContext(4, 3, g.rotation)
        c.set_jvp_mode(mode)
        y = qd.clone()
        for _ in range(3):
            c.epi_step(4, 900.0, y, tol=1e-12)
        res[f"epi_mode{mode}"] = y.cpu().numpy()
        c.close()
    status()
    rng = np.random.Generator(np.random.PCG64(7))
    members = [synth.EnsembleMember(i, ne, p, order, 900.0, int(rng.integers(1 << 31)))
               for i, (ne, p, order) in enumerate([(2, 3, 4), (3, 4, 5), (2, 5, 4)])]
    ctxs, qs = ensemble.build(members, workers=1)
    ens = swepi.SWEnsemble(ctxs)                               # ens_iter_kernel (task decode checks)
    ys = [x.clone() for x in qs]
    ens.epi_run(3, [m.order for m in members], [m.dt for m in members], ys, tol=1e-10)
    ens.close()
    for i, y in enumerate(ys):
        res[f"ens{i}"] = y.cpu().numpy()
    checked = status()
    if inject:
        swepi.sw_check_inject(ctx.handle, 1)
        ctx.rhs(qd)
        torch.cuda.synchronize()
        status()                                               # the planted line: code 1
        swepi.sw_check_inject(ctx.handle, 0)
        res["rhs_after"] = ctx.rhs(qd).cpu().numpy()
        status()
    np.savez(out_path, checked=np.array(checked), codes=np.array(codes), **res)


if __name__ == "__main__":
    main(sys.argv[1], "--inject" in sys.argv[2:])
