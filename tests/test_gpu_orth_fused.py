"""Both vector passes of the fused incomplete orthogonalisation in one
cooperative launch (sw_set_orth_fused): the same arithmetic in the same order
as the two launches, so phi-function calls and EPI trajectories agree bit for
bit with the two-launch path, in both forms and both windows; and the fused
path itself against the oracle (Eq. 29 with the KIOPS reading)."""
import numpy as np
import pytest

from oracle import kiops as okiops
from oracle import shallow_water as osw
from tests.gpu_common import oracle_case, rel_l2_per_var, scaled_direction

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("workload,mode,iop,steps", [("small_ne4_p3", 1, 2, 6), ("ne30_p5", 1, 2, 3),
                                                     ("ne30_p5", 1, 3, 3), ("ne30_p5", 2, 3, 3)])
def test_fused_passes_equal_two_launches(workload, mode, iop, steps):
    from paper_2101_05617_gb300 import synth
    from paper_2101_05617_gb300.swepi import SWContext
    wl = synth.WORKLOADS[workload]
    f = synth.make_fields(wl, 7)
    out = []
    for fused in (0, 1):
        ctx = SWContext(wl.ne, wl.p, f.rotation)
        ctx.set_jvp_mode(mode)
        active = ctx.set_orth_fused(fused)
        assert active == fused, (fused, active)
        q = torch.tensor(ctx.state_from_fields(*f.evaluate(ctx.node_xyz())), device="cuda")
        stats = [ctx.epi_step(wl.order, wl.dt, q, tol=wl.tol, iop=iop) for _ in range(steps)]
        out.append((q.clone(), stats))
        ctx.close()
    (q0, s0), (q1, s1) = out
    assert s0 == s1, (s0, s1)
    assert torch.equal(q0, q1), float((q0 - q1).abs().max())


@pytest.mark.parametrize("iop", [2, 3])
def test_fused_passes_kiops_parity(iop):
    """A phi-function call of four vectors on 6 x 3 x 3 elements (p = 3) with the
    fused passes against the oracle: the same Krylov, substep and rejection
    counts, the product to 1e-10."""
    from paper_2101_05617_gb300.swepi import SWContext
    _, g, q, _ = oracle_case(3, 4, seed=11)
    dt, tol = 1800.0, 1e-10
    F = osw.rhs_real(g, q)
    bs = [None, dt * F] + [1e-3 * dt * scaled_direction(q, 70 + k) for k in range(2)]
    ctx = SWContext(g.ne, g.ns - 1, g.rotation)
    ctx.set_jvp_mode(1)
    assert ctx.set_orth_fused(1) == 1
    qd = torch.tensor(q.reshape(-1), device="cuda")
    bd = [None if b is None else torch.tensor(b.reshape(-1), device="cuda") for b in bs]
    w, st = ctx.kiops_phi(qd, dt, bd, tol=tol, iop=iop)
    ref, rst = okiops.kiops(1.0, lambda x: dt * osw.jvp(g, q, x.reshape(q.shape)).reshape(-1),
                            [np.zeros(q.size)] + [b.reshape(-1) for b in bs[1:]], tol=tol, iop=iop)
    err = rel_l2_per_var(w.cpu().numpy(), ref)
    assert max(err) < 1e-10, (err, st, rst)
    assert (st["krylov_iters"], st["substeps"], st["rejects"]) == \
        (rst["krylov_iters"], rst["substeps"], rst["rejects"]), (st, rst)
