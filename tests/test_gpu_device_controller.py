"""The phi-function solver with its adaptive controller on the device
(sw_set_kiops_driver 1): one CUDA graph per call whose conditional loops
(substep attempts, Krylov iterations, squarings of the small exponential) are
steered by device kernels running the same controller as the host driver.
Against the oracle (Eq. 29 and the KIOPS reading: identical Krylov, substep
and rejection counts) and against the host driver on EPI trajectories."""
import numpy as np
import pytest

from oracle import epi as oepi
from oracle import kiops as okiops
from oracle import shallow_water as osw
from tests.gpu_common import oracle_case, rel_l2_per_var, scaled_direction

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(g, mode=1, driver=1):
    from paper_2101_05617_gb300.swepi import SWContext
    c = SWContext(g.ne, g.ns - 1, g.rotation)
    c.set_jvp_mode(mode)
    c.set_kiops_driver(driver)
    return c


@pytest.mark.parametrize("iop", [2, 3])
@pytest.mark.parametrize("ne,ns,nb,dt,tol", [(2, 4, 2, 900.0, 1e-12), (3, 4, 4, 1800.0, 1e-10),
                                             (4, 4, 5, 900.0, 1e-12)])
def test_device_controller_kiops_parity(ne, ns, nb, dt, tol, iop):
    _, g, q, _ = oracle_case(ne, ns, seed=ne)
    F = osw.rhs_real(g, q)
    bs = [None, dt * F] + [1e-3 * dt * scaled_direction(q, 50 + k) for k in range(nb - 2)]
    ctx = _ctx(g)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    bd = [None if b is None else torch.tensor(b.reshape(-1), device="cuda") for b in bs]
    w, st = ctx.kiops_phi(qd, dt, bd, tol=tol, iop=iop)
    ref, rst = okiops.kiops(1.0, lambda x: dt * osw.jvp(g, q, x.reshape(q.shape)).reshape(-1),
                            [np.zeros(q.size)] + [b.reshape(-1) for b in bs[1:]], tol=tol, iop=iop)
    err = rel_l2_per_var(w.cpu().numpy(), ref)
    print(f"PARITY device controller kiops ne{ne} ns{ns} nb{nb} iop{iop}: {err} {st} oracle {rst}")
    assert max(err) < 1e-10, (err, st, rst)
    assert (st["krylov_iters"], st["substeps"], st["rejects"]) == \
        (rst["krylov_iters"], rst["substeps"], rst["rejects"]), (st, rst)


def test_device_controller_epi_parity():
    """The small configuration (6 x 4 x 4, p = 3, EPI4, tol 1e-12, dt = 900 s, 10
    steps, start-up included) with the device controller against the oracle."""
    _, g, q, _ = oracle_case(4, 4, seed=0)
    dt, tol = 900.0, 1e-12
    ctx = _ctx(g)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    it = oepi.EPI(lambda x: osw.rhs_real(g, x.reshape(q.shape)).reshape(-1),
                  lambda x, v: osw.jvp(g, x.reshape(q.shape), v.reshape(q.shape)).reshape(-1), 4, tol=tol)
    y = q.reshape(-1).copy()
    for _ in range(10):
        ctx.epi_step(4, dt, qd, tol=tol)
        y = it.step(y, dt)
    err = rel_l2_per_var(qd.cpu().numpy(), y)
    assert max(err) < 1e-11, err


@pytest.mark.parametrize("workload,mode,iop,steps", [("small_ne4_p3", 1, 2, 8), ("small_ne4_p3", 2, 3, 8),
                                                     ("ne30_p5", 1, 2, 4), ("ne30_p5", 2, 3, 4)])
def test_device_controller_equals_host_controller(workload, mode, iop, steps):
    """The same EPI trajectory (start-up and multistep steps) with the controller
    on the device and on the host: identical KIOPS statistics every step and the
    same state to rounding (both run the same kernels; the device computes the
    controller's logarithms and powers with its own math library)."""
    from paper_2101_05617_gb300 import synth
    from paper_2101_05617_gb300.swepi import SWContext
    wl = synth.WORKLOADS[workload]
    f = synth.make_fields(wl, 3)
    out = []
    for driver in (0, 1):
        ctx = SWContext(wl.ne, wl.p, f.rotation)
        ctx.set_jvp_mode(mode)
        ctx.set_kiops_driver(driver)
        q = torch.tensor(ctx.state_from_fields(*f.evaluate(ctx.node_xyz())), device="cuda")
        stats = [ctx.epi_step(wl.order, wl.dt, q, tol=wl.tol, iop=iop) for _ in range(steps)]
        out.append((q.view(3, -1).clone(), stats))
        ctx.close()
    (qh, sh), (qd, sd) = out
    assert sh == sd, (sh, sd)
    err = [float(torch.linalg.norm(qd[k] - qh[k]) / torch.linalg.norm(qh[k])) for k in range(3)]
    print(f"device vs host controller {workload} mode {mode} iop {iop}: {err}")
    assert max(err) < 1e-13, err


def test_device_controller_nonfinite_state():
    """A NaN in the state ends the call with SW_ENONFINITE from the device-side
    checks, and the context keeps working."""
    from paper_2101_05617_gb300 import swepi
    _, g, q, _ = oracle_case(3, 4, seed=1)
    ctx = _ctx(g)
    bad = q.reshape(-1).copy()
    bad[q.size // 3 + 17] = np.nan
    with pytest.raises(swepi.SWError) as ei:
        ctx.epi_step(4, 900.0, torch.tensor(bad, device="cuda"), tol=1e-12)
    assert ei.value.status == -6, ei.value
    ctx.epi_reset()
    qd = torch.tensor(q.reshape(-1), device="cuda")
    for _ in range(3):
        ctx.epi_step(4, 900.0, qd, tol=1e-12)
    assert torch.isfinite(qd).all()
