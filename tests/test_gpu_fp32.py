"""The complex64-bulk form (sw_set_jvp_mode 2): the per-Krylov-vector
imaginary half of the complex-step JVP in FP32, the Krylov basis,
orthogonalisation, exponential and error estimate in FP64.  Each result states
its error against the FP64 path/oracle and the EPI time-discretisation error."""
import numpy as np
import pytest

from oracle import shallow_water as osw
from tests.gpu_common import oracle_case, scaled_direction, scaled_err_per_var, term_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 arithmetic of the same formulas: ~500 FP32 roundings of the term scale
# (u32 = 6e-8), the analogue of the FP64 bound of the parity tests
TOL_JVP32 = 3e-5


def _ctx(g, mode):
    from paper_2101_05617_gb300.swepi import SWContext
    c = SWContext(g.ne, g.ns - 1, g.rotation)
    c.set_jvp_mode(mode)
    return c


@pytest.mark.parametrize("ne,ns,seed,bottom", [(4, 4, 0, 0.0), (3, 6, 1, 0.0), (5, 3, 3, 1500.0), (6, 7, 5, 800.0)])
def test_fp32_jvp_parity(ne, ns, seed, bottom):
    _, g, q, hB = oracle_case(ne, ns, seed=seed, bottom_amp=bottom)
    ctx = _ctx(g, 2)
    ctx.set_bottom(hB.reshape(-1))
    qd = torch.tensor(q.reshape(-1), device="cuda")
    ctx.linearize(qd)
    v = scaled_direction(q, seed + 300)
    Jv = ctx.jvp_linearized(torch.tensor(v.reshape(-1), device="cuda")).cpu().numpy()
    err = scaled_err_per_var(Jv, osw.jvp(g, q, v), term_scale(g, q, v))
    assert max(err) < TOL_JVP32, err
    assert max(err) > 1e-12, "FP32 form should not be bit-identical to FP64"


def _trajectory(wl, mode, dt, steps, seed=0, iop=2):
    from paper_2101_05617_gb300 import synth
    from paper_2101_05617_gb300.swepi import SWContext
    f = synth.make_fields(wl, seed)
    ctx = SWContext(wl.ne, wl.p, f.rotation)
    h, hB, V = f.evaluate(ctx.node_xyz())
    q = torch.tensor(ctx.state_from_fields(h, hB, V), device="cuda")
    ctx.set_jvp_mode(mode)
    for _ in range(steps):
        ctx.epi_step(wl.order, dt, q, tol=wl.tol, iop=iop)
    torch.cuda.synchronize()
    out = q.view(3, -1).clone()
    ctx.close()
    return out


def _rel(a, b):
    return [float(torch.linalg.norm(a[k] - b[k]) / torch.linalg.norm(b[k])) for k in range(3)]


@pytest.mark.parametrize("workload,steps", [("small_ne4_p3", 10), ("ne30_p5", 12)])
def test_fp32_error_below_time_discretisation_error(workload, steps):
    """FP32-bulk trajectory vs the FP64 path (itself pinned to the oracle by the
    parity tests) is smaller than the EPI time-discretisation error, measured as
    the FP64 trajectory at dt against the one at dt/4."""
    from paper_2101_05617_gb300 import synth
    wl = synth.WORKLOADS[workload]
    q64 = _trajectory(wl, 1, wl.dt, steps)
    q32 = _trajectory(wl, 2, wl.dt, steps)
    qfine = _trajectory(wl, 1, wl.dt / 4, 4 * steps)
    e32 = _rel(q32, q64)
    etime = _rel(q64, qfine)
    assert all(a < b for a, b in zip(e32, etime)), (e32, etime)


def test_fp32_window3_ne60_below_time_discretisation_error():
    """On the 6 x 60 x 60, p = 5 grid the complex64-bulk form runs with the
    orthogonalisation window of three: after 16 EPI5 steps its state differs from
    the FP64 path (default window two) by less than a tenth of the EPI
    time-discretisation error (FP64 at dt against dt/4) and stays finite."""
    from paper_2101_05617_gb300 import synth
    wl = synth.WORKLOADS["ne60_p5"]
    q64 = _trajectory(wl, 1, wl.dt, 16)
    q32 = _trajectory(wl, 2, wl.dt, 16, iop=3)
    qfine = _trajectory(wl, 1, wl.dt / 4, 64)
    assert torch.isfinite(q32).all()
    e32 = _rel(q32, q64)
    etime = _rel(q64, qfine)
    assert all(a < 0.1 * b for a, b in zip(e32, etime)), (e32, etime)


def test_precision_one_at_init_equals_mode_two():
    """sw_params.precision = 1 selects the complex64-bulk form at sw_init: its
    EPI trajectory (start-up and multistep steps) and statistics equal those of
    a precision-0 context switched by sw_set_jvp_mode(2), bit for bit."""
    from paper_2101_05617_gb300 import synth
    from paper_2101_05617_gb300.swepi import SWContext
    wl = synth.WORKLOADS["small_ne4_p3"]
    f = synth.make_fields("small_ne4_p3", 4)
    a = SWContext(wl.ne, wl.p, f.rotation, precision=1)
    b = SWContext(wl.ne, wl.p, f.rotation)
    b.set_jvp_mode(2)
    h, hB, V = f.evaluate(a.node_xyz())
    q0 = a.state_from_fields(h, hB, V)
    b.state_from_fields(h, hB, V)
    qa = torch.tensor(q0, device="cuda")
    qb = qa.clone()
    for _ in range(6):
        sa = a.epi_step(5, wl.dt, qa, tol=wl.tol)
        sb = b.epi_step(5, wl.dt, qb, tol=wl.tol)
        assert sa == sb, (sa, sb)
    assert torch.equal(qa, qb)
    c = SWContext(wl.ne, wl.p, f.rotation)          # precision 0 differs (the FP64 path)
    c.state_from_fields(h, hB, V)
    qc = torch.tensor(q0, device="cuda")
    for _ in range(6):
        c.epi_step(5, wl.dt, qc, tol=wl.tol)
    assert not torch.equal(qa, qc)


@pytest.mark.parametrize("ne,ns,seed", [(4, 6, 0), (4, 7, 2), (6, 3, 1)])
def test_fp32_staged_tile_kernel_equals_register_kernel(ne, ns, seed):
    """The complex64-bulk volume kernel stages each element tile in shared memory
    by bulk asynchronous copies when every address is 16-byte aligned, and
    otherwise runs the register-and-cache kernel; both perform the same FP32
    operations in the same order, so a direction vector given 8 bytes off
    alignment (the fallback) must give the same product bit for bit, and both
    match the oracle within the FP32 bound."""
    _, g, q, _ = oracle_case(ne, ns, seed=seed)
    ctx = _ctx(g, 2)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    ctx.linearize(qd)
    v = scaled_direction(q, seed + 500).reshape(-1)
    buf = torch.zeros(v.size + 2, dtype=torch.float64, device="cuda")
    aligned = torch.tensor(v, device="cuda")
    shifted = buf[1:v.size + 1]
    shifted.copy_(aligned)
    assert aligned.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 8
    a = ctx.jvp_linearized(aligned)
    b = ctx.jvp_linearized(shifted)
    assert torch.equal(a, b)
    err = scaled_err_per_var(a.cpu().numpy(), osw.jvp(g, q, v.reshape(q.shape)), term_scale(g, q, v.reshape(q.shape)))
    assert max(err) < TOL_JVP32, err
