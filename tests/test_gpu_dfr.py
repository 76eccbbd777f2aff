"""GPU parity of the DFR right-hand side and the complex-step JVP (Eq. 28)
through the C ABI, element by element against the oracle."""
import numpy as np
import pytest

from oracle import shallow_water as osw
from tests.gpu_common import oracle_case, rel_err_per_var, scaled_direction, scaled_err_per_var, term_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP64 evaluations of the same formulas in a different operation order.  The
# error is measured against the magnitude of the summed flux-divergence terms
# (term_scale): a balanced flow makes the tendency a small residual of them, so
# a bound relative to the result itself would measure cancellation, not the
# kernel.  Each output sums 2 N_s + 4 terms, each the result of ~30 rounded
# operations (traces, the AUSM flux, the App. C transforms): ~500 u = 1e-13 of
# the term scale bounds any evaluation order.  The errors reached on the GB300
# over every case below are at most 8.3e-15 (RHS) and 3.5e-14 (JVP, the split
# and the full evaluation, at eps 1e-30 and 1.5e-8); the bounds sit a factor
# 2-4 above them.
TOL_RHS = 3e-14
TOL_JVP = 8e-14

CASES = [(4, 4, 0, 0.0), (3, 6, 1, 0.0), (2, 8, 2, 0.0), (5, 3, 3, 1500.0), (1, 2, 4, 0.0), (6, 7, 5, 800.0)]


def _ctx(g):
    from paper_2101_05617_gb300.swepi import SWContext
    return SWContext(g.ne, g.ns - 1, g.rotation)


def _report(name, err, tol):
    """Print the reached error beside its bound (visible with pytest -s), then check it."""
    print(f"PARITY {name}: max error / term scale per variable "
          f"{' '.join('%.2e' % e for e in err)} (bound {tol:.0e})")
    assert max(err) < tol, (name, err)


@pytest.mark.parametrize("ne,ns,seed,bottom", CASES)
def test_rhs_parity(ne, ns, seed, bottom):
    _, g, q, hB = oracle_case(ne, ns, seed=seed, bottom_amp=bottom)
    ctx = _ctx(g)
    ctx.set_bottom(hB.reshape(-1))
    qd = torch.tensor(q.reshape(-1), device="cuda")
    F = ctx.rhs(qd)
    torch.cuda.synchronize()
    ref = osw.rhs_real(g, q)
    err = scaled_err_per_var(F.cpu().numpy(), ref, term_scale(g, q))
    _report(f"rhs ne{ne} ns{ns} seed{seed} bottom{bottom:g}", err, TOL_RHS)


@pytest.mark.parametrize("ne,ns,seed,bottom", CASES)
def test_jvp_parity(ne, ns, seed, bottom):
    _, g, q, hB = oracle_case(ne, ns, seed=seed, bottom_amp=bottom)
    ctx = _ctx(g)
    ctx.set_bottom(hB.reshape(-1))
    v = scaled_direction(q, seed + 100)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    vd = torch.tensor(v.reshape(-1), device="cuda")
    Jv = ctx.jvp(qd, vd, 1e-30)
    torch.cuda.synchronize()
    ref = osw.jvp(g, q, v, 1e-30)
    err = scaled_err_per_var(Jv.cpu().numpy(), ref, term_scale(g, q, v))
    _report(f"jvp ne{ne} ns{ns} seed{seed} bottom{bottom:g}", err, TOL_JVP)


def test_geometry_and_state_conversion():
    """Node positions and the fields->state conversion of the library agree with
    the oracle's (independent implementations of App. B)."""
    f, g, q, hB = oracle_case(3, 5, seed=7)
    ctx = _ctx(g)
    xyz = ctx.node_xyz()
    np.testing.assert_allclose(xyz, g.node_xyz().reshape(3, -1), atol=2e-15)
    h, hB2, V = f.evaluate(g.node_xyz())
    qg = ctx.state_from_fields(h.reshape(-1), hB2.reshape(-1), V.reshape(3, -1))
    err = rel_err_per_var(qg, q)
    assert max(err) < 1e-13, err


@pytest.mark.parametrize("workload", ["small_ne4_p3", "ne30_p5"])
def test_mass_conservation_gpu(workload):
    """sum w_m w_n dq^0/dt = 0 to round-off (Sec. 5.4.2) on the GPU path: the
    interface mass fluxes cancel pairwise, so the budget is bounded by the
    rounding of the summed divergence terms (a wrong or one-sided interface
    flux would leave a residual ~1e-6 of that scale)."""
    _, g, q, _ = oracle_case(6, 5, workload=workload, seed=3)
    ctx = _ctx(g)
    F = ctx.rhs(torch.tensor(q.reshape(-1), device="cuda")).cpu().numpy().reshape(q.shape)
    w2 = g.w[:, None] * g.w[None, :]
    budget = abs(np.sum(F[0] * w2))
    assert budget < 1e-14 * np.sum(w2) * F[0].size / w2.size * term_scale(g, q)[0]


def test_jvp_linearity_and_determinism():
    _, g, q, _ = oracle_case(4, 6, seed=9)
    ctx = _ctx(g)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    v = torch.tensor(scaled_direction(q, 1).reshape(-1), device="cuda")
    w = torch.tensor(scaled_direction(q, 2).reshape(-1), device="cuda")
    a = ctx.jvp(qd, v)
    b = ctx.jvp(qd, w)
    c = ctx.jvp(qd, 2 * v + 3 * w)
    assert torch.linalg.norm(c - 2 * a - 3 * b) < 1e-14 * torch.linalg.norm(c)
    a2 = ctx.jvp(qd, v)
    assert torch.equal(a, a2)


def test_ragged_and_invalid_arguments():
    from paper_2101_05617_gb300 import swepi
    with pytest.raises(swepi.SWError):
        swepi.sw_init(0, 3)
    with pytest.raises(swepi.SWError):
        swepi.sw_init(4, 8)
    _, g, q, _ = oracle_case(2, 3, seed=1)
    ctx = _ctx(g)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    with pytest.raises(swepi.SWError):
        swepi.sw_jvp(ctx.handle, qd, qd, 0.0, torch.empty_like(qd))
    with pytest.raises(swepi.SWError):
        swepi.sw_rhs(ctx.handle, qd, qd)


@pytest.mark.parametrize("ne,ns,workload", [(60, 6, "ne60_p5"), (90, 7, "ne90_p6")])
def test_full_size_parity(ne, ns, workload):
    """The benchmark grids at full size (6 x 60 x 60, p = 5 and 6 x 90 x 90,
    p = 6 with topography): RHS and JVP compared element by element."""
    from paper_2101_05617_gb300 import synth
    wl = synth.WORKLOADS[workload]
    _, g, q, hB = oracle_case(ne, ns, workload=workload, seed=0,
                              bottom_amp=wl.bottom_amp)
    ctx = _ctx(g)
    ctx.set_bottom(hB.reshape(-1))
    qd = torch.tensor(q.reshape(-1), device="cuda")
    F = ctx.rhs(qd).cpu().numpy()
    err = scaled_err_per_var(F, osw.rhs_real(g, q), term_scale(g, q))
    _report(f"rhs full size ne{ne} ns{ns}", err, TOL_RHS)
    v = scaled_direction(q, 3)
    Jv = ctx.jvp(qd, torch.tensor(v.reshape(-1), device="cuda")).cpu().numpy()
    err = scaled_err_per_var(Jv, osw.jvp(g, q, v), term_scale(g, q, v))
    _report(f"jvp full size ne{ne} ns{ns}", err, TOL_JVP)


@pytest.mark.parametrize("ne,ns,seed,bottom", CASES)
def test_split_jvp_parity(ne, ns, seed, bottom):
    """sw_linearize + sw_jvp_linearized (real half once, imaginary half per v)
    against the oracle's complex-step JVP, and against the plain sw_jvp."""
    _, g, q, hB = oracle_case(ne, ns, seed=seed, bottom_amp=bottom)
    ctx = _ctx(g)
    ctx.set_bottom(hB.reshape(-1))
    qd = torch.tensor(q.reshape(-1), device="cuda")
    ctx.linearize(qd)
    for k in range(2):
        v = scaled_direction(q, seed + 200 + k)
        vd = torch.tensor(v.reshape(-1), device="cuda")
        Jv = ctx.jvp_linearized(vd).cpu().numpy()
        ref = osw.jvp(g, q, v, 1e-30)
        err = scaled_err_per_var(Jv, ref, term_scale(g, q, v))
        _report(f"split jvp ne{ne} ns{ns} seed{seed} bottom{bottom:g} v{k}", err, TOL_JVP)
        plain = ctx.jvp(qd, vd).cpu().numpy()
        err2 = scaled_err_per_var(Jv, plain, term_scale(g, q, v))
        assert max(err2) < TOL_JVP, (k, err2)


def test_split_requires_linearize():
    from paper_2101_05617_gb300 import swepi
    _, g, q, _ = oracle_case(2, 3, seed=1)
    ctx = _ctx(g)
    v = torch.ones(ctx.n, dtype=torch.float64, device="cuda")
    with pytest.raises(swepi.SWError):
        ctx.jvp_linearized(v)


@pytest.mark.parametrize("ne,ns,seed", [(4, 4, 0), (3, 6, 1)])
def test_jvp_parity_paper_eps(ne, ns, seed):
    """The paper's complex step eps ~ 1.5e-8 (Sec. 5 preamble) with v scaled like
    q: the kernels return the eps -> 0 limit, and the oracle's full complex
    evaluation of Im F(q + i eps v)/eps (Eq. 28) differs from it by O(eps^2)
    (relative (eps |v| / |q|)^2 ~ 2e-16), below the parity bound."""
    _, g, q, _ = oracle_case(ne, ns, seed=seed)
    ctx = _ctx(g)
    v = scaled_direction(q, seed + 300)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    vd = torch.tensor(v.reshape(-1), device="cuda")
    ref = osw.jvp(g, q, v, 1.5e-8)
    Jv = ctx.jvp(qd, vd, 1.5e-8).cpu().numpy()
    _report(f"jvp eps 1.5e-8 ne{ne} ns{ns}", scaled_err_per_var(Jv, ref, term_scale(g, q, v)), TOL_JVP)
    ctx.linearize(qd)
    Js = ctx.jvp_linearized(vd).cpu().numpy()
    _report(f"split jvp vs eps 1.5e-8 ne{ne} ns{ns}", scaled_err_per_var(Js, ref, term_scale(g, q, v)), TOL_JVP)


def _supersonic_case(ne, ns, seed):
    """A shallow layer (H = 20 m +- 10 m) under a strong wind (the balanced
    wind of the seeded height, scaled to a 60 m/s peak): Froude numbers u^d/a^d
    from ~0 to ~4 of both signs, so the AUSM splittings take the |M| > 1
    upwind branches (App. D, Eq. 138-143) at many interfaces and the
    subsonic polynomials at the others."""
    from oracle import fields as ofields
    f, g, _, _ = oracle_case(ne, ns, seed=seed)
    h, hB, V = f.evaluate(g.node_xyz())
    H = 20.0 + 0.1 * (h - 8000.0)
    V = V * (60.0 / np.max(np.linalg.norm(V.reshape(3, -1), axis=0)))
    q = ofields.state_from_fields(g, hB + H, hB, V)
    m = g.m
    Hn = q[0] / m['sqrtg']
    M1 = (q[1] / q[0]) / np.sqrt(m['h11'] * g.gr * Hn)
    M2 = (q[2] / q[0]) / np.sqrt(m['h22'] * g.gr * Hn)
    return g, q, M1, M2


@pytest.mark.parametrize("ne,ns,seed", [(4, 4, 2), (3, 5, 6)])
def test_supersonic_interface_parity(ne, ns, seed):
    g, q, M1, M2 = _supersonic_case(ne, ns, seed)
    for M in (M1, M2):
        frac = np.mean(np.abs(M) > 1.0)
        assert 0.2 < frac < 0.9, frac
        assert np.any(M > 1.0) and np.any(M < -1.0)
    ctx = _ctx(g)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    F = ctx.rhs(qd).cpu().numpy()
    _report(f"rhs supersonic ne{ne} ns{ns}", scaled_err_per_var(F, osw.rhs_real(g, q), term_scale(g, q)), TOL_RHS)
    v = scaled_direction(q, seed + 400)
    vd = torch.tensor(v.reshape(-1), device="cuda")
    ref = osw.jvp(g, q, v, 1e-30)
    Jv = ctx.jvp(qd, vd).cpu().numpy()
    _report(f"jvp supersonic ne{ne} ns{ns}", scaled_err_per_var(Jv, ref, term_scale(g, q, v)), TOL_JVP)
    ctx.linearize(qd)
    Js = ctx.jvp_linearized(vd).cpu().numpy()
    _report(f"split jvp supersonic ne{ne} ns{ns}", scaled_err_per_var(Js, ref, term_scale(g, q, v)), TOL_JVP)


def test_set_bottom_device_equals_host():
    """sw_set_bottom (device pointer) and sw_set_bottom_host give the same
    topography terms: RHS bit for bit, and both match the oracle."""
    from paper_2101_05617_gb300 import swepi
    _, g, q, hB = oracle_case(3, 5, seed=3, bottom_amp=1500.0)
    a, b = _ctx(g), _ctx(g)
    a.set_bottom(torch.tensor(hB.reshape(-1), device="cuda"))
    b.set_bottom(hB.reshape(-1))
    qd = torch.tensor(q.reshape(-1), device="cuda")
    Fa, Fb = a.rhs(qd), b.rhs(qd)
    assert torch.equal(Fa, Fb)
    _report("rhs device bottom", scaled_err_per_var(Fa.cpu().numpy(), osw.rhs_real(g, q), term_scale(g, q)), TOL_RHS)
    with pytest.raises(swepi.SWError):            # a host array given as the device pointer is refused
        host = np.ascontiguousarray(hB.reshape(-1))
        rc = swepi.lib().sw_set_bottom(a.handle, host.ctypes.data_as(swepi.ctypes.c_void_p))
        swepi._check("sw_set_bottom", rc)


def test_profile_brackets_every_nth_launch():
    """sw_profile_every(ctx, k): of the timed JVP kernel family only every k-th
    launch is bracketed by events (the counts say how many); the results of the
    JVPs are those of an unprofiled run bit for bit."""
    _, g, q, _ = oracle_case(4, 4, seed=0)
    ctx, ref_ctx = _ctx(g), _ctx(g)
    qd = torch.tensor(q.reshape(-1), device="cuda")
    vd = torch.tensor(scaled_direction(q, 3).reshape(-1), device="cuda")
    ctx.linearize(qd)
    ref_ctx.linearize(qd)
    ctx.profile_every(4)
    ctx.profile_kinds("volume_jvp")
    for _ in range(10):
        out = ctx.jvp_linearized(vd)
    st = ctx.profile_read()
    assert st["volume_jvp"]["count"] == 3 and st["volume_jvp"]["ms"] > 0     # launches 1, 5 and 9
    assert st["face_jvp"]["count"] == 0
    assert torch.equal(out, ref_ctx.jvp_linearized(vd))
    ctx.profile_every(1)
    ctx.profile_kinds("volume_jvp", "face_jvp")
    for _ in range(5):
        ctx.jvp_linearized(vd)
    st = ctx.profile_read()
    assert st["volume_jvp"]["count"] == 5 and st["face_jvp"]["count"] == 5
    from paper_2101_05617_gb300.swepi import SWError
    with pytest.raises(SWError):
        ctx.profile_every(0)
