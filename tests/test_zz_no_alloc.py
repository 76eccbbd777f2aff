"""sw_jvp_static_scratch: the JVP for callers that may not allocate device
memory while running (their memory manager owns the device memory, or they run
where cudaMalloc is not allowed or its implicit synchronisation cannot be
afforded).  It keeps its interface-flux scratch in a fixed array inside the
library; these tests call it through the C ABI and check it against the oracle's
complex-step JVP (Eq. 28) and against sw_jvp, and that its calls leave the
device's free memory unchanged.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from oracle import shallow_water as osw
from tests.gpu_common import oracle_case, scaled_direction, scaled_err_per_var, term_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_JVP = 8e-14     # same bound as the JVP parity tests (fraction of the term scale)


def _raw_call(lib, ctx, q, v, eps, out):
    return lib.sw_jvp_static_scratch(ctx, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                     ctypes.c_double(eps), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("ne,ns,seed", [(4, 4, 0), (6, 6, 3)])
def test_static_scratch_matches_oracle_two_calls(ne, ns, seed):
    from paper_2101_05617_gb300 import swepi
    _, g, q, hB = oracle_case(ne, ns, seed=seed)
    ctx = swepi.SWContext(g.ne, g.ns - 1, g.rotation)
    lib = swepi.lib()
    qd = torch.tensor(q.reshape(-1), device="cuda")
    for call, vseed in enumerate((seed + 1, seed + 2)):       # two calls in a row reuse the array
        v = scaled_direction(q, vseed)
        vd = torch.tensor(v.reshape(-1), device="cuda")
        ref = osw.jvp(g, q, v, 1e-30)
        out = torch.full_like(qd, float("nan"))
        rc = _raw_call(lib, ctx.handle, qd, vd, 1e-30, out)
        assert rc == 0, swepi.sw_status_str(rc)
        torch.cuda.synchronize()
        a = out.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}: unwritten entries"
        err = scaled_err_per_var(a, ref, term_scale(g, q, v))
        assert max(err) < TOL_JVP, (call, err)
        err2 = scaled_err_per_var(a, ctx.jvp(qd, vd, 1e-30).cpu().numpy(), term_scale(g, q, v))
        assert max(err2) < TOL_JVP, (call, err2)


def test_static_scratch_allocates_nothing():
    """After a first call (the one-time address lookup), further calls leave the
    device's free memory as it was: the library makes no cudaMalloc of its own,
    which torch's allocator statistics would not show."""
    from paper_2101_05617_gb300 import swepi
    _, g, q, _ = oracle_case(5, 5, seed=2)
    ctx = swepi.SWContext(g.ne, g.ns - 1, g.rotation)
    lib = swepi.lib()
    qd = torch.tensor(q.reshape(-1), device="cuda")
    vd = torch.tensor(scaled_direction(q, 11).reshape(-1), device="cuda")
    out = torch.empty_like(qd)
    assert _raw_call(lib, ctx.handle, qd, vd, 1e-30, out) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert _raw_call(lib, ctx.handle, qd, vd, 1e-30, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_rejects_oversized_grid():
    from paper_2101_05617_gb300 import swepi
    ctx = swepi.SWContext(70, 6)            # 6*70^2 elements * 12 * 7 = 2,469,600 > 2^21 scratch doubles
    n = ctx.n
    q = torch.ones(n, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(q)
    rc = _raw_call(swepi.lib(), ctx.handle, q, q.clone(), 1e-30, out)
    assert rc == -7
    assert "scratch" in swepi.sw_status_str(rc)
    assert torch.count_nonzero(out).item() == 0
