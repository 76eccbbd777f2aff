"""Checkpoint and resume of the multistep EPI state (sw_epi_checkpoint_*):
the history pairs (q_{n-i}, F(q_{n-i})) that the remainders of Eq. 33-38 read,
the KIOPS warm start and the learned controller's previous-call features.  A
context restored from a checkpoint continues bit for bit as the saved one."""
import numpy as np
import pytest

from tests.gpu_common import oracle_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(g, mode=1):
    from paper_2101_05617_gb300.swepi import SWContext
    c = SWContext(g.ne, g.ns - 1, g.rotation)
    c.set_jvp_mode(mode)
    return c


@pytest.mark.parametrize("order,n_save,n_more,mode,learned", [
    (5, 4, 3, 1, False),     # history full (P = 3, four entries held)
    (6, 2, 4, 1, False),     # saved during the EPI2 start-up (two of four entries)
    (4, 3, 3, 2, False),     # complex64-bulk form
    (5, 3, 3, 1, True),      # learned initial substep: the previous-call features travel too
    (4, 0, 3, 1, False),     # empty history: the resumed run starts up like a fresh one
])
def test_resume_is_bitwise(order, n_save, n_more, mode, learned):
    from paper_2101_05617_gb300 import learned as lrn
    from paper_2101_05617_gb300 import swepi
    _, g, q, _ = oracle_case(4, 4, seed=1)
    dt, tol = 900.0, 1e-12
    a, b = _ctx(g, mode), _ctx(g, mode)
    ctl = lrn.Controller.load() if learned else None
    if ctl is not None:
        swepi.sw_set_controller(a.handle, ctl.handle)
        swepi.sw_set_controller(b.handle, ctl.handle)
    try:
        qa = torch.tensor(q.reshape(-1), device="cuda")
        for _ in range(n_save):
            a.epi_step(order, dt, qa, tol=tol)
        ck = a.epi_checkpoint()
        assert ck.size == swepi.sw_epi_checkpoint_size(a.handle) == 144 + 16 * qa.numel() * min(n_save, 4)
        qb = qa.clone()
        sa = [a.epi_step(order, dt, qa, tol=tol) for _ in range(n_more)]
        b.epi_restore(ck)
        sb = [b.epi_step(order, dt, qb, tol=tol) for _ in range(n_more)]
        assert sa == sb, (sa, sb)
        assert torch.equal(qa, qb)
    finally:
        if ctl is not None:
            swepi.sw_set_controller(a.handle, None)
            swepi.sw_set_controller(b.handle, None)


def test_resume_differs_from_restart():
    """The checkpoint carries state that matters: the same q continued without
    it (a fresh context, which starts up with EPI2) takes another trajectory."""
    _, g, q, _ = oracle_case(4, 4, seed=1)
    a, b = _ctx(g), _ctx(g)
    qa = torch.tensor(q.reshape(-1), device="cuda")
    for _ in range(3):
        a.epi_step(4, 900.0, qa, tol=1e-12)
    qb = qa.clone()
    a.epi_step(4, 900.0, qa, tol=1e-12)
    b.epi_step(4, 900.0, qb, tol=1e-12)
    assert not torch.equal(qa, qb)


def test_load_rejects_foreign_or_damaged_checkpoints():
    """A checkpoint of another grid or rotation, a damaged payload or a wrong
    size is refused with SW_EINVAL and leaves the context's state untouched."""
    from paper_2101_05617_gb300.swepi import SWContext, SWError
    _, g, q, _ = oracle_case(4, 4, seed=1)
    a, b = _ctx(g), _ctx(g)
    qa = torch.tensor(q.reshape(-1), device="cuda")
    for _ in range(3):
        a.epi_step(4, 900.0, qa, tol=1e-12)
    ck = a.epi_checkpoint()
    b.epi_restore(ck)
    good_b = b.epi_checkpoint()
    assert np.array_equal(good_b, ck)

    other_grid = SWContext(3, 3, g.rotation)
    other_rot = SWContext(4, 3, tuple(r + 0.1 for r in g.rotation))
    bad_payload = ck.copy()
    bad_payload[-5] ^= 0x40
    bad_magic = ck.copy()
    bad_magic[0] ^= 1
    for ctx, buf in [(other_grid, ck), (other_rot, ck), (b, bad_payload), (b, bad_magic), (b, ck[:-8]),
                     (b, np.concatenate([ck, np.zeros(8, np.uint8)])), (b, ck[:100])]:
        with pytest.raises(SWError) as e:
            ctx.epi_restore(buf)
        assert e.value.status == -1          # SW_EINVAL
    assert np.array_equal(b.epi_checkpoint(), ck)     # b kept the state it had
    # and continues as a does
    qb = qa.clone()
    sa = a.epi_step(4, 900.0, qa, tol=1e-12)
    sb = b.epi_step(4, 900.0, qb, tol=1e-12)
    assert sa == sb and torch.equal(qa, qb)
