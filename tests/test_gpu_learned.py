"""Learned Krylov control: the network's hand-written BF16/FP32 kernels against
the FP64 reference network, training, the KIOPS call log, and what the trained
controller gains over the plain adaptive rule at the same tolerance."""
import numpy as np
import pytest

from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _random_net(seed):
    from paper_2101_05617_gb300 import learned, swepi
    rng = np.random.default_rng(seed)
    norm = np.concatenate([rng.standard_normal(16), rng.uniform(0.5, 2, 16), rng.standard_normal(2),
                           rng.uniform(0.5, 2, 2)]).astype(np.float32)
    ctl = learned.Controller(learned.glorot_init(seed), norm)
    X = (rng.standard_normal((300, 16)) * norm[16:32] + norm[:16]).astype(np.float32)
    T = rng.standard_normal((300, 2)).astype(np.float32)
    return ctl, norm, X, T, swepi


def test_forward_and_gradient_match_fp64_reference():
    """BF16 weights with FP32 accumulation against the FP64 network evaluated
    on the same (BF16-rounded) weights."""
    ctl, norm, X, T, swepi = _random_net(1)
    _, wb = swepi.sw_mlp_get_params(ctl.handle)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
    swepi.sw_mlp_forward(ctl.handle, Xd, Y)
    ref = omlp.predict(wb.astype(np.float64), norm, X)
    assert np.linalg.norm(Y.cpu().numpy() - ref) < 1e-5 * np.linalg.norm(ref)
    g, loss = swepi.sw_mlp_gradient(ctl.handle, Xd, Td)
    lo, go = omlp.loss_and_grad(wb.astype(np.float64), norm, X, T)
    assert abs(loss - lo) < 1e-5 * lo
    assert np.linalg.norm(g - go) < 1e-4 * np.linalg.norm(go)


def test_training_fits_a_smooth_map():
    ctl, norm, X, _, swepi = _random_net(2)
    Xs = (X - norm[:16]) / norm[16:32]
    T = np.stack([np.tanh(Xs[:, 0] - 0.5 * Xs[:, 3]), 0.3 * Xs[:, 5] * Xs[:, 7]], axis=1).astype(np.float32)
    T = T * norm[34:36] + norm[32:34]
    losses = swepi.sw_mlp_train(ctl.handle, torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"),
                                1500, 3e-3)
    assert losses[-1] < 0.05 * losses[0], (losses[0], losses[-1])


def test_kiops_log_records():
    from paper_2101_05617_gb300 import swepi, synth
    wl = synth.WORKLOADS["small_ne4_p3"]
    f = synth.make_fields(wl, 0)
    ctx = swepi.SWContext(wl.ne, wl.p, f.rotation)
    h, hB, V = f.evaluate(ctx.node_xyz())
    q = torch.tensor(ctx.state_from_fields(h, hB, V), device="cuda")
    for _ in range(4):
        ctx.epi_step(wl.order, wl.dt, q, tol=wl.tol)
    rec = swepi.sw_kiops_log(ctx.handle)
    # 2 start-up steps x 8 EPI2 substeps + 2 EPI4 steps
    assert rec.shape == (18, swepi.KIOPS_LOG_FIELDS)
    assert np.all(rec[:, 22] >= rec[:, 16] - 1e-6)        # tau_star >= accepted tau_1
    assert np.all(rec[:, 16] <= 1e-6)                      # tau_1 <= tau_out
    assert np.all(rec[-2:, 12] == 4) and np.all(rec[:16, 13] == 1)
    swepi.sw_kiops_log_clear(ctx.handle)
    assert swepi.sw_kiops_log(ctx.handle).shape[0] == 0


def test_nonfinite_prediction_falls_back_to_plain_rule():
    from paper_2101_05617_gb300 import learned, swepi, synth
    wl = synth.WORKLOADS["small_ne4_p3"]
    bad = learned.Controller(np.full(swepi.MLP_PARAMS, np.nan, dtype=np.float32), np.ones(swepi.MLP_NORM,
                                                                                          dtype=np.float32))
    stats = []
    for use in (False, True):
        f = synth.make_fields(wl, 0)
        ctx = swepi.SWContext(wl.ne, wl.p, f.rotation)
        h, hB, V = f.evaluate(ctx.node_xyz())
        q = torch.tensor(ctx.state_from_fields(h, hB, V), device="cuda")
        if use:
            swepi.sw_set_controller(ctx.handle, bad.handle)
        stats.append([ctx.epi_step(wl.order, wl.dt, q, tol=wl.tol) for _ in range(4)])
        swepi.sw_set_controller(ctx.handle, None)
    assert stats[0] == stats[1]


def test_trained_controller_gains_on_held_out_fields():
    """The committed network (trained on plain-rule logs of the small, 6x30x30
    and 6x90x90 grids, seed 0) on unseen fields (seed 2) of the 6x30x30 grid:
    fewer Krylov iterations than the plain rule at the same tolerance, and the
    same solution to the tolerance."""
    from paper_2101_05617_gb300 import learned
    ctl = learned.Controller.load()
    res = learned.evaluate(ctl, "ne30_p5", steps=8, seed=2)
    assert res["learned"]["krylov_iters"] < res["plain"]["krylov_iters"], res
    assert max(res["state_rel_diff"]) < 1e-7, res
