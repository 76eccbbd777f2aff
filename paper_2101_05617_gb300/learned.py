"""Learned Krylov control: data collection, training and evaluation driver.

The network (16 -> 64 -> 64 -> 2, GELU, BF16 weights, FP32 accumulation) and
its forward/backward/Adam kernels live in the library (sw_mlp_*).  This module
only marshals data: it runs the plain adaptive KIOPS rule inside multistep EPI
integrations, reads the per-call log (sw_kiops_log), trains the network on the
GPU to predict each call's first accepted substep log(tau_1/tau_out) and Krylov
size m_1/m_max from the call's features, and evaluates the learned initial
choice against the plain rule.  The KIOPS error estimate keeps accepting or
rejecting every substep in both.  The substep target is the largest first
substep the error model admits, tau_star = tau_1 (0.8/omega_1)^(1/order), rather
than the accepted tau_1 itself: a too-small first substep costs a whole extra
Krylov basis, a too-large one only a rejection that reuses the basis.

    python -m paper_2101_05617_gb300.learned train --out weights.npz
    python -m paper_2101_05617_gb300.learned eval --weights weights.npz
"""
import argparse
import json
import os
import time

import numpy as np

from . import swepi, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "controller_weights.npz")

# (workload, EPI steps, time-step factors): the small, 6x30x30 and 6x90x90 grids
TRAINING_RUNS = [("small_ne4_p3", 12, (0.5, 1.0, 2.0, 4.0)), ("ne30_p5", 10, (0.5, 1.0, 2.0)),
                 ("ne90_p6", 6, (1.0,))]


def _initial_state(wl, seed, dev):
    import torch
    f = synth.make_fields(wl, seed)
    ctx = swepi.SWContext(wl.ne, wl.p, f.rotation)
    h, hB, V = f.evaluate(ctx.node_xyz())
    q = torch.tensor(ctx.state_from_fields(h, hB, V), device=dev)
    return ctx, q


def collect_logs(runs=TRAINING_RUNS, seed=0, dev="cuda"):
    """Per-call KIOPS records of plain-rule EPI integrations."""
    recs = []
    for name, steps, factors in runs:
        wl = synth.WORKLOADS[name]
        for fac in factors:
            ctx, q = _initial_state(wl, seed, dev)
            for _ in range(steps):
                ctx.epi_step(wl.order, wl.dt * fac, q, tol=wl.tol)
            recs.append(swepi.sw_kiops_log(ctx.handle))
            ctx.close()
    return np.concatenate(recs, axis=0)


def training_pairs(records):
    """Features and targets: log(tau_star/tau_out) (the largest first substep the
    error model admitted) and m_1/m_max of the first accepted substep."""
    X = records[:, :16].astype(np.float32)
    T = np.stack([records[:, 22], records[:, 17]], axis=1).astype(np.float32)
    return X, T


def normalisation(X, T):
    mx, sx = X.mean(axis=0), X.std(axis=0)
    sx = np.where(sx < 1e-6, 1.0, sx)
    mt, st = T.mean(axis=0), T.std(axis=0)
    st = np.where(st < 1e-6, 1.0, st)
    return np.concatenate([mx, sx, mt, st]).astype(np.float32)


def glorot_init(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((64, 16), (64, 0), (64, 64), (64, 0), (2, 64), (2, 0)):
        if fan_in == 0:
            parts.append(np.zeros(fan_out))
        else:
            lim = np.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
    return np.concatenate(parts).astype(np.float32)


class Controller:
    """A trained network on the device (sw_mlp_t)."""

    def __init__(self, params, norm):
        self.handle = swepi.sw_mlp_create()
        self.params = np.asarray(params, dtype=np.float32)
        self.norm = np.asarray(norm, dtype=np.float32)
        swepi.sw_mlp_set_params(self.handle, self.params, self.norm)

    def close(self):
        if self.handle:
            swepi.sw_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path, meta=None):
        np.savez(path, params=self.params, norm=self.norm, meta=json.dumps(meta or {}))

    @classmethod
    def load(cls, path=DEFAULT_WEIGHTS):
        d = np.load(path)
        return cls(d["params"], d["norm"])


def train(records, steps=3000, lr=3e-3, seed=0, dev="cuda"):
    import torch
    X, T = training_pairs(records)
    norm = normalisation(X, T)
    ctl = Controller(glorot_init(seed), norm)
    Xd = torch.tensor(X, device=dev)
    Td = torch.tensor(T, device=dev)
    losses = swepi.sw_mlp_train(ctl.handle, Xd, Td, steps, lr)
    ctl.params, _ = swepi.sw_mlp_get_params(ctl.handle)
    return ctl, losses


def evaluate(ctl, workload="ne60_p5", steps=8, seed=1, dev="cuda"):
    """Plain rule against the learned initial choice from the same state, at the
    same tolerance: Krylov iterations, rejections, substeps, steps/s and the
    relative difference of the final states."""
    import torch
    wl = synth.WORKLOADS[workload]
    out = {}
    finals = {}
    for name, use in (("plain", False), ("learned", True)):
        ctx, q = _initial_state(wl, seed, dev)
        P = {2: 0, 3: 1, 4: 2, 5: 3, 6: 4}[wl.order]
        for _ in range(P):                       # start-up steps, plain in both
            ctx.epi_step(wl.order, wl.dt, q, tol=wl.tol)
        if use:
            swepi.sw_set_controller(ctx.handle, ctl.handle)
        tot = {"krylov_iters": 0, "rejects": 0, "substeps": 0}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            st = ctx.epi_step(wl.order, wl.dt, q, tol=wl.tol)
            for k in tot:
                tot[k] += st[k]
        torch.cuda.synchronize()
        tot["steps_per_s"] = steps / (time.perf_counter() - t0)
        out[name] = tot
        finals[name] = q.view(3, -1).clone()
        swepi.sw_set_controller(ctx.handle, None)
        ctx.close()
    a, b = finals["learned"], finals["plain"]
    out["state_rel_diff"] = [float(torch.linalg.norm(a[k] - b[k]) / torch.linalg.norm(b[k])) for k in range(3)]
    out["workload"] = workload
    out["steps"] = steps
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--weights", default=DEFAULT_WEIGHTS)
    ap.add_argument("--steps", type=int, default=3000)
    args = ap.parse_args()
    if args.cmd == "train":
        t0 = time.time()
        rec = collect_logs()
        t1 = time.time()
        ctl, losses = train(rec, steps=args.steps)
        meta = {"records": int(rec.shape[0]), "final_loss": float(losses[-1]), "first_loss": float(losses[0]),
                "collect_s": t1 - t0, "train_s": time.time() - t1,
                "runs": [[n, s, list(f)] for n, s, f in TRAINING_RUNS]}
        ctl.save(args.out, meta)
        print(json.dumps(meta))
        print(json.dumps(evaluate(ctl)))
    else:
        print(json.dumps(evaluate(Controller.load(args.weights))))


if __name__ == "__main__":
    main()
