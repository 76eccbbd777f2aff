"""Batched ensemble driver: builds the members of a seeded ensemble (one
library context per member, on its own grid and rotation) with their initial
states, and runs them through sw_ens_epi_run.  Marshalling only: the time
stepping runs in the library (ensemble.cu)."""
import os
import time

import numpy as np

from . import swepi, synth


def reset(ctxs):
    """Fresh EPI history (and KIOPS warm start) for every member."""
    for c in ctxs:
        swepi.sw_epi_reset(c.handle)


def build(members, ensemble_seed=0, workers=None, device="cuda"):
    """Contexts and initial states (float64 CUDA tensors) of `members`."""
    import torch
    ctxs = [swepi.SWContext(m.ne, m.p, synth.ensemble_rotation(m)) for m in members]
    xyz = [c.node_xyz().reshape(3, -1) for c in ctxs]
    if workers is None:
        workers = min(16, os.cpu_count() or 1) if sum(m.nodes for m in members) > 200000 else 1
    fields = synth.ensemble_member_fields(members, xyz, ensemble_seed, workers)
    qs = []
    for c, (h, hB, V) in zip(ctxs, fields):
        qs.append(torch.tensor(c.state_from_fields(h, hB, V).reshape(-1), device=device))
    return ctxs, qs


def run_single(members, ctxs, qs, steps, **opts):
    """Reference: every member alone through sw_epi_step from a fresh EPI
    history (on copies of qs); returns final states, per-member summed
    statistics and seconds."""
    import torch
    outs, stats = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m, c, q in zip(members, ctxs, qs):
        swepi.sw_epi_reset(c.handle)
        y = q.clone()
        tot = {"krylov_iters": 0, "rejects": 0, "substeps": 0}
        for _ in range(steps):
            st = c.epi_step(m.order, m.dt, y, **opts)
            for k in tot:
                tot[k] += st[k]
        outs.append(y)
        stats.append(tot)
    torch.cuda.synchronize()
    return outs, stats, time.perf_counter() - t0


def main():
    """Run a seeded ensemble and print one JSON line (members/s, statistics)."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--members", type=int, default=96)
    ap.add_argument("--one-per-class", action="store_true", help="keep the first member of each (n_e, p) class")
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--m-max", type=int, default=128)
    ap.add_argument("--no-tune", action="store_true")
    args = ap.parse_args()
    members = synth.ensemble_members(args.members, seed=args.seed)
    if args.one_per_class:
        seen, keep = set(), []
        for m in members:
            if (m.ne, m.p) not in seen:
                seen.add((m.ne, m.p))
                keep.append(m)
        members = keep
    ctxs, qs = build(members)
    ens = swepi.SWEnsemble(ctxs)
    block = None if args.no_tune else ens.tune(qs, iters=4)
    ys = [q.clone() for q in qs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ens.epi_run(args.steps, [m.order for m in members], [m.dt for m in members], ys, m_max=args.m_max)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    out = {"members": len(members), "steps": args.steps, "seconds": sec, "members_per_s": len(members) / sec,
           "krylov_iters": sum(s["krylov_iters"] for s in st), "tuned_block": block, **ens.stats()}
    ens.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
