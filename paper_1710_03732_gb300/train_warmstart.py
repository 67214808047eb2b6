"""Train the learned warm start of the Z-LAPs on the GPU.

Training pairs are (Z-LAP tile, its canonical optimal row duals) with the row
duals of the previous iteration as an extra feature, harvested from dual-ascent
runs on seeded synthetic instances with n = 20..25 (grid-distance instances of
the Nugent family and one dense instance of the Taillard-a family).  Feature
extraction, forward, backward and AdamW all run in the library's own CUDA
kernels (rlt2_mlp_*).  The trained weights go to an .npz file that
rlt2.Mlp.load() reads.

    python -m paper_1710_03732_gb300.train_warmstart --out weights/warmstart_h256.npz
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1710_03732_gb300 import instances as I  # noqa: E402

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart_h256.npz")


def training_instances():
    return [I.grid_instance("train_n20_4x5", 4, 5, 9, 0.5, 10, 0),
            I.grid_instance("train_n21_3x7", 3, 7, 9, 0.5, 11, 0),
            I.grid_instance("train_n22_2x11", 2, 11, 9, 0.6, 12, 0),
            I.grid_instance("train_n24_4x6", 4, 6, 9, 0.5, 13, 0),
            I.grid_instance("train_n25_5x5", 5, 5, 9, 0.5, 14, 0),
            I.dense_instance("train_n20_dense", 20, 99, 15, 0)]


def harvest(R, torch, mlp, inst, iters, snaps, tiles_per_snap, seed):
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0)) as ctx:
        T, m = ctx.T, ctx.n - 2
        D = torch.empty(ctx.E, dtype=torch.float64, device="cuda")
        xi = torch.empty(T * m, dtype=torch.float64, device="cuda")
        prev = torch.zeros(T * m, dtype=torch.float64, device="cuda")
        added = 0
        for it in range(1, iters + 1):
            ctx.iterate(1)
            R.rlt2_duals(ctx.ctx, xi=xi, on_device=1)
            if it in snaps:
                R.rlt2_export_state(ctx.ctx, Dhat=D, on_device=1)
                idx = torch.randperm(T, generator=gen, device="cuda")[:tiles_per_snap]
                mlp.add_samples(D.view(T, m, m)[idx].contiguous(), xi.view(T, m)[idx].contiguous(),
                                prev.view(T, m)[idx].contiguous())
                added += int(idx.numel())
            prev.copy_(xi)
    return added


def evaluate(R, mlp, inst, iters):
    """Z-stage augmenting searches and bounds: cold, previous-dual and learned starts."""
    out = {}
    for warm in (0, 1, 2):
        with R.Context(inst.F, inst.D, inst.B, prm=R.params(feas_tol=0.0, warm=warm)) as ctx:
            if warm == 2:
                ctx.set_mlp(mlp)
            lbs, _ = ctx.iterate(iters)
            st = ctx.stats()
        out[warm] = {"z_aug": int(st[1]), "z_relax": int(st[2]), "lb_last": float(lbs[-1])}
    out["same_bounds_rel"] = max(abs(out[w]["lb_last"] - out[0]["lb_last"]) / abs(out[0]["lb_last"]) for w in (1, 2))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--hidden", type=int, default=256)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--tiles-per-snap", type=int, default=20000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args()
    import torch
    from paper_1710_03732_gb300 import rlt2 as R
    R.lib()
    mlp = R.Mlp(args.hidden, seed=7)
    snaps = {2, 4, 8, 12, 20, 30, 40}
    t0 = time.time()
    rows = 0
    for k, inst in enumerate(training_instances()):
        rows += harvest(R, torch, mlp, inst, args.iters, snaps, args.tiles_per_snap, 100 + k) * (inst.n - 2)
    t1 = time.time()
    n1 = int(args.steps * 2 / 3)
    h1 = mlp.fit(n1, batch_rows=args.batch, lr=args.lr, weight_decay=1e-4, seed=1)
    h2 = mlp.fit(args.steps - n1, batch_rows=args.batch, lr=args.lr / 10, weight_decay=1e-4, seed=2)
    t2 = time.time()
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    mlp.save(args.out)
    held_out = I.grid_instance("heldout_n22_2x11", 2, 11, 9, 0.5, 99, 0)
    ev = evaluate(R, mlp, held_out, 30)
    hist = np.concatenate([h1, h2])
    print(json.dumps({"rows": rows, "harvest_s": t1 - t0, "train_s": t2 - t1,
                      "loss_first": float(hist[:50].mean()), "loss_last": float(hist[-50:].mean()),
                      "heldout_n22_30it": ev, "out": args.out}))


if __name__ == "__main__":
    main()
