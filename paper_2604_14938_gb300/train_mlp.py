"""Trains the isovalue-guess MLP on the GPU with the library's BF16 kernels.

Input: an .npz with float32 features X [n, 40] and targets t [n] (oracle-labelled cut cells).
Output: float32 parameters (.npy) in the layout of vof_mlp_create, and one JSON line per epoch.

    python -m paper_2604_14938_gb300.train_mlp --data iso_train.npz --out mlp_iso.npy
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np


def init_params(seed: int) -> np.ndarray:
    """Seeded initial parameters: normal weights with variance 1/fan-in, zero biases, b4 = 0.5."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, 1 / math.sqrt(40), 64 * 40), np.zeros(64), rng.normal(0, 1 / 8, 64 * 64), np.zeros(64),
             rng.normal(0, 1 / 8, 64 * 64), np.zeros(64), rng.normal(0, 1 / 8, 64), [0.5]]
    return np.concatenate(parts).astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--epochs", type=int, default=16)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--val", type=float, default=0.05)
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import paper_2604_14938_gb300 as vof

    d = np.load(args.data)
    X = torch.as_tensor(d["X"], dtype=torch.float32, device="cuda")
    t = torch.as_tensor(d["t"], dtype=torch.float32, device="cuda")
    n = len(t)
    nval = int(n * args.val)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed)
    order = torch.randperm(n, generator=gen, device="cuda")
    val, tr = order[:nval], order[nval:]
    mlp = vof.Mlp(init_params(args.seed))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    steps = args.epochs * ((len(tr) + args.batch - 1) // args.batch)
    k = 0
    t0 = time.time()
    Xv, tv = X[val].contiguous(), t[val].contiguous()
    for ep in range(args.epochs):
        # one shuffled copy per epoch; the batches are contiguous slices of it
        perm = tr[torch.randperm(len(tr), generator=gen, device="cuda")]
        Xe, te = X[perm].contiguous(), t[perm].contiguous()
        torch.cuda.synchronize()
        te0 = time.time()
        for b0 in range(0, len(perm), args.batch):
            lr = args.lr * 0.5 * (1 + math.cos(math.pi * k / steps))  # cosine schedule
            mlp.train_step(Xe[b0:b0 + args.batch], te[b0:b0 + args.batch], lr, loss)
            k += 1
        torch.cuda.synchronize()
        train_s = time.time() - te0
        yv = mlp.forward(Xv)
        err = (yv - tv).abs()
        print(json.dumps({"epoch": ep, "val_mse": float((err * err).mean()), "val_mae": float(err.mean()),
                          "val_p99": float(err.quantile(0.99)), "train_seconds": round(train_s, 3),
                          "seconds": round(time.time() - t0, 1)}), flush=True)
    np.save(args.out, mlp.params())


if __name__ == "__main__":
    main()
