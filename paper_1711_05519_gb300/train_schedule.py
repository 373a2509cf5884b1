"""Trains the learned threshold schedule and writes its packed parameters.

Training instances follow the planted recipe of Section 3 at m = n = 3000 with r drawn from
{3, 5, 10}, alpha ~ U[0.05, 0.3] and c ~ U[0.5, 3]; each training step unrolls 12
iterations of the library's iteration on one instance (soft gate, tau = 0.05) and updates
the parameters with the library's backward and Adam kernels.  Usage:

    python -m paper_1711_05519_gb300.train_schedule --out paper_1711_05519_gb300/schedule_theta.npz
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_1711_05519_gb300 import learned as PL  # noqa: E402


def make_instance(n, seed, rng, r=None, alpha=None, c=None, device="cuda"):
    r = int(r if r is not None else rng.choice([3, 5, 10]))
    alpha = float(alpha if alpha is not None else rng.uniform(0.05, 0.3))
    c = float(c if c is not None else rng.uniform(0.5, 3.0))
    inst = synth.planted_instance(n, n, r, alpha, c, seed)
    p = inst.params()
    return {"D": torch.from_numpy(inst.D).float().to(device), "r": r, "beta": p["beta"], "gamma": p["gamma"],
            "mu": p["mu"], "P": torch.from_numpy(inst.P).to(device), "Q": torch.from_numpy(inst.Q).to(device),
            "alpha": alpha, "c": c, "seed": seed}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=3000)
    ap.add_argument("--instances", type=int, default=8)
    ap.add_argument("--steps", type=int, default=160)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedule_theta.npz"))
    args = ap.parse_args()
    from paper_1711_05519_gb300 import build

    build.build()
    rng = np.random.default_rng(1000)
    train = [make_instance(args.n, 1000 + i, rng) for i in range(args.instances)]
    log = []
    t0 = time.time()
    theta = PL.train(train, K=12, steps=args.steps, lr=args.lr, log=log)
    torch.cuda.synchronize()
    PL.save_theta(theta, args.out)
    print(json.dumps({"trained_s": round(time.time() - t0, 1), "loss_first": log[:5], "loss_last": log[-5:],
                      "out": args.out}))


if __name__ == "__main__":
    main()
