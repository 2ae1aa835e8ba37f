"""Train the learned per-step (tau, delta) policy on a large generated set and
store its weights.

    python -m paper_2106_03138_gb300.train_policy --matrices 2000 --n-hi 2048 \
        --out paper_2106_03138_gb300/policy_weights.npz

The set is the module's recipe (policy.training_entries): square matrices, n
log-uniform in [n_lo, n_hi], the three spectrum kinds in turn.  It is swept in
chunks (each chunk: the (tau, delta) grid with the batched kernel, the labels
of policy.collect), then the MLP is trained by the library's own kernels
(qrdm_mlp_train).  The weights (FP32 master copy) and a summary of the run go
to the output file; ``policy.Policy.load`` reads them back.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main() -> int:
    import torch

    from . import load
    from . import policy as P

    ap = argparse.ArgumentParser()
    ap.add_argument("--matrices", type=int, default=2000)
    ap.add_argument("--n-lo", type=int, default=64)
    ap.add_argument("--n-hi", type=int, default=2048)
    ap.add_argument("--chunk", type=int, default=250, help="matrices per sweep")
    ap.add_argument("--seed", type=int, default=21)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--quality-factor", type=float, default=0.75)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    load()
    entries = P.training_entries(args.matrices, seed=args.seed, n_lo=args.n_lo, n_hi=args.n_hi)
    Xs, Ts = [], []
    labels: dict = {}
    t0 = time.perf_counter()
    for c in range(0, len(entries), args.chunk):
        part = entries[c:c + args.chunk]
        pristine = [e.build_gpu() for e in part]
        X, T, info = P.collect(part, pristine, quality_factor=args.quality_factor, grid_tau=P.GRID_TAU_FINE)
        Xs.append(X)
        Ts.append(T)
        for k, v in info["label_counts"].items():
            labels[k] = labels.get(k, 0) + v
        del pristine
        torch.cuda.empty_cache()
        print(json.dumps({"chunk": c // args.chunk, "matrices": len(part), "samples": int(X.shape[0]),
                          "elapsed_s": round(time.perf_counter() - t0, 1)}), flush=True)
    X = np.concatenate(Xs)
    T = np.concatenate(Ts)
    sweep_s = time.perf_counter() - t0
    pol = P.Policy(seed=2)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss = pol.train(X, T, steps=args.steps, batch=args.batch, lr=args.lr)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    summary = {"matrices": len(entries), "n_range": [args.n_lo, args.n_hi], "seed": args.seed,
               "samples": int(X.shape[0]), "label_counts": labels, "sweep_and_label_s": sweep_s,
               "train_steps": args.steps, "batch": args.batch, "lr": args.lr, "train_s": train_s,
               "quality_factor": args.quality_factor,
               "loss_first50": float(loss[:50].mean()), "loss_last50": float(loss[-50:].mean()),
               "grid_tau": list(P.GRID_TAU_FINE), "grid_delta": list(P.GRID_DELTA)}
    np.savez(args.out, w32=pol.w32.cpu().numpy(), summary=json.dumps(summary))
    print(json.dumps(summary), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
