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


VALIDATION_SEEDS = tuple(range(2000, 2010))  # 4096^2 validation matrices, apart from the held-out 1000..1009
RHO_GRID = (0.5, 0.6, 0.7, 0.8, 0.9)


def calibrate_rho(path: str, bar: float = 0.6, n: int = 4096) -> dict:
    """Choose the guard threshold rho_min of stored weights on validation
    matrices (n x n, sigma geometric 1 -> 1e-12 over 3n/4 values then 1e-15,
    seeds VALIDATION_SEEDS): every rho in RHO_GRID is tried, and the smallest
    one for which every validation matrix keeps sigma_min(R11) / sigma_r at
    least `bar` times that of fixed (0.9, 0.9) (exact sigma_min of the r x r
    block) is taken; the largest rho when none does.  Writes it into the
    file's summary and returns the calibration record (per rho: the worst and
    median quality ratio and the median time ratio against fixed)."""
    import torch

    from . import factor, inputs, qrdm_workspace_size
    from . import policy as P

    r = 3 * n // 4
    sig = inputs.sigma_rank_geometric(n, r)
    ws = torch.empty(qrdm_workspace_size(n, n, 64), dtype=torch.uint8, device="cuda")
    pol = P.Policy.load(path)

    def run(A0, kw):
        best = None
        for _ in range(2):  # the second run is timed warm
            dA = A0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            f = factor(dA, 0.9, 0.9, 64, workspace=ws, **kw)
            torch.cuda.synchronize()
            best = 1e3 * (time.perf_counter() - t0)
        q = float(torch.linalg.svdvals(torch.triu(dA[:r, :r]))[-1]) / float(sig[r - 1])
        return best, f.nsteps, q

    record = {"seeds": list(VALIDATION_SEEDS), "bar": bar, "trials": []}
    ref, got = [], {rho: [] for rho in RHO_GRID}
    for sd in VALIDATION_SEEDS:
        A0 = inputs.from_spectrum_gpu(n, n, sig, sd)
        ref.append(run(A0, {}))
        for rho in RHO_GRID:
            pol.rho_min = rho
            got[rho].append(run(A0, {"policy": pol.struct()}))
        del A0
    chosen = None
    for rho in RHO_GRID:
        ratios = [g[2] / rf[2] for g, rf in zip(got[rho], ref)]
        times = [g[0] / rf[0] for g, rf in zip(got[rho], ref)]
        record["trials"].append({"rho_min": rho, "quality_ratio_min": min(ratios),
                                 "quality_ratio_median": float(np.median(ratios)),
                                 "time_ratio_median": float(np.median(times))})
        if chosen is None and min(ratios) >= bar:
            chosen = rho
    record["rho_min"] = chosen if chosen is not None else RHO_GRID[-1]
    with np.load(path) as z:
        w = z["w32"]
        summary = json.loads(str(z["summary"]))
    summary["rho_min"] = record["rho_min"]
    summary["rho_calibration"] = record
    np.savez(path, w32=w, summary=json.dumps(summary))
    return record


def main() -> int:
    import torch

    from . import load
    from . import policy as P

    ap = argparse.ArgumentParser()
    ap.add_argument("--matrices", type=int, default=2000)
    ap.add_argument("--n-lo", type=int, default=256)
    ap.add_argument("--n-hi", type=int, default=2048)
    ap.add_argument("--chunk", type=int, default=250, help="matrices per sweep")
    ap.add_argument("--seed", type=int, default=21)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--quality-factor", type=float, default=0.9)
    ap.add_argument("--grid-tau", default="0.5,0.6,0.7,0.8,0.9", help="comma-separated tau grid")
    ap.add_argument("--grid-delta", default="0.5,0.7,0.9", help="comma-separated delta grid")
    ap.add_argument("--tau-lo", type=float, default=0.5, help="lower end of the policy's tau output range")
    ap.add_argument("--out", required=True)
    ap.add_argument("--calibrate-only", action="store_true",
                    help="only choose rho_min for the weights already in --out (validation matrices)")
    args = ap.parse_args()
    load()
    if args.calibrate_only:
        print(json.dumps(calibrate_rho(args.out)), flush=True)
        return 0
    grid_tau = tuple(float(x) for x in args.grid_tau.split(","))
    grid_delta = tuple(float(x) for x in args.grid_delta.split(","))
    tau_range = (args.tau_lo, P.TAU_RANGE[1])
    if P.REFERENCE[0] not in grid_tau or P.REFERENCE[1] not in grid_delta:
        raise SystemExit("the grid must hold the reference (0.9, 0.9)")
    entries = P.training_entries(args.matrices, seed=args.seed, n_lo=args.n_lo, n_hi=args.n_hi)
    Xs, Ts = [], []
    labels: dict = {}
    t0 = time.perf_counter()
    for c in range(0, len(entries), args.chunk):
        part = entries[c:c + args.chunk]
        pristine = [e.build_gpu() for e in part]
        X, T, info = P.collect(part, pristine, quality_factor=args.quality_factor, grid_tau=grid_tau,
                               grid_delta=grid_delta, tau_range=tau_range)
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
    pol = P.Policy(seed=2, tau_range=tau_range)
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
               "grid_tau": list(grid_tau), "grid_delta": list(grid_delta), "tau_range": list(tau_range),
               "delta_range": list(P.DELTA_RANGE), "rho_min": P.RHO_MIN}
    np.savez(args.out, w32=pol.w32.cpu().numpy(), summary=json.dumps(summary))
    summary["rho_calibration"] = calibrate_rho(args.out)
    print(json.dumps(summary), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
