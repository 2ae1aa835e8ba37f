#!/usr/bin/env python
"""QRDM benchmark on GB300.

One step = factor the plain-FP64 single-matrix workload: a 4096 x 4096 and an
8192 x 2048 matrix with geometric singular values 1 -> 1e-15, and the Kahan
matrix of order 2048 (c = 0.285), each A Pi = QR with QRDM2 at the paper's
recommended tau = 0.15, delta = 0.9 and block size k_DM = 64 (Sec. 5).
Metric: GFLOP/s = sum over the matrices of (4 m n^2 - 4 n^3 / 3) / time.

Inputs are seeded synthetic matrices built on the host, copied to HBM once;
before every step the factored matrices are restored from pristine device
copies and L2 is flushed (a 256 MB write), both outside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank factors its own replica of the workload (the path
does not shard; there is no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QRDM GFLOP/s (4mn²−4n³/3) vs plain FP64 GPU QRDM at equal rank quality"
TAU, DELTA, KMAX = 0.15, 0.9, 64
WORKLOAD = ("geo4096", "geo8192x2048", "kahan2048")
WORKLOAD_DESC = ("plain FP64 QRDM on single matrices: 4096x4096 and 8192x2048 with geometric sigma 1->1e-15, "
                 "Kahan n=2048 (c=0.285)")
# the CPU sample: the same recipes at half the linear size
CPU_SAMPLE = (("geo", 2048, 2048), ("geo", 4096, 1024), ("kahan", 1024, 1024))
FP64_FLOP_PER_CLK_PER_SM = 4.0  # 2 FP64 FMA per clock per SM on GB300 (1.25 TFLOP/s nominal at 2070 MHz)
L2_FLUSH_BYTES = 256 << 20


def metric_flops(m: int, n: int) -> float:
    return 4.0 * m * n * n - 4.0 * n ** 3 / 3.0


def executed_flops(m: int, n: int, r: int) -> float:
    """The metric's count for the work actually done when the factorization
    stops after r columns: twice the Householder flops of the first r
    columns, 2 * sum_{i<r} 4 (m - i)(n - i) ~ 8 (m n r - (m + n) r^2 / 2 +
    r^3 / 3); equals metric_flops(m, n) at r = n <= m."""
    return 8.0 * (m * n * r - (m + n) * r * r / 2.0 + r ** 3 / 3.0)


def host_cpu() -> dict:
    """Core count and CPU model of this host."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown", "machine": os.uname().machine}


def cpu_sample_matrices():
    from paper_2106_03138_gb300 import inputs

    out = []
    for kind, m, n in CPU_SAMPLE:
        if kind == "geo":
            out.append(inputs.from_spectrum(m, n, inputs.sigma_geometric(n, 1e-15), 0))
        else:
            out.append(inputs.kahan(n))
    return out


def time_oracle_sample(mats, parallel: bool = False) -> tuple[float, float]:
    """(seconds, metric flops) of the CPU oracle on the sample: the plain
    single-threaded build, or (parallel) its OpenMP build on every host core
    (identical results)."""
    from oracle import oracle as orc

    t0 = time.perf_counter()
    fl = 0.0
    for A in mats:
        r = orc.qrdm(A, TAU, DELTA, KMAX, parallel=parallel)
        assert r["status"] == 0
        fl += metric_flops(*A.shape)
    return time.perf_counter() - t0, fl


def time_dgeqp3_sample(mats) -> tuple[float, float]:
    """(seconds, metric flops) of LAPACK's column-pivoting QR (xGEQP3 through
    scipy, its own BLAS threads on the host cores) on the sample: the
    comparator the paper measures QRDM against (Sec. 5)."""
    import scipy.linalg

    t0 = time.perf_counter()
    fl = 0.0
    for A in mats:
        scipy.linalg.qr(A, mode="raw", pivoting=True, check_finite=False)
        fl += metric_flops(*A.shape)
    return time.perf_counter() - t0, fl


def oracle_parallel_available() -> bool:
    from oracle import oracle as orc

    return orc.build_omp() is not None


CPU_SAMPLE_DESC = ("the workload's recipes at half linear size: " +
                   ", ".join(f"{k} {m}x{n}" for k, m, n in CPU_SAMPLE) + f" (tau {TAU}, delta {DELTA}, k_max {KMAX})")


def sample_desc(parallel: bool) -> str:
    kind = ("the oracle's OpenMP build (C, -O2, trailing update on every host core, results identical to the "
            "single-threaded build)" if parallel else "the oracle (single-threaded C, -O2)")
    return f"{kind} on {CPU_SAMPLE_DESC}"


def cpu_config() -> dict:
    return {"workload": "CPU sample: " + CPU_SAMPLE_DESC, "matrices": [f"{k}{m}x{n}" for k, m, n in CPU_SAMPLE],
            "tau": TAU, "delta": DELTA, "k_max": KMAX, "global_batch": len(CPU_SAMPLE), "parallelism": "host cores"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()
        return False

    def summary(self) -> dict:
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(kernel: str):
    """dram bytes per launch from the committed ncu summary, if it still
    matches the kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256") != kernel_source_hash():
        return None
    return rec.get("kernels", {}).get(kernel, {}).get("dram_bytes_per_launch")


def kernel_source_hash() -> str:
    """sha256 of the trailing-update section of the kernel source (the code
    of k_trail_w, k_trail_wreduce and k_trail_update)."""
    with open(os.path.join(ROOT, "paper_2106_03138_gb300", "csrc", "qrdm_kernels.cuh")) as fh:
        src = fh.read()
    a = src.index("// a9: block reflector application")
    b = src.index("// a10/a11: partial norm update")
    return hashlib.sha256(src[a:b].encode()).hexdigest()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks of the default process group (the
    benchmark's step time is the slowest replica's)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gflops(world: int, flops_per_step: float, steps: int, total_ms: float) -> float:
    """Whole-job GFLOP/s: every replica factors the workload once per step;
    the job takes as long as the slowest replica."""
    return world * flops_per_step * steps / (total_ms * 1e-3) / 1e9


def run_reference(args, sample=None) -> int:
    """The oracle timed on the host cores, one bounded CPU sample per step.
    Under torchrun only rank 0 runs; the other ranks exit at once."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    mats = cpu_sample_matrices() if sample is None else sample
    par = oracle_parallel_available()
    cpu = host_cpu()
    for _ in range(args.warmup):
        time_oracle_sample(mats, parallel=par)
    secs, fl = 0.0, 0.0
    for _ in range(args.steps):
        s, f = time_oracle_sample(mats, parallel=par)
        secs += s
        fl += f
    value = fl / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cpu_config(),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cpu["nproc"] if par else 1, "kind": "oracle",
                         "sample": sample_desc(par), **cpu},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(name: str, max_steps: int, precision: int = 0) -> int:
    """One factorization of a named workload matrix (tau, delta, k_max as in
    the benchmark), for capturing kernels under a profiler."""
    import torch

    import paper_2106_03138_gb300 as q
    from paper_2106_03138_gb300 import inputs

    if name.startswith("batch"):
        # the first N matrices of the 2000-matrix batch, one batched launch at
        # the tuning the autotuner picks on the full batch
        count = int(name[len("batch"):])
        ents = inputs.batch_entries(2000, seed=0)[:count]
        mats = [q.colmajor(e.build()) for e in ents]  # host-built: no library linear algebra under a profiler
        plan = q.BatchPlan(mats, KMAX)
        plan.set_tuning(2, 512, 4)
        plan.run(TAU, DELTA)
        res = plan.results()
        print(json.dumps({"profile_case": name, "matrices": count, "status_ok": int((res.status == 0).sum()),
                          "block_steps": int(res.steps.sum()), "tuning": plan.tuning}), flush=True)
        plan.close()
        return 0
    A = inputs.named(name).build()
    dA = q.colmajor(A)
    f = q.factor(dA, TAU, DELTA, KMAX, max_steps=max_steps, precision=precision)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "precision": precision, "m": A.shape[0], "n": A.shape[1], "steps": f.nsteps,
                      "launches": f.launches}), flush=True)
    return 0


def measure_c3(q, inputs, torch, stream, hbm_gbs: float | None = None) -> dict:
    """The mixed-precision workload: 16384 x 16384 with sigma geometric
    1 -> 1e-3 over 8192 values then 1e-14 (numerical rank 8192), generated on
    the GPU; the FP64 form, the FP32-class form on the CUDA cores and the two
    tensor-core forms (3xTF32, split-BF16x3), all stopping at the rank (the
    rank-revealing use), each timed once after one untimed run.  For the
    tensor-core forms a third, profiled run gives the HBM rate of the merged
    update's two passes over the trailing block (W = V^T A22 reads it once,
    A22 -= V W reads and writes it: 8 and 16 bytes per element per step)."""
    import numpy as np

    from paper_2106_03138_gb300 import policy as Pol

    n = 16384
    r = n // 2
    sig = inputs.sigma_gap_geometric(n, r)
    A0 = inputs.from_spectrum_gpu(n, n, sig, 0)
    ws = torch.empty(q.qrdm_workspace_size(n, n, KMAX), dtype=torch.uint8, device=A0.device)
    out = {"workload": "16384x16384, sigma geometric 1->1e-3 over 8192 values then 1e-14; stop at the rank",
           "tau": TAU, "delta": DELTA, "k_max": KMAX,
           "flops_note": "GFLOP/s applies the metric 4mn^2-4n^3/3 to the whole matrix (full-rank equivalent); "
                         "executed_GFLOP/s counts the metric's convention (2x Householder) for the columns "
                         "factored before the stop at the rank"}
    flops = metric_flops(n, n)
    forms = ((0, "fp64"), (1, "mixed_fp32"), (3, "tc_3xtf32"), (2, "tc_bf16x3"))
    for prec, key in forms:
        for rep in range(2):
            dA = A0.clone()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f = q.factor(dA, TAU, DELTA, KMAX, workspace=ws, stream=stream, precision=prec, stop_at_rank=True)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1)
        # rank quality as in the paper (Sec. 5): d_i / sigma_i, d_i the sorted |R_ii|, i < r
        d = torch.sort(torch.diagonal(dA)[:r].abs(), descending=True).values.cpu().numpy()
        ratio = d / sig[:r]
        # and the acceptance measure sigma_min(R11) / sigma_r (inverse iteration,
        # the same start and iteration count for every form)
        smin = float(Pol.smin_r11([dA], [r], iters=80)[0]) / float(sig[r - 1])
        exe = executed_flops(n, n, f.rank)
        out[key] = {"ms": ms, "GFLOP/s": flops / ms / 1e6, "executed_GFLOP/s": exe / ms / 1e6,
                    "executed_columns": f.rank, "rank": f.rank, "rank_colmax": f.rank_colmax,
                    "steps": f.nsteps, "d_over_sigma_min": float(ratio.min()), "d_over_sigma_max": float(ratio.max()),
                    "smin_R11_over_sigma_r": smin}
        if key != "fp64":
            out[key]["quality_vs_fp64"] = smin / out["fp64"]["smin_R11_over_sigma_r"]
        if prec >= 2:
            pr = q.qrdm_profile()
            dA = A0.clone()
            torch.cuda.synchronize()
            f = q.factor(dA, TAU, DELTA, KMAX, workspace=ws, stream=stream, precision=prec, stop_at_rank=True,
                         profile=pr, trace=True)
            torch.cuda.synchronize()
            t = f.trace
            ns = np.asarray(t["ns"], dtype=np.float64)
            kk = np.asarray(t["k"], dtype=np.float64)
            elems = float(np.sum((n - ns) * np.maximum(n - ns - kk, 0.0)))
            kms = {q.KERNEL_NAMES[i]: float(pr.ms[i]) for i in range(len(q.KERNEL_NAMES))}
            w_gbs = 8.0 * elems / (kms["k_tc_w"] * 1e-3) / 1e9
            u_gbs = 16.0 * elems / (kms["k_tc_update"] * 1e-3) / 1e9
            out[key]["merged_update"] = {
                "trailing_elements_over_steps": elems,
                "w_pass_ms": kms["k_tc_w"], "w_pass_GBps": w_gbs,
                "update_pass_ms": kms["k_tc_update"], "update_pass_GBps": u_gbs,
                "subpanel_w_ms": kms["k_trail_w"], "subpanel_update_ms": kms["k_trail_update"],
                "t_build_ms": kms["k_tc_vtv+k_tc_tbuild"], "v_images_ms": kms["k_tc_vimg"],
                "w_sum_ms": kms["k_tc_wsum"], "subpanel_w_reduce_ms": kms["k_trail_wreduce"],
                "hbm_frac_of_measured": {"w_pass": w_gbs / hbm_gbs if hbm_gbs else None,
                                         "update_pass": u_gbs / hbm_gbs if hbm_gbs else None},
                "note": "k_tc_w / k_tc_update: the merged tensor-core passes over the trailing block; the "
                        "subpanel_* entries are the FP64 updates of the panel's own columns; profiled run, "
                        "events around every launch",
                "kernel_ms": {k: round(v, 2) for k, v in kms.items() if v > 0},
            }
        if prec == 1:
            # least squares on the mixed factorization, refined in FP64 on the
            # original matrix: a compatible right-hand side b = A x0
            g = torch.Generator(device=A0.device)
            g.manual_seed(7)
            x0 = torch.randn(n, dtype=torch.float64, device=A0.device, generator=g)
            b = A0 @ x0
            torch.cuda.synchronize()
            e0.record(stream)
            x, res = q.ls_solve(A0, f, b, rank=r, refine=3, stream=stream)
            e1.record(stream)
            e1.synchronize()
            nb = float(torch.linalg.vector_norm(b))
            out["ls_refinement"] = {"rank_used": r, "refine_iters": 3, "ms_incl_residual_norms": e0.elapsed_time(e1),
                                    "residual_over_b": [float(v) / nb for v in res[:, 0]],
                                    "rhs": "b = A x0, x0 ~ N(0,1) (seed 7, torch CUDA generator)"}
            del x, b, x0
        del dA
    out["speedup"] = out["fp64"]["ms"] / out["mixed_fp32"]["ms"]
    out["speedup_vs_fp64"] = {key: out["fp64"]["ms"] / out[key]["ms"] for _, key in forms[1:]}
    del A0, ws
    torch.cuda.empty_cache()
    return out


BATCH_PHASES = ("norms", "argmax_candidates", "gram", "dm_pick", "swaps", "panel", "block_reflector", "downdate")


def measure_c4(q, inputs, torch, stream, fp64_peak_tflops: float, count: int = 2000, reps: int = 3) -> dict:
    """The uneven batch: 2000 matrices, m ~ U[64, 1024], n ~ U[32, m], rank
    ~ U[n/4, n], sigma geometric 1 -> 1e-12 over the rank and 1e-15 below,
    generated on the GPU.  Factored by one persistent launch replayed from a
    CUDA graph (tuning picked by the library's autotuner on this batch), and,
    as the comparator, one qrdm_factor call per matrix (the plain FP64 GPU
    form).  Rank quality on a sample: sigma_min(R11) / sigma_r(A)."""
    import numpy as np

    ents = inputs.batch_entries(count, seed=0)
    t0 = time.perf_counter()
    pristine = [e.build_gpu() for e in ents]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    work = [p.clone() for p in pristine]
    flops = sum(metric_flops(e.m, e.n) for e in ents)
    out = {"workload": f"{count} matrices, m~U[64,1024], n~U[32,m], rank~U[n/4,n], sigma geometric 1->1e-12 "
                       "over the rank then 1e-15 (seed 0)", "tau": TAU, "delta": DELTA, "k_max": KMAX,
           "metric_gflop": flops / 1e9, "generate_s": gen_s,
           "l2": "inputs (%.1f GB) larger than L2; restored from device copies untimed" %
                 (sum(e.m * e.n for e in ents) * 8 / 1e9)}

    def restore():
        for w, p0 in zip(work, pristine):
            w.copy_(p0)

    plan = q.BatchPlan(work, KMAX, stream=stream)
    best, tune_ms = plan.autotune(TAU, DELTA, stream=stream)
    out["tuning"] = best
    out["autotune_best_ms"] = tune_ms

    def timed(graph: bool) -> float:
        restore()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.run(TAU, DELTA, graph=graph, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    timed(True)  # capture + first replay
    g_ms = [timed(True) for _ in range(reps)]
    d_ms = timed(False)
    ms = statistics.median(g_ms)
    res = plan.results(stream=stream)
    out["batched"] = {"ms": ms, "ms_runs": g_ms, "GFLOP/s": flops / ms / 1e6, "direct_launch_ms": d_ms,
                      "launches": 1, "status_ok": int((res.status == 0).sum()), "block_steps": int(res.steps.sum()),
                      "fp64_frac_of_derived_peak": (flops / 2) / (ms * 1e-3) / 1e12 / fp64_peak_tflops}
    # phase split of one profiled run
    restore()
    pr = q.qrdm_profile()
    plan.run(TAU, DELTA, q.make_opts(profile=pr), stream=stream)
    out["batched"]["phase_ms"] = {k: round(pr.ms[i], 2) for i, k in enumerate(BATCH_PHASES)}
    out["batched"]["cta_balance"] = pr.flops[0]
    sample = sorted(range(count), key=lambda i: ents[i].m * ents[i].n * min(ents[i].m, ents[i].n), reverse=True)[:4]
    sample += list(range(12))
    Rb = {i: work[i].clone() for i in sample}
    rank_b = {i: int(res.rank_colmax[i]) for i in sample}
    # plain FP64 GPU QRDM, one qrdm_factor call per matrix
    restore()
    mmax = max(e.m for e in ents)
    nmax = max(e.n for e in ents)
    ws = torch.empty(q.qrdm_workspace_size(mmax, nmax, KMAX), dtype=torch.uint8, device=work[0].device)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plain_info = {}
    for i, A in enumerate(work):
        f = q.factor(A, TAU, DELTA, KMAX, workspace=ws, stream=stream)
        if i in Rb:
            plain_info[i] = f.rank_colmax
    e1.record(stream)
    e1.synchronize()
    pms = e0.elapsed_time(e1)
    out["plain_fp64_per_matrix"] = {"ms": pms, "GFLOP/s": flops / pms / 1e6, "launch": "one qrdm_factor per matrix"}
    out["speedup_vs_plain"] = pms / ms
    # rank quality, sigma_min(R11) / sigma_r over the spectrum's rank r
    qual = []
    for i in sample:
        e = ents[i]
        r = e.rank
        sr = float(e.sigma()[r - 1])
        rb = np.triu(Rb[i][:r, :r].cpu().numpy())
        rp = np.triu(work[i][:r, :r].cpu().numpy())
        qb = float(np.linalg.svd(rb, compute_uv=False)[-1]) / sr
        qp = float(np.linalg.svd(rp, compute_uv=False)[-1]) / sr
        qual.append({"m": e.m, "n": e.n, "r": r, "batched": qb, "plain": qp,
                     "rank_colmax_batched": rank_b[i], "rank_colmax_plain": plain_info[i]})
    out["rank_quality_sample"] = {
        "matrices": len(qual), "min_ratio_batched_over_plain": min(x["batched"] / x["plain"] for x in qual),
        "min_sigma_ratio_batched": min(x["batched"] for x in qual),
        "min_sigma_ratio_plain": min(x["plain"] for x in qual),
        "rank_colmax_equal": sum(x["rank_colmax_batched"] == x["rank_colmax_plain"] for x in qual)}
    plan.close()
    del pristine, work, ws, Rb
    torch.cuda.empty_cache()
    return out


def measure_c5(q, torch, stream, n_train: int = 150, n_held: int = 60, big: int = 4096) -> dict:
    """The learned per-step (tau, delta): plain-QRDM (tau, delta) sweeps of
    generated training matrices label the steps, the MLP is trained by the
    library's kernels, then held-out matrices are factored with the policy
    and with fixed (0.9, 0.9) (and the paper's (0.15, 0.9) for context):
    block steps, time and rank quality."""
    import numpy as np

    from paper_2106_03138_gb300 import inputs
    from paper_2106_03138_gb300 import policy as P

    out = {"grid_tau": list(P.GRID_TAU), "grid_delta": list(P.GRID_DELTA), "rho_min": P.RHO_MIN,
           "label_quality_factor": P.QUALITY_FACTOR,
           "quality": "sigma_min(R11)/sigma_r by inverse power iteration on R11 (two triangular solves per step)",
           "tau_range": list(P.TAU_RANGE), "delta_range": list(P.DELTA_RANGE)}
    t0 = time.perf_counter()
    train = P.training_entries(n_train, seed=21, n_lo=64, n_hi=512)
    pristine = [e.build_gpu() for e in train]
    X, T, info = P.collect(train, pristine)
    t1 = time.perf_counter()
    pol = P.Policy(seed=2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    loss = pol.train(X, T, steps=2000, batch=1024, lr=2e-3)
    e1.record()
    e1.synchronize()
    out["training"] = {"matrices": n_train, "n_range": [64, 512], "samples": int(X.shape[0]),
                       "label_counts": info["label_counts"], "sweep_and_label_s": t1 - t0,
                       "train_steps": 2000, "batch": 1024, "train_ms": e0.elapsed_time(e1),
                       "loss_first50": float(loss[:50].mean()), "loss_last50": float(loss[-50:].mean())}
    del pristine
    held = P.training_entries(n_held, seed=99, n_lo=64, n_hi=512)
    hp = [e.build_gpu() for e in held]
    runs = {"fixed_0.9_0.9": P.run_batch(hp, held, 0.9, 0.9), "fixed_0.15_0.9": P.run_batch(hp, held, 0.15, 0.9),
            "learned": P.run_batch(hp, held, 0.9, 0.9, policy=pol)}
    ref = runs["fixed_0.9_0.9"]
    flops = sum(metric_flops(e.n, e.n) for e in held)
    bat = {}
    for k, r in runs.items():
        ratio = r.smin / np.maximum(ref.smin, 1e-300)
        dratio = r.quality / np.maximum(ref.quality, 1e-300)
        bat[k] = {"block_steps": int(r.steps.sum()), "kernel_ms": r.ms, "GFLOP/s": flops / r.ms / 1e6,
                  "smin_ratio_vs_fixed_0.9_min": float(ratio.min()),
                  "smin_ratio_vs_fixed_0.9_median": float(np.median(ratio)),
                  "smin_within_2x": float(np.mean(ratio >= 0.5)),
                  "min_Rii_over_sigma_ratio_median": float(np.median(dratio))}
    out["held_out_batch"] = {"matrices": n_held, "n_range": [64, 512], "batched_kernel": bat}
    del hp
    # one held-out large matrix through the single-matrix path
    n = big
    r = 3 * n // 4
    sig = inputs.sigma_rank_geometric(n, r)
    A0 = inputs.from_spectrum_gpu(n, n, sig, 1000)
    ws = torch.empty(q.qrdm_workspace_size(n, n, KMAX), dtype=torch.uint8, device=A0.device)
    single = {}
    for key, kw in (("fixed_0.9_0.9", {}), ("learned", {"policy": pol.struct()})):
        for rep in range(2):
            dA = A0.clone()
            torch.cuda.synchronize()
            e0.record(stream)
            f = q.factor(dA, 0.9, 0.9, KMAX, workspace=ws, stream=stream, **kw)
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1)
        smin = float(P.smin_r11([dA], [r], iters=60)[0])
        d = torch.diagonal(dA)[:r].abs().cpu().numpy()
        single[key] = {"ms": ms, "GFLOP/s": metric_flops(n, n) / ms / 1e6, "block_steps": f.nsteps,
                       "rank": f.rank, "rank_colmax": f.rank_colmax, "sigma_min_R11_over_sigma_r": smin / sig[r - 1],
                       "min_Rii_over_sigma_i": float(np.min(d / sig[:r]))}
        del dA
    single["speedup"] = single["fixed_0.9_0.9"]["ms"] / single["learned"]["ms"]
    single["quality_ratio"] = (single["learned"]["sigma_min_R11_over_sigma_r"] /
                               single["fixed_0.9_0.9"]["sigma_min_R11_over_sigma_r"])
    out["held_out_single"] = {"matrix": f"{n}x{n}, sigma geometric 1->1e-12 over {r} values then 1e-15, seed 1000",
                              "k_max": KMAX, **single}
    del A0
    # the policy trained at scale (paper_2106_03138_gb300/train_policy.py; weights stored beside it), on
    # the held-out 4096^2 seeds 1000..1009 against fixed (0.9, 0.9); quality sigma_min(R11) / sigma_r
    # with sigma_min exact (singular values of the r x r block)
    wpath = os.path.join(ROOT, "paper_2106_03138_gb300", "policy_weights.npz")
    if os.path.exists(wpath):
        big = P.Policy.load(wpath)
        with np.load(wpath) as z:
            tsum = json.loads(str(z["summary"]))
        rows = []
        for sd in range(1000, 1010):
            A0 = inputs.from_spectrum_gpu(n, n, sig, sd)
            res = {}
            for key, kw in (("fixed_0.9_0.9", {}), ("learned", {"policy": big.struct()})):
                for rep in range(2):
                    dA = A0.clone()
                    torch.cuda.synchronize()
                    e0.record(stream)
                    f = q.factor(dA, 0.9, 0.9, KMAX, workspace=ws, stream=stream, **kw)
                    e1.record(stream)
                    e1.synchronize()
                ms = e0.elapsed_time(e1)
                smin = float(torch.linalg.svdvals(torch.triu(dA[:r, :r]))[-1])
                res[key] = {"ms": ms, "block_steps": f.nsteps, "quality": smin / float(sig[r - 1])}
                del dA
            rows.append({"seed": sd, **res, "speedup": res["fixed_0.9_0.9"]["ms"] / res["learned"]["ms"],
                         "quality_ratio": res["learned"]["quality"] / res["fixed_0.9_0.9"]["quality"]})
            del A0
        sp = np.array([x["speedup"] for x in rows])
        qr = np.array([x["quality_ratio"] for x in rows])
        out["held_out_seeds"] = {
            "matrix": f"{n}x{n}, sigma geometric 1->1e-12 over {r} values then 1e-15, seeds 1000..1009",
            "weights": "paper_2106_03138_gb300/policy_weights.npz", "training": tsum, "seeds": len(rows),
            "speedup_median": float(np.median(sp)), "speedup_min": float(sp.min()),
            "quality_ratio_median": float(np.median(qr)), "quality_ratio_min": float(qr.min()),
            "within_2x": int(np.sum(qr >= 0.5)), "per_seed": rows,
            "quality": "sigma_min(R11)/sigma_r, sigma_min exact (torch.linalg.svdvals of the r x r block)"}
    del ws
    torch.cuda.empty_cache()
    return out


def forms_summary(c3, c4, c5) -> dict:
    """The forms of the metric's comparison "vs plain FP64 GPU QRDM at equal
    rank quality", compactly: the 16384^2 mixed-precision forms, the batched
    form and the learned (tau, delta), each against its plain FP64 GPU
    comparator."""
    out = {}
    if c3:
        f3 = {}
        for key in ("fp64", "mixed_fp32", "tc_3xtf32", "tc_bf16x3"):
            r = c3.get(key)
            if r:
                f3[key] = {"ms": round(r["ms"], 1), "speedup": round(c3["fp64"]["ms"] / r["ms"], 2),
                           "executed_GFLOP/s": round(r["executed_GFLOP/s"], 1),
                           "smin_R11_over_sigma_r": r.get("smin_R11_over_sigma_r"),
                           "quality_vs_fp64": r.get("quality_vs_fp64"), "rank_colmax": r["rank_colmax"]}
        out["c3_16384_gap"] = f3
    if c4:
        out["c4_batch2000"] = {"batched_ms": round(c4["batched"]["ms"], 1),
                               "plain_ms": round(c4["plain_fp64_per_matrix"]["ms"], 1),
                               "speedup": round(c4["speedup_vs_plain"], 2),
                               "quality_min_ratio": c4["rank_quality_sample"]["min_ratio_batched_over_plain"]}
    if c5:
        hs = c5.get("held_out_seeds")
        if hs:
            out["c5_learned_4096"] = {"seeds": hs["seeds"], "speedup_median": hs["speedup_median"],
                                      "speedup_min": hs["speedup_min"], "quality_ratio_min": hs["quality_ratio_min"],
                                      "quality_ratio_median": hs["quality_ratio_median"]}
        else:
            hsn = c5["held_out_single"]
            out["c5_learned_4096"] = {"speedup": round(hsn["speedup"], 3),
                                      "quality_ratio": round(hsn["quality_ratio"], 3)}
    return out


def run_fp64_probe() -> int:
    """The FP64 rates of this GPU (FFMA64 chains, DMMA mma.sync m8n8k4, and a
    cuBLAS DGEMM through torch), with the SM clocks sampled meanwhile: the
    measured counterpart of the derived FP64 peak the roofline divides by."""
    import torch

    import paper_2106_03138_gb300 as q
    from paper_2106_03138_gb300 import _binding as b

    q.load()
    dev = torch.device("cuda", 0)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    res = {}
    with ClockSampler(0) as clk:
        for which, name, iters in ((0, "ffma64", 200000), (1, "dmma_m8n8k4", 50000)):
            b.qrdm_fp64_probe(which, blocks, max(1, iters // 20), out.data_ptr(), out.numel() * 8, stream)  # warm
            best = None
            for _ in range(3):
                rc, fl, ms = b.qrdm_fp64_probe(which, blocks, iters, out.data_ptr(), out.numel() * 8, stream)
                assert rc == 0, rc
                best = ms if best is None else min(best, ms)
            res[name] = {"TFLOP/s": fl / (best * 1e-3) / 1e12, "ms": best, "blocks": blocks, "iters": iters}
        n = 8192
        x = torch.randn(n, n, dtype=torch.float64, device=dev)
        y = torch.randn(n, n, dtype=torch.float64, device=dev)
        torch.matmul(x, y)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(x, y)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        res["cublas_dgemm_8192"] = {"TFLOP/s": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "ms": best}
    csum = clk.summary()
    smax = csum.get("sm_max_mhz") or 2070.0
    derived = FP64_FLOP_PER_CLK_PER_SM * sms * smax * 1e6 / 1e12
    print(json.dumps({"fp64_probe": res, "derived_peak_TFLOP/s": derived,
                      "derived_peak": f"{FP64_FLOP_PER_CLK_PER_SM:g} flop/clk/SM x {sms} SMs x {smax:g} MHz",
                      "clocks": csum, "gpu": props.name}), flush=True)
    return 0


def config_dict(world: int) -> dict:
    return {"workload": WORKLOAD_DESC, "matrices": list(WORKLOAD), "tau": TAU, "delta": DELTA, "k_max": KMAX,
            "global_batch": 3 * world, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "flushed (256 MB write) before every timed step; inputs restored from device copies untimed"}


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="skip the 16384^2 mixed-precision measurement")
    ap.add_argument("--no-c4", action="store_true", help="skip the 2000-matrix batched measurement")
    ap.add_argument("--no-c5", action="store_true", help="skip the learned (tau, delta) training and evaluation")
    ap.add_argument("--profile-case", default=None,
                    help="factor one named matrix once at the benchmark's parameters and exit (profiler target)")
    ap.add_argument("--max-steps", type=int, default=0, help="with --profile-case: stop after this many block steps")
    ap.add_argument("--precision", type=int, default=0, help="with --profile-case: 0 FP64, 1 FP32-class mixed")
    ap.add_argument("--fp64-probe", action="store_true", help="measure this GPU's FP64 rates and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.fp64_probe:
        return run_fp64_probe()
    if args.profile_case:
        return run_profile_case(args.profile_case, args.max_steps, args.precision)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2106_03138_gb300 as q
    from paper_2106_03138_gb300 import inputs

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    q.load()

    specs = [inputs.named(nm) for nm in WORKLOAD]
    host = [s.build() for s in specs]
    shapes = [a.shape for a in host]
    flops_step = sum(metric_flops(m, n) for m, n in shapes)
    pristine = [q.colmajor(a, device=dev) for a in host]
    work = [p.clone() for p in pristine]
    wsz = max(q.qrdm_workspace_size(m, n, KMAX) for m, n in shapes)
    ws = torch.empty(wsz, dtype=torch.uint8, device=dev)
    htau = [torch.empty(min(m, n), dtype=torch.float64, device=dev) for m, n in shapes]
    perm = [torch.empty(n, dtype=torch.int32, device=dev) for m, n in shapes]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def restore():
        for w, p in zip(work, pristine):
            w.copy_(p)
        flush.fill_(1.0)

    def step(profile=None):
        launches = 0
        infos = []
        for i in range(len(work)):
            f = q.factor(work[i], TAU, DELTA, KMAX, workspace=ws, out_htau=htau[i], out_perm=perm[i], stream=stream,
                         profile=profile)
            launches += f.launches
            infos.append(f)
        return launches, infos

    for _ in range(args.warmup):
        restore()
        step()
    torch.cuda.synchronize()

    step_ms = []
    launches = 0
    infos = None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")
        for _ in range(args.steps):
            restore()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nl, infos = step()
            e1.record(stream)
            e1.synchronize()
            launches += nl
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(step_ms), device=dev)
    value = aggregate_gflops(world, flops_step, args.steps, total_ms)

    # kernel durations: a second timed pass over the same steps with CUDA
    # events around every launch (the events add host work between launches,
    # not device time to a kernel), kept apart from the headline value
    prof = q.qrdm_profile()
    prof_steps = max(1, min(args.steps, 2))
    prof_ms = 0.0
    for _ in range(prof_steps):
        restore()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(prof)
        e1.record(stream)
        e1.synchronize()
        prof_ms += e0.elapsed_time(e1)

    # dominant kernel and its roofline (FP64 ALU bound)
    ms = list(prof.ms)
    kid = max(range(len(q.KERNEL_NAMES)), key=lambda i: ms[i])
    kname = q.KERNEL_NAMES[kid]
    nlaunch = max(int(prof.launches[kid]), 1)
    achieved = (prof.flops[kid] / nlaunch) / (ms[kid] / nlaunch * 1e-3) / 1e12 if ms[kid] > 0 else 0.0
    csum = clk.summary()
    sm_max = csum.get("sm_max_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    peak = FP64_FLOP_PER_CLK_PER_SM * props.multi_processor_count * sm_max * 1e6 / 1e12
    total_kernel_ms = sum(ms)
    roofline = {
        "bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
        "frac": achieved / peak if peak else None, "traffic": traffic_for(kname),
        "peak_source": "FP64 FMA rate 2/clk/SM x 152 SMs x sm_max_mhz (derived; nominal 1.25 TFLOP/s)",
        "share_of_kernel_time": ms[kid] / total_kernel_ms if total_kernel_ms else None,
        "launches_timed": nlaunch, "profiled_steps": prof_steps,
        "profiled_ms_per_step": prof_ms / prof_steps,
        "kernel_ms_per_step": {q.KERNEL_NAMES[i]: round(ms[i] / prof_steps, 3) for i in range(len(q.KERNEL_NAMES))},
    }

    # end to end through the public API with host buffers (pinned)
    # pinned host buffers hold A^T in row-major order, i.e. A column-major
    pin_in = []
    for a in host:
        t = torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64).pin_memory()
        t.copy_(torch.from_numpy(np.ascontiguousarray(a.T)))
        pin_in.append(t)
    pin_out = [torch.empty_like(p).pin_memory() for p in pin_in]
    pin_ht = [torch.empty(min(m, n), dtype=torch.float64).pin_memory() for m, n in shapes]
    pin_pm = [torch.empty(n, dtype=torch.int32).pin_memory() for m, n in shapes]
    h2d = sum(p.numel() * 8 for p in pin_in)
    d2h = sum(p.numel() * 8 for p in pin_in) + sum(h.numel() * 8 for h in pin_ht) + sum(p.numel() * 4 for p in pin_pm)
    e2e_steps = max(1, min(args.steps, 3))
    e2e_ms = 0.0
    for _ in range(e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(len(work)):
            # host -> device: the column-major input into the work buffer
            work[i].t().copy_(pin_in[i], non_blocking=True)
            q.factor(work[i], TAU, DELTA, KMAX, workspace=ws, out_htau=htau[i], out_perm=perm[i], stream=stream)
            pin_out[i].copy_(work[i].t(), non_blocking=True)
            pin_ht[i].copy_(htau[i], non_blocking=True)
            pin_pm[i].copy_(perm[i], non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_value = aggregate_gflops(world, flops_step, e2e_steps, max_over_ranks(e2e_ms, device=dev))

    comparators = {}
    if not args.no_comparators and rank == 0:
        for label, tau, delta, kmax in (("qrp_kmax1", 0.9, 0.9, 1), ("tau0.9_delta0.9_kmax32", 0.9, 0.9, 32)):
            wk = pristine[0].clone()
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f = q.factor(wk, tau, delta, kmax, workspace=ws, stream=stream)
            e1.record(stream)
            e1.synchronize()
            msc = e0.elapsed_time(e1)
            m, n = shapes[0]
            comparators[label] = {"matrix": WORKLOAD[0], "ms": msc, "GFLOP/s": metric_flops(m, n) / msc / 1e6,
                                  "steps": f.nsteps, "rank": f.rank}
            del wk
        # blocked column pivoting with lazy updates (the xGEQP3 scheme), nb = 16
        qws = None
        for rep in range(2):
            wk = pristine[0].clone()
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f = q.qp3_factor(wk, 16, workspace=qws, stream=stream)
            e1.record(stream)
            e1.synchronize()
        msc = e0.elapsed_time(e1)
        m, n = shapes[0]
        comparators["qp3_lazy_nb16"] = {"matrix": WORKLOAD[0], "ms": msc, "GFLOP/s": metric_flops(m, n) / msc / 1e6,
                                        "blocks": f.nsteps, "rank": f.rank}
        del wk

    c3 = None
    if rank == 0 and not args.no_c3:
        hbm = None
        try:
            with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fp:
                hbm = float(json.load(fp)["hbm_gbs"])
        except (OSError, KeyError, ValueError):
            hbm = 6800.0  # fallback copy bandwidth of a GB300 (GB/s)
        c3 = measure_c3(q, inputs, torch, stream, hbm)

    c4 = None
    if rank == 0 and not args.no_c4:
        c4 = measure_c4(q, inputs, torch, stream, peak)

    c5 = None
    if rank == 0 and not args.no_c5:
        c5 = measure_c5(q, torch, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        mats = cpu_sample_matrices()
        host = host_cpu()
        secs1, fl = time_oracle_sample(mats)
        single = {"value": fl / secs1 / 1e9, "cores": 1, "seconds": secs1, "sample": sample_desc(False)}
        if oracle_parallel_available():
            secs, fl = time_oracle_sample(mats, parallel=True)
            cpu = {"value": fl / secs / 1e9, "unit": "GFLOP/s", "cores": host["nproc"], "kind": "oracle",
                   "sample": sample_desc(True), "seconds": secs, **host, "single_thread": single}
        else:
            cpu = {"value": single["value"], "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                   "sample": single["sample"], "seconds": secs1, **host,
                   "all_cores": "unavailable: the C compiler has no OpenMP"}
        try:
            secs_q, fl_q = time_dgeqp3_sample(mats)
            cpu["lapack_dgeqp3"] = {"value": fl_q / secs_q / 1e9, "unit": "GFLOP/s", "seconds": secs_q,
                                    "what": "scipy.linalg.qr(pivoting=True), LAPACK xGEQP3 with the host BLAS "
                                            "threads, same sample, metric flops (4mn^2-4n^3/3)"}
        except Exception as exc:  # noqa: BLE001 - context only
            cpu["lapack_dgeqp3"] = {"unavailable": str(exc)[:200]}

    if rank == 0:
        per = [{"matrix": nm, "m": m, "n": n, "rank": f.rank, "rank_colmax": f.rank_colmax, "steps": f.nsteps}
               for nm, (m, n), f in zip(WORKLOAD, shapes, infos)]
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            # the same rate by LAPACK's xGEQRF count 2mn^2 - 2n^3/3, half the metric's
            "value_lapack_count": value / 2.0,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(world), "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": csum, "gpu_launches": launches, "wall_s": t_wall, "per_matrix": per,
            "comparators": comparators, "mixed_precision_c3": c3, "batched_c4": c4, "learned_c5": c5,
            "forms": forms_summary(c3, c4, c5),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
