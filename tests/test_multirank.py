"""The N > 1 path of bench.py is replicas only (the factorization does not
shard): each rank factors its own copy of the workload, the job's time is the
slowest rank's, and the value is the whole job's throughput.  This host-side
logic runs here as two gloo ranks on the CPU."""
from __future__ import annotations

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank step times: the job time is the slowest rank's
        mine = 100.0 + 37.5 * rank
        tmax = bench.max_over_ranks(mine)
        val = bench.aggregate_gflops(world, 1e9, 4, tmax)
        # the reference arm: only rank 0 prints, the others return 0 at once
        from paper_2106_03138_gb300 import inputs

        args = type("A", (), {"gpus": world, "steps": 1, "warmup": 0})()
        buf = io.StringIO()
        with redirect_stdout(buf):
            rc = bench.run_reference(args, sample=[inputs.random_dense(24, 16, rank)])
        dist.barrier()
        q.put((rank, tmax, val, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, tmax, val, rc, text in out:
        assert tmax == pytest.approx(137.5)
        # 2 replicas x 4 steps x 1 GFLOP in 137.5 ms
        assert val == pytest.approx(2 * 4 * 1e9 / 0.1375 / 1e9)
        assert rc == 0
        if rank == 0:
            line = json.loads(text.strip())
            assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
            assert np.isfinite(line["value"]) and line["value"] > 0
            # the base contract's keys, with this arm's own config and an
            # e2e that moves no bytes between host and device
            for key, typ in (("metric", str), ("unit", str), ("n_gpus", int), ("steps", int), ("warmup", int),
                             ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                             ("dtype", str), ("data", str), ("config", dict), ("e2e", dict)):
                assert isinstance(line[key], typ), key
            assert line["n_gpus"] == world and line["higher_is_better"] is True and line["vs_baseline"] is None
            assert line["dtype"] == "f64" and line["config"]["workload"].startswith("CPU sample")
            assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                                   "d2h_bytes_per_step": 0}
            cb = line["cpu_baseline"]
            assert cb["value"] == line["value"] and isinstance(cb["cores"], int) and cb["cores"] >= 1
            assert isinstance(cb["sample"], str) and cb["nproc"] >= cb["cores"]
        else:
            assert text == ""


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.aggregate_gflops(1, 2e9, 2, 1000.0) == pytest.approx(4.0)
    assert bench.metric_flops(4096, 4096) == pytest.approx(4 * 4096 ** 3 - 4 * 4096 ** 3 / 3)
    # the metric is twice LAPACK's xGEQRF count 2 m n^2 - 2 n^3 / 3
    assert bench.metric_flops(8192, 2048) == pytest.approx(2 * (2 * 8192 * 2048 ** 2 - 2 * 2048 ** 3 / 3))
    # the count up to a stop after r columns: all of it at r = n, and within
    # O(1/r) of twice the Householder sum 4 (m - i)(n - i) over i < r
    for m, n in ((4096, 4096), (8192, 2048), (16384, 16384)):
        assert bench.executed_flops(m, n, n) == pytest.approx(bench.metric_flops(m, n), rel=1e-12)
        for r in (64, n // 2, n):
            i = np.arange(r, dtype=np.float64)
            exact = 2.0 * float(np.sum(4.0 * (m - i) * (n - i)))
            assert bench.executed_flops(m, n, r) == pytest.approx(exact, rel=2.0 / r)
    assert bench.executed_flops(100, 50, 0) == 0.0
