"""Failure detection on the GPU without a GPU fault.

Every device-side wait of the library is bounded (opts.wait_limit_us).  The
test hooks of opts.test_fault make one wait wait for something that never
happens (an arrival nobody makes, an mbarrier nobody arrives on); the wait
must run out, every CTA must leave, the call must return QRDM_ERR_TIMEOUT
with the record of where, and the next call must work.  The checked path
(opts.checked) must give results identical to the unchecked one, and refuse
a planted out-of-range column index before using it (QRDM_ERR_CHECKED).
Nothing here traps, asserts on the device, touches a bad address or spins
without a limit."""
from __future__ import annotations

import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._helpers import factorization_errors
from tests._parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402

QRDM_K_PICK = 4
QRDM_K_TC_UPDATE = 17


def _gpu_dict(dA, f):
    return {"A": dA.cpu().numpy(), "htau": f.htau.cpu().numpy(), "perm": f.perm.cpu().numpy().astype(np.int64),
            "trace": f.trace, "J": f.J.astype(np.int64), "rank": f.rank, "rank_colmax": f.rank_colmax}


def test_grid_barrier_wait_runs_out_and_the_next_call_works():
    """k_max = 1 runs in the cooperative single-column kernel; hook 1 makes
    its first grid barrier wait for one arrival more than the grid makes."""
    A = inputs.from_spectrum(300, 200, inputs.sigma_geometric(200, 1e-12), 31)
    dA = q.colmajor(A)
    t0 = time.perf_counter()
    with pytest.raises(q.QRDMError) as ei:
        q.factor(dA, 0.9, 0.9, 1, wait_limit_us=2000, test_fault=1)
    wall = time.perf_counter() - t0
    e = ei.value
    assert e.code == q.QRDM_ERR_TIMEOUT
    assert e.info.fail_code == q.QRDM_FAIL_GRID_BARRIER
    assert e.info.fail_step == 0 and e.info.fail_ns == 0
    assert wall < 30.0
    # the context is usable and the next call starts afresh
    dA = q.colmajor(A)
    f = q.factor(dA, 0.9, 0.9, 1, trace=True)
    torch.cuda.synchronize()
    o = O.qrdm(A, 0.9, 0.9, 1)
    compare(A, _gpu_dict(dA, f), o)


@pytest.mark.parametrize("precision", [2, 3])
def test_tensor_core_update_wait_runs_out_and_frees_its_tensor_memory(precision):
    """Hook 3: the first tile of the tensor-core update waits on an mbarrier
    nobody arrives on.  Every CTA gives up, drains the copies it issued and
    frees its tensor memory; the factorization stops with QRDM_ERR_TIMEOUT.
    The next run (which allocates tensor memory again in every CTA) gives
    the same bits as a run made before the fault."""
    A = inputs.from_spectrum(1024, 512, inputs.sigma_gap_geometric(512, 256), 3)
    ref = q.colmajor(A)
    fr = q.factor(ref, 0.15, 0.9, 64, precision=precision)
    torch.cuda.synchronize()
    dA = q.colmajor(A)
    with pytest.raises(q.QRDMError) as ei:
        q.factor(dA, 0.15, 0.9, 64, precision=precision, wait_limit_us=2000, test_fault=3)
    e = ei.value
    assert e.code == q.QRDM_ERR_TIMEOUT
    assert e.info.fail_code == q.QRDM_FAIL_MMA_WAIT
    assert e.info.fail_value == QRDM_K_TC_UPDATE
    assert e.info.fail_step == 0
    for _ in range(2):
        dA = q.colmajor(A)
        f = q.factor(dA, 0.15, 0.9, 64, precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(dA, ref) and torch.equal(f.perm, fr.perm) and torch.equal(f.htau, fr.htau)


CHECKED_CASES = [
    # (kind, m, n, tau, delta, kmax, precision)
    ("gap", 256, 256, 0.9, 0.9, 32, 0),
    ("geo", 513, 300, 0.15, 0.9, 64, 0),
    ("dense", 90, 333, 0.6, 0.8, 7, 0),
    ("geo", 400, 300, 0.9, 0.9, 1, 0),
    ("gapgeo", 768, 512, 0.15, 0.9, 64, 2),
    ("gapgeo", 768, 512, 0.15, 0.9, 64, 4),
]


def _mat(kind, m, n, seed):
    if kind == "gap":
        return inputs.from_spectrum(m, n, inputs.sigma_gap(min(m, n), min(m, n) // 2), seed)
    if kind == "geo":
        return inputs.from_spectrum(m, n, inputs.sigma_geometric(min(m, n), 1e-14), seed)
    if kind == "gapgeo":
        return inputs.from_spectrum(m, n, inputs.sigma_gap_geometric(min(m, n), min(m, n) // 2), seed)
    return inputs.random_dense(m, n, seed)


@pytest.mark.parametrize("kind,m,n,tau,delta,kmax,precision", CHECKED_CASES)
def test_checked_path_gives_the_unchecked_results(kind, m, n, tau, delta, kmax, precision):
    A = _mat(kind, m, n, 5 + m)
    d0, d1 = q.colmajor(A), q.colmajor(A)
    f0 = q.factor(d0, tau, delta, kmax, precision=precision, trace=True)
    f1 = q.factor(d1, tau, delta, kmax, precision=precision, trace=True, checked=True)
    torch.cuda.synchronize()
    assert torch.equal(d0, d1) and torch.equal(f0.perm, f1.perm) and torch.equal(f0.htau, f1.htau)
    assert (f0.rank, f0.rank_colmax, f0.nsteps) == (f1.rank, f1.rank_colmax, f1.nsteps)
    if precision in (0, 4):
        o = O.qrdm(A, tau, delta, kmax)
        compare(A, _gpu_dict(d1, f1), o)
    res, orth = factorization_errors(A, d1.cpu().numpy(), f1.htau.cpu().numpy(), f1.perm.cpu().numpy())
    assert orth <= 1e-13 and res <= (1e-13 if precision in (0, 4) else 5e-5)


def test_checked_path_refuses_a_planted_column_index():
    """Hook 2 plants a column-move destination one past the last column into
    the first step's move list.  The matrix is the left part of a wider
    allocation, so that index names a guard column the call does not own:
    the checked path must refuse it before any access (the guard stays
    untouched) and return QRDM_ERR_CHECKED with the kernel and the index."""
    m, n = 120, 80
    A = inputs.from_spectrum(m, n, inputs.sigma_geometric(n, 1e-10), 12)
    big = torch.full((m, n + 2), 7.25, dtype=torch.float64, device="cuda").t().contiguous().t()
    big[:, :n] = torch.from_numpy(A).cuda()
    sub = big[:, :n]
    assert sub.stride() == (1, m)
    with pytest.raises(q.QRDMError) as ei:
        q.factor(sub, 0.5, 0.9, 16, checked=True, test_fault=2)
    e = ei.value
    assert e.code == q.QRDM_ERR_CHECKED
    assert e.info.fail_code == q.QRDM_FAIL_CHECK
    assert e.info.fail_cta == QRDM_K_PICK and e.info.fail_value == n
    assert e.info.fail_step == 0
    assert torch.all(big[:, n:] == 7.25)
    # a checked call without the hook goes through and matches the oracle
    sub.copy_(torch.from_numpy(A).cuda())
    f = q.factor(sub, 0.5, 0.9, 16, checked=True, trace=True)
    torch.cuda.synchronize()
    compare(A, _gpu_dict(sub, f), O.qrdm(A, 0.5, 0.9, 16))
    assert torch.all(big[:, n:] == 7.25)
