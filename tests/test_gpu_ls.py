"""Least squares on a QRDM factorization (qrdm_ls_solve) against the oracle's
basic solution, and FP64 iterative refinement of the FP32-class
factorization back to FP64 accuracy."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402


def _factor(A, precision=0, **kw):
    dA = q.colmajor(A)
    f = q.factor(dA, 0.15, 0.9, 64, precision=precision, **kw)
    torch.cuda.synchronize()
    return f


@pytest.mark.parametrize("m,n,r,nrhs", [(300, 300, 300, 1), (500, 200, 200, 3), (400, 300, 120, 2),
                                         (257, 129, 129, 5)])
def test_fp64_basic_solution_matches_the_oracle(m, n, r, nrhs):
    sig = inputs.sigma_gap(min(m, n), r, lo=1e-15) if r < min(m, n) else np.geomspace(1.0, 1e-3, min(m, n))
    A = inputs.from_spectrum(m, n, sig, 31 + m)
    B = np.random.default_rng(m + n).standard_normal((m, nrhs))
    f = _factor(A)
    X, _ = q.ls_solve(None, f, torch.as_tensor(B, device="cuda"), rank=r)
    o = O.qrdm(A, 0.15, 0.9, 64)
    xo = O.ls_basic(A, B, rank=r, fact=o).reshape(n, nrhs)
    xg = X.cpu().numpy().reshape(n, nrhs)
    cond = sig[0] / sig[r - 1]
    tol = 100 * np.sqrt(m * n) * cond * 2.0 ** -52 * np.abs(xo).max()
    same_cols = np.array_equal(np.sort(o["perm"][:r]), np.sort(f.perm.cpu().numpy()[:r]))
    if r == n or same_cols:
        # the same basic solution (unique when r = n) from two backward-stable programs
        assert np.max(np.abs(xg - xo)) <= tol, (np.max(np.abs(xg - xo)), tol)
    else:  # a tie chose other columns: both must be basic least-squares solutions
        assert np.count_nonzero(np.abs(xg).sum(axis=1)) <= r
    rg = np.linalg.norm(A @ xg - B, axis=0)
    ro = np.linalg.norm(A @ xo - B, axis=0)
    np.testing.assert_allclose(rg, ro, rtol=1e-10, atol=1e-12 * np.linalg.norm(B))


def test_refinement_recovers_fp64_accuracy_from_the_fp32_class_factorization():
    m, n = 1536, 1024
    sig = np.geomspace(1.0, 1e-3, n)  # full rank, cond 1e3
    A = inputs.from_spectrum(m, n, sig, 5)
    x0 = np.random.default_rng(9).standard_normal(n)
    b = A @ x0  # compatible system
    A_orig = q.colmajor(A)
    f32 = _factor(A, precision=1)
    assert f32.rank == n
    X, res = q.ls_solve(A_orig, f32, torch.as_tensor(b, device="cuda"), refine=6)
    x = X.cpu().numpy()
    nb = np.linalg.norm(b)
    print("\n[ls] residual ||b - A x_k|| / ||b||:", (res[:, 0] / nb).tolist())
    assert res[0, 0] / nb > 1e-9  # the unrefined mixed solution is FP32-accurate only
    assert res[-1, 0] / nb <= 1e-14
    assert np.linalg.norm(x - x0) / np.linalg.norm(x0) <= 1e-12
    # the residual norms the library reports are the host's
    assert res[-1, 0] == pytest.approx(np.linalg.norm(b - A @ x), rel=1e-6, abs=1e-14 * nb)


def test_rank_deficient_compatible_system():
    m, n, r = 600, 400, 150
    A = inputs.from_spectrum(m, n, inputs.sigma_gap(n, r, lo=1e-15), 12)
    x0 = np.random.default_rng(2).standard_normal(n)
    b = A @ x0
    f = _factor(A, precision=1)
    X, res = q.ls_solve(q.colmajor(A), f, torch.as_tensor(b, device="cuda"), rank=r, refine=4)
    x = X.cpu().numpy()
    assert np.count_nonzero(x) <= r
    assert np.linalg.norm(A @ x - b) <= 1e-13 * np.linalg.norm(b)
