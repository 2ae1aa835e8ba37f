"""The FP32-class mixed-precision form (precision=1): trailing update and
candidate Gram matrix in FP32 from FP64 storage, panel, norms and rank in
FP64.  Its results are not expected to match the FP64 oracle digit for digit,
so each case reports its error against the oracle and checks the bounds of
this precision class and the rank quality the FP64 form reaches:

  ||A Pi - Q R|| / ||A|| <= 1e-5 (FP32 roundoff accumulated over the updates),
  ||Q^T Q - I|| <= 1e-13 (the reflectors themselves are FP64),
  the precision-aware criterion finds the gap rank,
  sigma_min(R11) / sigma_r(A) within 2x of the plain FP64 form (the north
  star's acceptance for the variants)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._helpers import factorization_errors, upper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402

CASES = [
    # name, m, n, sigma builder, numerical rank (gap position)
    ("gapgeo1024", 1024, 1024, lambda p: inputs.sigma_gap_geometric(p, 512), 512),
    ("gapgeo2048x1024", 2048, 1024, lambda p: inputs.sigma_gap_geometric(p, 600), 600),
    ("gap768", 768, 768, lambda p: inputs.sigma_gap(p, 300), 300),
]


def _gpu(A, precision):
    dA = q.colmajor(A)
    f = q.factor(dA, 0.15, 0.9, 64, precision=precision, trace=True)
    torch.cuda.synchronize()
    return dA.cpu().numpy(), f.htau.cpu().numpy(), f.perm.cpu().numpy().astype(np.int64), f


@pytest.mark.parametrize("name,m,n,sig,r", CASES, ids=[c[0] for c in CASES])
def test_mixed_precision_against_oracle_and_plain(name, m, n, sig, r):
    s = sig(min(m, n))
    A = inputs.from_spectrum(m, n, s, 1234)
    o = O.qrdm(A, 0.15, 0.9, 64)
    A64, h64, p64, f64 = _gpu(A, 0)
    A32, h32, p32, f32 = _gpu(A, 1)
    res32, orth32 = factorization_errors(A, A32, h32, p32)
    res64, orth64 = factorization_errors(A, A64, h64, p64)
    assert res64 <= 1e-13 and orth64 <= 1e-13
    assert res32 <= 1e-5, res32
    assert orth32 <= 1e-13, orth32
    # the precision-aware criterion finds the gap within one block (the test
    # runs at block starts and approaches eps1 ||A|| from below, Sec. 3.4/5)
    assert r <= f32.rank_colmax <= r + 64, (f32.rank, f32.rank_colmax, r)
    assert f32.rank >= f32.rank_colmax
    # rank quality against the plain FP64 form
    s11_32 = np.linalg.svd(upper(A32)[:r, :r], compute_uv=False)[-1]
    s11_64 = np.linalg.svd(upper(A64)[:r, :r], compute_uv=False)[-1]
    q32, q64 = s11_32 / s[r - 1], s11_64 / s[r - 1]
    assert q32 >= 0.5 * q64, (q32, q64)
    # per-result error: R of the mixed form against the FP64 R of the same
    # permuted matrix A Pi_32 (a library QR, rows normalized to |R|)
    R32 = upper(A32)
    Rref = np.linalg.qr(A[:, p32], mode="r")[: min(m, n)]
    anorm = np.linalg.norm(A, 2)
    err_R = float(np.max(np.abs(np.abs(R32) - np.abs(Rref)))) / anorm
    d32, dref = np.abs(np.diag(R32))[:r], np.abs(np.diag(Rref))[:r]
    rel = float(np.max(np.abs(d32 - dref) / dref))
    same = 0
    for st in range(min(len(f32.trace), len(o["trace"]))):
        if f32.trace["k"][st] != o["trace"]["k"][st] or f32.trace["l"][st] != o["trace"]["l"][st]:
            break
        same += 1
    print(f"\n[mixed] {name}: residual {res32:.2e} (fp64 {res64:.2e}), orth {orth32:.1e}, "
          f"rank {f32.rank}/{f32.rank_colmax} (oracle {o['rank']}/{o['rank_colmax']}, gap {r}), "
          f"sigma_min(R11)/sigma_r {q32:.3f} (fp64 {q64:.3f}), max |R - R64(A Pi)| / ||A|| {err_R:.2e}, "
          f"max rel err |R_ii| (i < r) {rel:.2e}, steps identical to the oracle {same}")
    assert err_R <= 1e-5
    assert rel <= 1e-3
