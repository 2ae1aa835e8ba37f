"""The blocked column-pivoting comparator (qrdm_qp3_factor, lazy updates)
against the CPU oracle at k_max = 1 (column pivoting): the same permutation
until the first step where the oracle logged a near-tie of the argmax or of
the norm-recompute test, |R_ii| and htau within the perturbation bound, a
backward-stable factorization, and the same numerical rank."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._helpers import factorization_errors
from tests._parity import compare_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402


def _first_tie(o) -> int:
    tr = o["trace"]
    sc = np.minimum(tr["s_argmax"], tr["s_recomp"])
    bad = np.nonzero(sc < 1.0)[0]
    return int(tr["ns"][bad[0]]) if bad.size else min(o["A"].shape)


CASES = [
    ("geo", 300, 200, 32), ("geo", 300, 200, 8), ("geo", 300, 200, 1), ("gap", 256, 256, 32),
    ("dense", 300, 257, 32), ("geo", 200, 300, 16), ("kahan", 200, 200, 32), ("geo", 1024, 700, 32),
]


def _mat(kind, m, n, seed=3):
    if kind == "geo":
        return inputs.from_spectrum(m, n, inputs.sigma_geometric(min(m, n), 1e-14), seed)
    if kind == "gap":
        return inputs.from_spectrum(m, n, inputs.sigma_gap(min(m, n), min(m, n) // 2), seed)
    if kind == "kahan":
        return inputs.kahan(n)
    return inputs.random_dense(m, n, seed)


@pytest.mark.parametrize("kind,m,n,nb", CASES, ids=[f"{c[0]}{c[1]}x{c[2]}nb{c[3]}" for c in CASES])
def test_qp3_matches_column_pivoting_oracle(kind, m, n, nb):
    A = _mat(kind, m, n)
    dA = q.colmajor(A)
    f = q.qp3_factor(dA, nb)
    torch.cuda.synchronize()
    o = O.qrdm(A, 0.5, 0.5, 1)
    Ag, hg, pg = dA.cpu().numpy(), f.htau.cpu().numpy(), f.perm.cpu().numpy().astype(np.int64)
    s = _first_tie(o)
    assert np.array_equal(pg[:s], o["perm"][:s]), (s, np.nonzero(pg[:s] != o["perm"][:s])[0][:5])
    # R rows and reflectors up to the first tie, element by element
    compare_rows(A, {"A": Ag, "htau": hg, "perm": pg}, o, s)
    res, orth = factorization_errors(A, Ag, hg, pg)
    assert res <= 1e-13 and orth <= 1e-13, (res, orth)
    if s == min(m, n):
        assert f.rank == o["rank"] and f.rank_colmax == o["rank_colmax"]
    print(f"\n[qp3] {kind} {m}x{n} nb {nb}: identical for {s} of {min(m, n)} columns, {f.nsteps} blocks")


def test_qp3_edge_cases():
    # empty, one column, zero matrix, non-finite
    for shape in ((0, 4), (4, 0), (5, 1), (1, 5)):
        A = np.random.default_rng(0).standard_normal(shape)
        dA = q.colmajor(A)
        f = q.qp3_factor(dA, 32)
        assert f.perm.cpu().numpy().tolist() == list(range(shape[1])) or min(shape) > 0
    Z = np.zeros((40, 30))
    fz = q.qp3_factor(q.colmajor(Z), 32)
    assert fz.rank == 0 and np.all(fz.htau.cpu().numpy() == 0.0)
    B = inputs.random_dense(30, 20, 1)
    B[3, 4] = np.inf
    dB = q.colmajor(B)
    with pytest.raises(q.QRDMError) as ei:
        q.qp3_factor(dB, 32)
    assert ei.value.code == q.QRDM_ERR_NONFINITE
    assert np.array_equal(dB.cpu().numpy(), B)
