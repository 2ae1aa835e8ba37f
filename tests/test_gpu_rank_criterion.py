"""The paper's stopping test and the DM safeguard on the GPU, on the exact
diagonal matrix of tests/test_oracle_pins.py (every reflector the identity,
every downdate exact): the single-matrix path through the C ABI must report
rank 82 by the paper's criterion (Sec. 3.4, sqrt(n - n_s) mu <= eps n
max||a_i|| at block starts), rank_colmax 50, and finish with single-column
steps once the criterion holds (Sec. 4, reading R12), step for step as the
oracle does."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_pins import criterion_diagonal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402


@pytest.mark.parametrize("kmax", [8, 32])
def test_rank_criterion_and_dm_safeguard_match_the_oracle(kmax):
    A = criterion_diagonal()
    o = O.qrdm(A, 0.9, 0.9, kmax)
    dA = q.colmajor(A)
    f = q.factor(dA, 0.9, 0.9, kmax, trace=True)
    torch.cuda.synchronize()
    assert f.rank == o["rank"] and f.rank_colmax == o["rank_colmax"] == 50
    if kmax == 8:
        assert f.rank == 82
    ns = int(f.nsteps)
    assert ns == len(o["trace"])
    for key in ("ns", "k", "l", "dm_on"):
        np.testing.assert_array_equal(np.asarray(f.trace[key][:ns], dtype=np.int64),
                                      np.asarray(o["trace"][key], dtype=np.int64), err_msg=key)
    np.testing.assert_array_equal(f.perm.cpu().numpy().astype(np.int64), np.arange(100))
    # nothing but the diagonal moved: R is A itself (zero tails, htau = 0)
    np.testing.assert_array_equal(np.abs(np.diag(dA.cpu().numpy())), np.abs(np.diag(A)))
    assert float(f.htau.abs().max()) == 0.0
