"""The shared numpy checks that every GPU test leans on (tests/_helpers.py),
checked themselves: the explicit Q from stored reflectors against LAPACK's
own QR (same storage convention), and the factorization errors against
planted mistakes, so that a check that passes everything cannot go unseen."""
from __future__ import annotations

import numpy as np
import pytest

from tests._helpers import factorization_errors, form_q, qrp_bruteforce


@pytest.mark.parametrize("m,n", [(40, 40), (60, 25), (25, 60)])
def test_form_q_equals_lapack_q(m, n):
    """numpy's raw QR returns LAPACK xGEQRF's reflectors (v below the
    diagonal with an implicit unit entry, H_i = I - tau_i v_i v_i^T): form_q
    must rebuild exactly the Q of the same factorization."""
    A = np.random.default_rng(m + n).standard_normal((m, n))
    h, tau = np.linalg.qr(A, mode="raw")
    fac = np.asfortranarray(h.T)  # raw mode returns the transposed array
    p = min(m, n)
    Q = form_q(fac, tau, ncols=p)
    Qref = np.linalg.qr(A, mode="reduced")[0]
    np.testing.assert_allclose(Q, Qref, atol=1e-13)
    res, orth = factorization_errors(A, fac, tau, np.arange(n))
    assert res < 1e-14 and orth < 1e-13


def test_factorization_errors_see_planted_mistakes():
    m, n = 50, 30
    A = np.random.default_rng(1).standard_normal((m, n))
    h, tau = np.linalg.qr(A, mode="raw")
    fac = np.asfortranarray(h.T)
    perm = np.arange(n)
    res, orth = factorization_errors(A, fac, tau, perm)
    assert res < 1e-14 and orth < 1e-13
    bad = perm.copy()
    bad[[3, 7]] = bad[[7, 3]]
    assert factorization_errors(A, fac, tau, bad)[0] > 1e-2  # a wrong permutation
    t2 = tau.copy()
    t2[4] *= 1.0 + 1e-6
    assert factorization_errors(A, fac, t2, perm)[1] > 1e-7  # htau off: Q no longer orthogonal
    f2 = fac.copy()
    f2[10, 2] += 1e-6
    assert factorization_errors(A, f2, tau, perm)[1] > 1e-7  # a reflector entry off
    f3 = fac.copy()
    f3[1, 5] += 1e-6
    assert factorization_errors(A, f3, tau, perm)[0] > 1e-8  # an R entry off


def test_bruteforce_column_pivoting_on_a_known_order():
    """Orthogonal columns of distinct norms are chosen by decreasing norm;
    a column parallel to an earlier one has no residual left and comes last."""
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 5)))
    A = Q * np.array([1.0, 3.0, 2.0, 5.0, 4.0])
    A = np.hstack([A, 2.0 * A[:, [1]]])  # parallel to column 1, norm 6
    order, gaps = qrp_bruteforce(A)
    # column 5 (norm 6) first; then column 1 has no residual left
    assert order[:5] == [5, 3, 4, 2, 0] and order[5] == 1
    assert gaps[0] == pytest.approx(1 / 6)
