"""The rank thresholds of the reduced-precision forms, as a CPU model.

The stopping criterion of Sec. 3.4 fires once sqrt(n - ns) * mu <= eps1 * anorm.
Here mu is the largest remaining column norm and anorm the largest initial
one. With the FP64 choice eps1 = eps * n, an update carried out in lower
precision never gets there: past the gap, its roundoff leaves the trailing
block at a noise floor far above eps. The forms therefore raise eps1 to
their own class:
  * FP32: 8 * 2^-24 * sqrt(n);
  * 3xTF32: 8 * 2^-21 * sqrt(n);
  * split-BF16x3: 2^-16 * sqrt(n).

The model factors a matrix whose last n - r columns lie in the span of the
first r (up to 1e-14), in blocks of 64 Householder reflectors. The panel is
FP64; each block's trailing update runs in the form's arithmetic:
  * FP32: operands and results rounded to FP32;
  * 3xTF32 and BF16x3: operands split bit-exactly as hi + lo, with the
    products hi*hi + hi*lo + lo*hi and the results rounded to FP32.
The noise left in the trailing block after r columns is checked three ways:
  * It sits at least 2x below each form's threshold, so the criterion fires
    at the gap. The model gives 11x for FP32, 48x for 3xTF32 and 4x for
    BF16x3.
  * It sits within 100x of that threshold, so the constant matches its
    class. A BF16 constant on the TF32 form would be thousands of times too
    loose.
  * It sits above the FP64 threshold, which shows why the form needs its
    own."""
from __future__ import annotations

import numpy as np
import pytest

EPS = 2.0**-52


def _bf16_rne(x64):
    x32 = np.asarray(x64, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _tf32_rna(x64):
    x32 = np.asarray(x64, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x1000) >> 13) << 13
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _split(x, rnd):
    x32 = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = rnd(x32)
    lo = rnd(x32 - hi)
    return hi, lo


def _matmul(a, b, form):
    """a @ b in the arithmetic of a form (FP64 result): operands rounded to
    FP32 or split, exact products summed in FP64, the result rounded to FP32.
    Every form is modelled at this one level (representation, not
    accumulation order, which the GPU tests measure), so that the model does
    not depend on the host BLAS."""
    if form == "fp64":
        return a @ b
    if form == "fp32":
        a32 = a.astype(np.float32).astype(np.float64)
        b32 = b.astype(np.float32).astype(np.float64)
        return (a32 @ b32).astype(np.float32).astype(np.float64)
    rnd = _tf32_rna if form == "tf32x3" else _bf16_rne
    ah, al = _split(a, rnd)
    bh, bl = _split(b, rnd)
    return (ah @ bh + ah @ bl + al @ bh).astype(np.float32).astype(np.float64)


def _householder_panel(P):
    """FP64 Householder QR of a panel (LAPACK sign convention): V unit lower
    trapezoidal, htau, and R in place."""
    m, k = P.shape
    V = np.zeros((m, k))
    htau = np.zeros(k)
    for j in range(k):
        x = P[j:, j]
        alpha = x[0]
        nrm = np.linalg.norm(x)
        beta = -np.copysign(nrm, alpha)
        v = x / (alpha - beta)
        v[0] = 1.0
        htau[j] = (beta - alpha) / beta
        P[j:, j:] -= htau[j] * np.outer(v, v @ P[j:, j:])
        V[j:, j] = v
    return V, htau


def _larft(V, htau):
    k = V.shape[1]
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = htau[j]
        if j:
            T[:j, j] = -htau[j] * T[:j, :j] @ (V[:, :j].T @ V[:, j])
    return T


def _trailing_noise(form, m=512, n=384, r=192, nb=64, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, r)) / np.sqrt(m)
    C = rng.standard_normal((r, n - r)) / np.sqrt(r)
    A = np.hstack([X, X @ C + 1e-14 * rng.standard_normal((m, n - r)) / np.sqrt(m)])
    anorm = np.linalg.norm(A, axis=0).max()
    for ns in range(0, r, nb):
        V, htau = _householder_panel(A[ns:, ns:ns + nb])
        T = _larft(V, htau)
        A22 = A[ns:, ns + nb:]
        W = T.T @ _matmul(V.T, A22, form)  # T applied in FP64 (FP32 in the GPU forms; a small term)
        A[ns:, ns + nb:] = A22 - _matmul(V, W, form)
    mu = np.linalg.norm(A[r:, r:], axis=0).max()
    return np.sqrt(n - r) * mu / anorm, n


EPS1 = {
    "fp32": lambda n: 8 * 2.0**-24 * np.sqrt(n),
    "tf32x3": lambda n: 8 * 2.0**-21 * np.sqrt(n),
    "bf16x3": lambda n: 2.0**-16 * np.sqrt(n),
}


@pytest.mark.parametrize("form", ["fp32", "tf32x3", "bf16x3"])
def test_form_threshold_sits_above_its_noise_and_fp64_below(form):
    lhs, n = _trailing_noise(form)
    assert 2 * lhs <= EPS1[form](n), (form, lhs, EPS1[form](n))
    assert 100 * lhs >= EPS1[form](n), (form, lhs, EPS1[form](n))
    assert lhs > EPS * n, (form, lhs)  # eps * n would never fire


def test_the_fp64_update_reaches_the_fp64_threshold():
    lhs, n = _trailing_noise("fp64")
    assert lhs <= EPS * n * 10, lhs
