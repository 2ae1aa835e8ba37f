"""The seeded input generators against the recipes they implement.

Every parity case and every benchmark line runs on these matrices, so each
recipe is checked against its definition: prescribed singular values, Haar
factors with the column signs fixed, the Kahan matrix and its diagonal
perturbation, the named workloads' shapes, and the uneven batch's ranges."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2106_03138_gb300 import inputs

EPS = 2.0 ** -52


def test_haar_is_orthonormal_with_the_signs_fixed():
    """Q from the QR of an m x k normal draw, each column's sign chosen so
    that the triangular factor has a positive diagonal: Q^T G is then upper
    triangular with a positive diagonal, G being the same draw."""
    for m, k, seed in ((50, 50, 1), (80, 30, 2), (7, 1, 3)):
        g = np.random.Generator(np.random.PCG64(seed)).standard_normal((m, k))
        q = inputs.haar(m, k, np.random.Generator(np.random.PCG64(seed)))
        assert q.flags.f_contiguous
        np.testing.assert_allclose(q.T @ q, np.eye(k), atol=1e-14)
        r = q.T @ g
        assert np.all(np.abs(np.tril(r, -1)) <= 1e-12 * np.abs(r).max())
        assert np.all(np.diag(r) > 0.0)
    assert inputs.haar(0, 3, np.random.default_rng(0)).shape == (0, 3)


@pytest.mark.parametrize("m,n", [(120, 120), (200, 80), (60, 150)])
def test_from_spectrum_has_the_prescribed_singular_values(m, n):
    p = min(m, n)
    sig = inputs.sigma_geometric(p, 1e-8)
    A = inputs.from_spectrum(m, n, sig, 5)
    assert A.shape == (m, n) and A.flags.f_contiguous
    # within the SVD's own backward error, a few eps sigma_1 (sigma_1 = 1)
    np.testing.assert_allclose(np.linalg.svd(A, compute_uv=False), sig, rtol=1e-12, atol=20 * EPS)
    # a roundoff-level tail likewise
    gap = inputs.sigma_gap(p, p // 2)
    s = np.linalg.svd(inputs.from_spectrum(m, n, gap, 5), compute_uv=False)
    np.testing.assert_allclose(s[: p // 2], 1.0, rtol=1e-13)
    assert np.all(np.abs(s[p // 2:] - 1e-14) <= 50 * EPS)
    # seeded: the same seed gives the same bytes, another seed another matrix
    assert np.array_equal(A, inputs.from_spectrum(m, n, sig, 5))
    assert not np.allclose(A, inputs.from_spectrum(m, n, sig, 6))
    with pytest.raises(ValueError):
        inputs.from_spectrum(m, n, np.ones(p + 1), 0)


def test_device_recipe_has_the_prescribed_singular_values():
    """The generator used for the 16384^2 workload, run on the host device:
    the same recipe, so the same singular values (not the same draws)."""
    torch = pytest.importorskip("torch")
    sig = inputs.sigma_gap_geometric(96, 48)
    a = inputs.from_spectrum_gpu(128, 96, sig, 3, device="cpu")
    assert a.dtype == torch.float64 and a.shape == (128, 96) and a.stride() == (1, 128)
    s = np.linalg.svd(a.numpy(), compute_uv=False)
    np.testing.assert_allclose(s[:48], sig[:48], rtol=1e-12)
    assert np.all(np.abs(s[48:] - 1e-14) <= 50 * EPS)


def test_spectra():
    g = inputs.sigma_geometric(301, 1e-15)
    assert g[0] == 1.0 and g[-1] == pytest.approx(1e-15, rel=1e-12)
    np.testing.assert_allclose(g[1:] / g[:-1], 1e-15 ** (1 / 300), rtol=1e-12)
    assert np.array_equal(inputs.sigma_geometric(1), np.ones(1))
    s = inputs.sigma_gap(256, 128)
    assert np.all(s[:128] == 1.0) and np.all(s[128:] == 1e-14)
    t = inputs.sigma_gap_geometric(16384, 8192)
    assert t[0] == 1.0 and t[8191] == pytest.approx(1e-3, rel=1e-12) and np.all(t[8192:] == 1e-14)
    np.testing.assert_allclose(t[1:8192] / t[:8191], 1e-3 ** (1 / 8191), rtol=1e-12)
    b = inputs.sigma_rank_geometric(100, 40)
    assert b[39] == pytest.approx(1e-12, rel=1e-12) and np.all(b[40:] == 1e-15)
    assert inputs.sigma_gap_geometric(5, 1)[0] == 1.0


def test_kahan_matrix_and_its_perturbation():
    """K = diag(s^(i-1)) (I - c strict-upper ones), s = sqrt(1 - c^2): every
    column has unit norm (s^(2j) + c^2 (1 - s^(2j)) / (1 - s^2) = 1).  The
    perturbation adds 1e-10 eps (n - i + 1) s^(i-1) to K_ii and nothing else."""
    n, c = 300, 0.285
    s = math.sqrt(1 - c * c)
    K0 = inputs.kahan(n, c, pert=0.0)
    assert np.allclose(np.tril(K0, -1), 0.0)
    i, j = np.triu_indices(n, 1)
    np.testing.assert_allclose(K0[i, j], -c * s ** i, rtol=1e-14)
    np.testing.assert_allclose(np.diag(K0), s ** np.arange(n), rtol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(K0, axis=0), 1.0, rtol=1e-13)
    K = inputs.kahan(n, c)
    assert K.flags.f_contiguous
    D = K - K0
    assert np.all(D[~np.eye(n, dtype=bool)] == 0.0)
    want = 1e-10 * EPS * np.arange(n, 0, -1) * s ** np.arange(n)
    # K_ii + d rounds d to the spacing of K_ii: compare within half of it
    assert np.all(np.abs(np.diag(D) - want) <= 0.5 * np.spacing(np.diag(K0)))
    # at most 1e-10 (n - i + 1) ulps of K_ii for these sizes: the term rounds
    # away entirely, and the workload is the unperturbed Kahan matrix in FP64
    assert np.all(want < 0.5 * np.spacing(np.diag(K0)))
    for size in (n, 2048):
        assert np.array_equal(inputs.kahan(size, c), inputs.kahan(size, c, pert=0.0))


def test_named_workloads():
    """The workloads the benchmark and the parity tests name."""
    want = {
        "gap256": (256, 256, "gap", 128),
        "geo4096": (4096, 4096, "geometric", 0),
        "geo8192x2048": (8192, 2048, "geometric", 0),
        "kahan2048": (2048, 2048, "kahan", 0),
        "gapgeo16384": (16384, 16384, "gap_geometric", 8192),
        "gapgeo4096": (4096, 4096, "gap_geometric", 2048),
    }
    for name, (m, n, kind, r) in want.items():
        sp = inputs.named(name)
        assert (sp.m, sp.n, sp.kind, sp.rank) == (m, n, kind, r), name
    assert inputs.named("gap256").sigma()[127:129].tolist() == [1.0, 1e-14]
    assert inputs.named("kahan2048").sigma() is None
    with pytest.raises(ValueError):
        inputs.MatrixSpec("k", 4, 5, "kahan").build()


def test_uneven_batch():
    """m ~ U[64, 1024], n ~ U[32, m], rank ~ U[ceil(n/4), n], one seed per
    matrix, the whole list fixed by the batch seed."""
    ents = inputs.batch_entries(2000, seed=0)
    assert len(ents) == 2000
    m = np.array([e.m for e in ents])
    n = np.array([e.n for e in ents])
    r = np.array([e.rank for e in ents])
    assert m.min() >= 64 and m.max() <= 1024 and np.all((n >= 32) & (n <= m))
    assert np.all((r >= -(-n // 4)) & (r <= n))
    assert len({e.seed for e in ents}) == 2000
    # uniform draws: the sample mean of m sits near (64 + 1024) / 2
    assert abs(m.mean() - 544.0) < 4 * 277.0 / math.sqrt(2000)
    assert inputs.batch_entries(50, seed=0) == ents[:50]
    assert inputs.batch_entries(50, seed=1) != ents[:50]
    e = ents[0]
    sv = np.linalg.svd(e.build(), compute_uv=False)
    sig = e.sigma()
    np.testing.assert_allclose(sv[: e.rank], sig[: e.rank], rtol=1e-12, atol=20 * EPS)
    assert np.all(sv[e.rank:] < 1e-13)
