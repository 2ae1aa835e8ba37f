"""Seeded synthetic test matrices for QRDM.

This module is shared by the tests, the benchmark and the CPU oracle's callers.
It holds none of the factorization's arithmetic: it only builds input matrices
A = U diag(sigma) V^T with prescribed singular values, and the Kahan matrix.

The paper measures on the San Jose State University Singular Matrix Database
(Sec. 5), which is not available here; these generators stand in for it with
spectra shaped like numerically singular matrices (a sharp gap, a geometric
decay to roundoff level, and the Kahan matrix the paper names as a failure case
of column pivoting, Sec. 1 and Sec. 3.3).

All matrices are float64, column-major (Fortran order), and fully determined
by their seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "haar",
    "from_spectrum",
    "sigma_gap",
    "sigma_geometric",
    "sigma_gap_geometric",
    "kahan",
    "random_dense",
    "MatrixSpec",
    "named",
    "sigma_rank_geometric",
    "BatchEntry",
    "batch_entries",
]


def haar(m: int, k: int, rng: np.random.Generator) -> np.ndarray:
    """m x k matrix with orthonormal columns, Haar-distributed.

    Built from the QR factorization of an m x k standard normal matrix, with
    each column's sign fixed so that diag(R) is positive (the library QR is a
    primitive here; the result is the same whatever its sign convention).
    """
    if k == 0 or m == 0:
        return np.zeros((m, k), order="F")
    g = rng.standard_normal((m, k))
    q, r = np.linalg.qr(g, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return np.asfortranarray(q * d[None, :])


def from_spectrum(m: int, n: int, sigma: np.ndarray, seed: int) -> np.ndarray:
    """A = U diag(sigma) V^T with U (m x p), V (n x p) Haar, p = len(sigma) <= min(m, n)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    p = sigma.shape[0]
    if p > min(m, n):
        raise ValueError("spectrum longer than min(m, n)")
    rng = np.random.Generator(np.random.PCG64(seed))
    u = haar(m, p, rng)
    v = haar(n, p, rng)
    return np.asfortranarray((u * sigma[None, :]) @ v.T)


def from_spectrum_gpu(m: int, n: int, sigma: np.ndarray, seed: int, device="cuda"):
    """A = U diag(sigma) V^T built on the GPU (for sizes where the host QR is
    too slow, e.g. 16384 x 16384): N(0,1) draws from a seeded torch CUDA
    generator, Haar factors from the library QR with sign(diag R) fixed.
    Returns a column-major float64 CUDA tensor.  Seeded and deterministic on
    a given GPU; not bit-identical to from_spectrum's numpy draws."""
    import torch

    sig = torch.as_tensor(np.asarray(sigma, dtype=np.float64), device=device)
    p = sig.shape[0]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def haar_t(rows):
        x = torch.randn((rows, p), generator=g, dtype=torch.float64, device=device)
        q, r = torch.linalg.qr(x, mode="reduced")
        d = torch.sign(torch.diagonal(r))
        d[d == 0] = 1.0
        return q * d[None, :]

    u = haar_t(m)
    v = haar_t(n)
    a = (u * sig[None, :]) @ v.T
    del u, v
    return a.t().contiguous().t()


def sigma_gap(p: int, r: int, hi: float = 1.0, lo: float = 1e-14) -> np.ndarray:
    """sigma_i = hi for i <= r, lo after (a numerically rank-r matrix)."""
    s = np.full(p, lo, dtype=np.float64)
    s[:r] = hi
    return s


def sigma_geometric(p: int, lo: float = 1e-15) -> np.ndarray:
    """sigma_i = lo ** ((i - 1) / (p - 1)), i = 1..p: a geometric decay 1 -> lo."""
    if p == 1:
        return np.ones(1)
    i = np.arange(p, dtype=np.float64)
    return lo ** (i / (p - 1))


def sigma_gap_geometric(p: int, r: int, lo_top: float = 1e-3, tail: float = 1e-14) -> np.ndarray:
    """Geometric 1 -> lo_top over the first r values, then a flat tail."""
    s = np.full(p, tail, dtype=np.float64)
    if r == 1:
        s[0] = 1.0
    elif r > 1:
        i = np.arange(r, dtype=np.float64)
        s[:r] = lo_top ** (i / (r - 1))
    return s


def sigma_rank_geometric(p: int, r: int, lo_top: float = 1e-12, below: float = 1e-15) -> np.ndarray:
    """Geometric 1 -> lo_top over the first r values, then `below` (rank r)."""
    return sigma_gap_geometric(p, r, lo_top=lo_top, tail=below)


def kahan(n: int, c: float = 0.285, pert: float = 1e-10) -> np.ndarray:
    """Kahan matrix K = diag(s^(i-1)) (I - c * strict-upper ones), s = sqrt(1 - c^2).

    Every column has unit norm in exact arithmetic.  A diagonal perturbation
    pert * eps * (n - i + 1) * s^(i-1) (eps = 2^-52) is added to K_ii, i = 1..n.
    At the default pert = 1e-10 that is far below half an ulp of K_ii (for
    n <= 2048), so in FP64 it rounds away and the result is the unperturbed
    Kahan matrix.
    """
    s = math.sqrt(1.0 - c * c)
    d = s ** np.arange(n, dtype=np.float64)
    k = np.triu(np.full((n, n), -c), 1) + np.eye(n)
    k = d[:, None] * k
    eps = 2.0 ** -52
    k[np.diag_indices(n)] += pert * eps * np.arange(n, 0, -1, dtype=np.float64) * d
    return np.asfortranarray(k)


def random_dense(m: int, n: int, seed: int) -> np.ndarray:
    """Plain i.i.d. N(0,1) entries (generic full-rank input)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.standard_normal((m, n)))


@dataclass(frozen=True)
class MatrixSpec:
    """A named workload: shape, spectrum recipe and seed."""

    name: str
    m: int
    n: int
    kind: str  # "gap" | "geometric" | "gap_geometric" | "kahan" | "dense"
    seed: int = 0
    rank: int = 0  # for "gap" and "gap_geometric"

    def build(self) -> np.ndarray:
        p = min(self.m, self.n)
        if self.kind == "gap":
            return from_spectrum(self.m, self.n, sigma_gap(p, self.rank), self.seed)
        if self.kind == "geometric":
            return from_spectrum(self.m, self.n, sigma_geometric(p), self.seed)
        if self.kind == "gap_geometric":
            return from_spectrum(self.m, self.n, sigma_gap_geometric(p, self.rank), self.seed)
        if self.kind == "kahan":
            if self.m != self.n:
                raise ValueError("kahan is square")
            return kahan(self.n)
        if self.kind == "dense":
            return random_dense(self.m, self.n, self.seed)
        raise ValueError(self.kind)

    def sigma(self) -> np.ndarray | None:
        """The prescribed singular values (None where the recipe fixes none)."""
        p = min(self.m, self.n)
        if self.kind == "gap":
            return sigma_gap(p, self.rank)
        if self.kind == "geometric":
            return sigma_geometric(p)
        if self.kind == "gap_geometric":
            return sigma_gap_geometric(p, self.rank)
        return None


_NAMED = {
    # 256 x 256, sigma = 1 (i <= 128) then 1e-14: numerical rank 128.
    "gap256": MatrixSpec("gap256", 256, 256, "gap", seed=0, rank=128),
    # geometric decay 1 -> 1e-15.
    "geo4096": MatrixSpec("geo4096", 4096, 4096, "geometric", seed=0),
    "geo8192x2048": MatrixSpec("geo8192x2048", 8192, 2048, "geometric", seed=0),
    "kahan2048": MatrixSpec("kahan2048", 2048, 2048, "kahan"),
    # rank-8192 gap spectrum: geometric 1 -> 1e-3 then 1e-14.
    "gapgeo16384": MatrixSpec("gapgeo16384", 16384, 16384, "gap_geometric", seed=0, rank=8192),
    # the same recipe at 4096 (rank 2048), a host-generated profiling case
    "gapgeo4096": MatrixSpec("gapgeo4096", 4096, 4096, "gap_geometric", seed=0, rank=2048),
}


def named(name: str) -> MatrixSpec:
    return _NAMED[name]


@dataclass(frozen=True)
class BatchEntry:
    """One matrix of a batched workload: shape, numerical rank and seed."""

    m: int
    n: int
    rank: int
    seed: int

    def sigma(self) -> np.ndarray:
        return sigma_rank_geometric(min(self.m, self.n), self.rank)

    def build(self) -> np.ndarray:
        return from_spectrum(self.m, self.n, self.sigma(), self.seed)

    def build_gpu(self, device="cuda"):
        return from_spectrum_gpu(self.m, self.n, self.sigma(), self.seed, device=device)


def batch_entries(count: int = 2000, seed: int = 0, m_lo: int = 64, m_hi: int = 1024, n_lo: int = 32) -> list:
    """The uneven batch: m ~ U[m_lo, m_hi], n ~ U[min(n_lo, m), m],
    rank ~ U[ceil(n/4), n], sigma geometric 1 -> 1e-12 over the rank and
    1e-15 below it; matrix i is seeded with seed * 1_000_003 + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(min(n_lo, m), m + 1))
        r = int(rng.integers(max(1, -(-n // 4)), n + 1))
        out.append(BatchEntry(m, n, r, seed * 1_000_003 + i))
    return out
