"""Test helpers: checks written from definitions, independent of both the
oracle and the CUDA path (numpy only)."""
from __future__ import annotations

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
EPS = 2.0 ** -52


def golden(name: str) -> dict:
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def form_q(Afac: np.ndarray, htau: np.ndarray, ncols: int | None = None) -> np.ndarray:
    """Explicit Q = H_1 ... H_p from stored reflectors: H_i = I - htau_i v_i v_i^T,
    v_i = (0,...,0, 1, Afac[i+1:, i])."""
    m = Afac.shape[0]
    p = htau.shape[0]
    ncols = m if ncols is None else ncols
    Q = np.eye(m, ncols)
    for i in range(p - 1, -1, -1):
        v = np.zeros(m)
        v[i] = 1.0
        v[i + 1:] = Afac[i + 1:, i]
        Q -= htau[i] * np.outer(v, v @ Q)
    return Q


def upper(Afac: np.ndarray, rows: int | None = None) -> np.ndarray:
    m, n = Afac.shape
    rows = min(m, n) if rows is None else rows
    return np.triu(Afac[:rows, :])


def factorization_errors(A: np.ndarray, Afac: np.ndarray, htau: np.ndarray, perm: np.ndarray):
    """(||A Pi - Q R||_F / ||A||_F, ||Q^T Q - I||_F) for a full factorization."""
    m, n = A.shape
    p = min(m, n)
    Q = form_q(Afac, htau[:p], ncols=p)
    R = upper(Afac, p)
    nrm = np.linalg.norm(A)
    res = np.linalg.norm(A[:, perm] - Q @ R) / (nrm if nrm > 0 else 1.0)
    orth = np.linalg.norm(Q.T @ Q - np.eye(p))
    return res, orth


def qrp_bruteforce(A: np.ndarray):
    """Column pivoting from its definition (Sec. 3.1, geometric remark): at
    each step pick the column whose component orthogonal to the span of the
    already chosen columns is largest.  Residuals are recomputed from scratch
    with a library QR; returns (order, gaps) where gaps[s] is the relative
    gap between the best and second-best residual norm at step s."""
    m, n = A.shape
    chosen: list[int] = []
    gaps = []
    for _ in range(min(m, n)):
        if chosen:
            q, _ = np.linalg.qr(A[:, chosen])
            res = A - q @ (q.T @ A)
        else:
            res = A
        rn = np.linalg.norm(res, axis=0)
        rn[chosen] = -1.0
        order = np.argsort(-rn, kind="stable")
        best, second = order[0], order[1] if len(order) > 1 else None
        if second is not None and rn[second] >= 0 and rn[best] > 0:
            gaps.append((rn[best] - rn[second]) / rn[best])
        else:
            gaps.append(np.inf)
        chosen.append(int(best))
    return chosen, np.array(gaps)
