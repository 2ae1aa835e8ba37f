"""GPU-vs-oracle comparison rules (tie-aware), shared by the GPU tests.

The permutation must be identical until the first step where the two sides
take a different decision; that step must be one where the oracle logged a
decision margin below the rounding uncertainty of the compared quantities
(a tie).  Every row of R finished before that step, and every reflector of
it, is then compared element by element, columns matched by original index.

Row i of R is column j after i reflector applications.  Each application
adds a rounding error of norm about sqrt(m) eps ||a_j|| (an inner product of
length <= m, probabilistic rounding model) in its own direction, so two FP64
programs that sum in different orders leave errors of norm about
e_i = sqrt(m (i + 1)) eps anorm in that column.  Hence:

* |R_ii| >= 1e-3 anorm: |R_ii| within 1e-11 relative, nothing else;
* every other entry of those rows: |dR_ij| <= 1e-11 |R_ij| + e_i;
* reflector tails and htau while the column stands above that error
  (|R_ii| >= 4 e_i): v = x / (alpha - beta) with |alpha - beta| >= |R_ii|
  and |v_k| <= 1 moves by at most 3 e_i / |R_ii| per entry, and
  htau = 1 - alpha / beta by at most 2 e_i / |R_ii| (first order).
* From the first row i0 whose column is rounding noise (|R_ii| < 4 e_i) on,
  the remaining rows are fixed only up to a rotation of that noise: there
  |R_ii| keeps its bound (the largest residual norm is known within e_i),
  the other entries agree within e_i plus twice the largest column norm of
  the oracle's rows i0.. (both are noise of that size), and the reflectors
  are checked only through ||A Pi - QR|| and ||Q^T Q - I||.

``compare`` returns a report with the largest error of each kind divided by
its bound, and how many diagonal entries the relative and the absolute term
each govern.
"""
from __future__ import annotations

import numpy as np

EPS = 2.0 ** -52
SCORES = ("s_argmax", "s_cand", "s_order", "s_cos", "s_break", "s_stop")


def walk(gtrace, gJ, otrace, oJ):
    """Return (first divergent step or None, columns factored identically)."""
    nsteps = min(len(gtrace), len(otrace))
    for s in range(nsteps):
        g, o = gtrace[s], otrace[s]
        k = int(o["k"])
        same = (int(g["ns"]) == int(o["ns"]) and int(g["k"]) == k and int(g["l"]) == int(o["l"])
                and int(g["dm_on"]) == int(o["dm_on"]) and np.array_equal(gJ[s][:k], oJ[s][:k]))
        if not same:
            return s, int(o["ns"])
    if len(gtrace) != len(otrace):
        s = nsteps
        ns = int(otrace[s]["ns"]) if s < len(otrace) else int(gtrace[s]["ns"])
        return s, ns
    return None, None


def is_tie(otrace, s, ostop=None) -> tuple[bool, float]:
    """Whether the oracle's step s was decided within its rounding margin.
    Past its last step, the oracle either ran out of columns (no tie: the
    other side cannot go on) or stopped at the rank, where the margin is that
    of its stopping test (``ostop``, the oracle's record of it)."""
    if s >= len(otrace):
        if ostop is None:
            return False, np.inf
        rec = ostop
    else:
        rec = otrace[s]
    score = min(float(rec[f]) for f in SCORES)
    # an earlier near-tie in the recompute test changes u by its uncertainty
    prev = min([float(r["s_recomp"]) for r in otrace[: s + 1]] + [np.inf])
    return (score < 1.0 or prev < 1.0), min(score, prev)


def row_err(m: int, ncmp: int, anorm: float) -> np.ndarray:
    """e_i = sqrt(m (i + 1)) eps anorm for rows i < ncmp (module docstring)."""
    return np.sqrt(float(max(m, 1)) * (np.arange(ncmp, dtype=np.float64) + 1.0)) * EPS * anorm


def rdiag_tol(rdiag_ref: np.ndarray, anorm: float, m: int) -> np.ndarray:
    """Bound on | |R_ii| - |R_ii ref| | (module docstring)."""
    d = np.abs(rdiag_ref)
    return np.where(d >= 1e-3 * anorm, 1e-11 * d, 1e-11 * d + row_err(m, d.size, anorm))


def compare(A: np.ndarray, g: dict, o: dict) -> dict:
    """g: {'A','htau','perm','trace','J','rank','rank_colmax'} (numpy), o: oracle dict."""
    m, n = A.shape
    p = min(m, n)
    anorm = float(np.max(np.linalg.norm(A, axis=0))) if n else 0.0
    div, ncols = walk(g["trace"], g["J"], o["trace"], o["J"])
    report = {"diverged_at": div, "tie_score": None}
    if div is not None:
        tie, score = is_tie(o["trace"], div, o.get("stop"))
        report["tie_score"] = score
        assert tie, f"GPU and oracle take different decisions at step {div} with no tie (score {score:.3g})"
        ncmp = ncols
    else:
        ncmp = p
        assert np.array_equal(g["perm"], o["perm"]), "identical decisions but different permutations"
        assert g["rank"] == o["rank"]
    report["ncmp"] = ncmp
    assert np.array_equal(g["perm"][:ncmp], o["perm"][:ncmp])
    report.update(compare_rows(A, g, o, ncmp))
    # rank_colmax (mu <= eps1 anorm, no sqrt factor) changes no decision, so it
    # is not in the trace walk; it may differ only where the oracle's mu at
    # that step lay within the roundoff band sqrt(mn) eps anorm of the
    # threshold.  Inside the compared columns both sides started the same
    # steps, so a value there must be one of those step starts.
    rc_g, rc_o = g["rank_colmax"], o["rank_colmax"]
    if rc_g != rc_o and min(rc_g, rc_o) < ncmp:
        eps1 = EPS * n
        band = np.sqrt(float(m) * n) * EPS * anorm
        tr = o["trace"]
        for rc in (rc_g, rc_o):
            if rc >= ncmp:
                continue
            hit = np.nonzero(tr["ns"] == rc)[0]
            assert hit.size, f"rank_colmax {rc} is not the start of a block step"
            mu = float(tr["mu"][hit[0]])
            assert abs(mu - eps1 * anorm) <= band, f"rank_colmax {rc_g} vs {rc_o} without a tie"
    return report


def compare_rows(A: np.ndarray, g: dict, o: dict, ncmp: int) -> dict:
    """Element-wise comparison of the first ncmp rows of R (columns matched by
    original index) and of the first ncmp reflectors, under the bounds of the
    module docstring.  Returns the report entries."""
    m, n = A.shape
    rep: dict = {}
    anorm = float(np.max(np.linalg.norm(A, axis=0))) if n else 0.0
    if ncmp == 0 or anorm == 0.0:
        if ncmp:  # a zero matrix: R and the reflectors are exactly zero on both sides
            assert np.array_equal(np.triu(g["A"][:ncmp, :]), np.triu(o["A"][:ncmp, :]))
        return rep
    e = row_err(m, ncmp, anorm)
    # R rows by original column
    Rg = np.triu(g["A"][:ncmp, :])
    Ro = np.triu(o["A"][:ncmp, :])
    Rg_o = np.empty_like(Rg)
    Ro_o = np.empty_like(Ro)
    Rg_o[:, g["perm"]] = Rg
    Ro_o[:, o["perm"]] = Ro
    do = np.abs(np.diag(o["A"])[:ncmp])
    dg = np.abs(np.diag(g["A"])[:ncmp])
    # diagonal: pure relative where |R_ii| >= 1e-3 anorm
    hi = do >= 1e-3 * anorm
    derr = np.abs(dg - do)
    tol_d = rdiag_tol(do, anorm, m)
    bad = np.nonzero(derr > tol_d)[0]
    assert bad.size == 0, f"|R_ii| differs at i={bad[:5]}: {derr[bad[:5]]} > {tol_d[bad[:5]]}"
    rep["rdiag_rows_relative_only"] = int(hi.sum())
    rep["rdiag_max_rel_above_1e-3"] = float(np.max(derr[hi] / do[hi])) if hi.any() else 0.0
    lo = ~hi
    rel_term = 1e-11 * do
    rep["rdiag_rows_relative_governs"] = int(hi.sum() + np.sum(lo & (rel_term >= e)))
    rep["rdiag_rows_absolute_governs"] = int(np.sum(lo & (rel_term < e)))
    rep["rdiag_max_err_over_bound"] = float(np.max(derr / tol_d))
    # every entry of the finished rows; from the noise onset i0 on, within
    # the size of the noise block
    noisy = np.nonzero(do < 4.0 * e)[0]
    i0 = int(noisy[0]) if noisy.size else ncmp
    rep["noise_onset_row"] = i0
    tol_r = 1e-11 * np.abs(Ro_o) + e[:, None]
    if i0 < ncmp:
        tol_r[i0:] += 2.0 * float(np.max(np.linalg.norm(Ro_o[i0:], axis=0)))
    rerr = np.abs(Rg_o - Ro_o)
    worst = np.unravel_index(np.argmax(rerr / tol_r), rerr.shape)
    rep["r_entries_compared"] = int(ncmp * n - ncmp * (ncmp - 1) // 2)
    rep["r_max_err_over_bound"] = float(rerr[worst] / tol_r[worst])
    rep["r_max_abs_err_over_eps_anorm"] = float(rerr.max() / (EPS * anorm))
    assert rep["r_max_err_over_bound"] <= 1.0, (
        f"R entry ({worst[0]}, original column {worst[1]}) differs by {rerr[worst]:.3e} > {tol_r[worst]:.3e}")
    # reflector tails and htau up to the noise onset
    live = range(i0)
    vmax, hmax = 0.0, 0.0
    for i in live:
        if i + 1 < m:
            dv = float(np.max(np.abs(g["A"][i + 1:, i] - o["A"][i + 1:, i])))
            vmax = max(vmax, dv / (3.0 * e[i] / do[i] + 1e-15))
        dh = abs(float(g["htau"][i]) - float(o["htau"][i]))
        hmax = max(hmax, dh / (2.0 * e[i] / do[i] + 1e-15))
    rep["reflectors_compared"] = i0
    rep["v_max_err_over_bound"] = float(vmax)
    rep["htau_max_err_over_bound"] = float(hmax)
    assert vmax <= 1.0, f"reflector tail differs by {vmax:.3g} x its bound"
    assert hmax <= 1.0, f"htau differs by {hmax:.3g} x its bound"
    return rep
