"""GPU-vs-oracle comparison rules (tie-aware), shared by the GPU tests.

The permutation must be identical until the first step where the two sides
take a different decision; that step must be one where the oracle logged a
decision margin below the rounding uncertainty of the compared quantities
(a tie).  Until then |R_ii| must agree within

    1e-11 |R_ii| + c eps anorm (1 + anorm / min_{i'<i} |R_i'i'|),  c = sqrt(m n),

the first-order perturbation of R_ii = dist(a_i, span(a_1..a_{i-1})) under a
backward error c eps anorm in A (two backward-stable FP64 programs differ by
that much); for well-separated leading columns the 1e-11 relative term
dominates.
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


def is_tie(otrace, s) -> tuple[bool, float]:
    if s >= len(otrace):
        return True, 0.0  # the oracle stopped (criterion) where the GPU went on: stop test
    rec = otrace[s]
    score = min(float(rec[f]) for f in SCORES)
    # an earlier near-tie in the recompute test changes u by its uncertainty
    prev = min([float(r["s_recomp"]) for r in otrace[: s + 1]] + [np.inf])
    return (score < 1.0 or prev < 1.0), min(score, prev)


def rdiag_tol(rdiag_ref: np.ndarray, anorm: float, m: int, n: int) -> np.ndarray:
    d = np.abs(rdiag_ref)
    run_min = np.minimum.accumulate(np.concatenate([[np.inf], d[:-1]]))
    run_min = np.where(np.isfinite(run_min), run_min, anorm)
    run_min = np.maximum(run_min, 1e-300)
    c = np.sqrt(float(m) * float(n))
    return 1e-11 * d + c * EPS * anorm * (1.0 + anorm / run_min)


def compare(A: np.ndarray, g: dict, o: dict) -> dict:
    """g: {'A','htau','perm','trace','J','rank','rank_colmax'} (numpy), o: oracle dict."""
    m, n = A.shape
    p = min(m, n)
    anorm = float(np.max(np.linalg.norm(A, axis=0))) if n else 0.0
    div, ncols = walk(g["trace"], g["J"], o["trace"], o["J"])
    report = {"diverged_at": div, "tie_score": None}
    if div is not None:
        tie, score = is_tie(o["trace"], div)
        report["tie_score"] = score
        assert tie, f"GPU and oracle take different decisions at step {div} with no tie (score {score:.3g})"
        ncmp = ncols
    else:
        ncmp = p
        assert np.array_equal(g["perm"], o["perm"]), "identical decisions but different permutations"
        assert g["rank"] == o["rank"]
    report["ncmp"] = ncmp
    assert np.array_equal(g["perm"][:ncmp], o["perm"][:ncmp])
    dg = np.abs(np.diag(g["A"])[:ncmp])
    do = np.abs(np.diag(o["A"])[:ncmp])
    tol = rdiag_tol(np.diag(o["A"])[:p], anorm, m, n)[:ncmp]
    err = np.abs(dg - do)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, f"|R_ii| differs at i={bad[:5]}: {err[bad[:5]]} > {tol[bad[:5]]}"
    rel = err / np.maximum(do, 1e-300)
    report["max_rel_rdiag"] = float(np.max(rel[do > 1e-3 * anorm])) if np.any(do > 1e-3 * anorm) else 0.0
    # htau_i = 1 - alpha_i/beta_i inherits R_ii's conditioning: |d htau| <= 2 tol_i / |R_ii|
    hg, ho = g["htau"][:ncmp], o["htau"][:ncmp]
    htol = 2.0 * tol / np.maximum(do, 1e-300) + 1e-15
    badh = np.nonzero(np.abs(hg - ho) > htol)[0]
    assert badh.size == 0, f"htau differs at i={badh[:5]}: {np.abs(hg - ho)[badh[:5]]} > {htol[badh[:5]]}"
    # rank_colmax (mu <= eps1 anorm, no sqrt factor) changes no decision, so it
    # is not in the trace walk; it may differ only where the oracle's mu at
    # that step lay within the roundoff band sqrt(mn) eps anorm of the threshold
    rc_g, rc_o = g["rank_colmax"], o["rank_colmax"]
    if rc_g != rc_o and min(rc_g, rc_o) < ncmp:
        eps1 = EPS * n
        band = np.sqrt(float(m) * n) * EPS * anorm
        tr = o["trace"]
        for rc in (rc_g, rc_o):
            hit = np.nonzero(tr["ns"] == rc)[0]
            if hit.size:
                mu = float(tr["mu"][hit[0]])
                assert abs(mu - eps1 * anorm) <= band, f"rank_colmax {rc_g} vs {rc_o} without a tie"
    return report
