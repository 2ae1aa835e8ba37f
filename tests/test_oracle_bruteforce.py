"""The oracle against a second, brute-force QRDM on small matrices.

The brute force is written from the paper's definitions in numpy with a
different structure from the oracle's:
* it recomputes every partial norm exactly at every step, with no downdate
  (Sec. 3.1 defines u_j as the norm of column j of the trailing block);
* it applies each Householder reflector to every remaining column at once
  instead of a compact-WY block update (Sec. 3.2 shows the two are equal);
* it picks candidates and tests cosines straight from their definitions
  (Alg. 1, eq. def_candidate_set), and follows every selected column through
  the pairwise swaps by its label (Sec. 4).
Both must take the same decisions step by step (J, k, l, the DM switch)
wherever both programs' margins are clear of the gap between exact and
downdated norms and the oracle's are clear of rounding, and give the same
rows of R there, signs included."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs

EPS = 2.0 ** -52


def _house(x):
    """(v with v[0] = 1, htau, beta): (I - htau v v^T) x = beta e_1, beta = -sign(x_0) ||x||."""
    alpha = x[0]
    s2 = float(np.dot(x[1:], x[1:]))
    v = np.zeros_like(x)
    v[0] = 1.0
    if s2 == 0.0:
        return v, 0.0, alpha
    nrm = np.sqrt(alpha * alpha + s2)
    beta = -nrm if alpha >= 0.0 else nrm
    v[1:] = x[1:] / (alpha - beta)
    return v, (beta - alpha) / beta, beta


def qrdm_bruteforce(A, tau, delta, kmax, schedule=None):
    """schedule: per-step (tau, delta) rows; steps past its end use (tau, delta)."""
    R = np.array(A, dtype=np.float64)
    m, n = R.shape
    kmin = min(m, n)
    label = np.arange(n)  # label[position] = original column index
    anorm = float(np.max(np.linalg.norm(R, axis=0)))
    eps1 = EPS * n
    ns, dm_on, rank = 0, True, None
    steps = []
    while ns < kmin:
        step_tau, step_delta = (tau, delta)
        if schedule is not None and len(steps) < len(schedule):
            step_tau, step_delta = float(schedule[len(steps)][0]), float(schedule[len(steps)][1])
        u = np.linalg.norm(R[ns:, ns:], axis=0)  # exact partial norms of positions ns..n-1
        jstar = int(np.argmax(u))  # first maximum: lowest position
        mu = float(u[jstar])
        # relative margins of this step's decisions on the exact norms
        margins = [np.inf]
        if u.size > 1 and mu > 0:
            margins.append((mu - np.partition(u, -2)[-2]) / mu)
            margins.append(np.min(np.abs(np.delete(u, jstar) - step_tau * mu)) / (step_tau * mu))
        if dm_on and anorm > 0:
            margins.append(abs(np.sqrt(n - ns) * mu - eps1 * anorm) / (eps1 * anorm))
        if dm_on and np.sqrt(n - ns) * mu <= eps1 * anorm:
            dm_on, rank = False, ns
        kcap = min(kmax if dm_on else 1, kmin - ns)
        cand = [j for j in range(n - ns) if j != jstar and u[j] >= step_tau * mu]
        cand.sort(key=lambda j: (-u[j], j))
        if kcap > 1:  # the order of the kept candidates and at the cap
            kept = cand[: kcap]
            margins += [(u[a] - u[b]) / u[a] for a, b in zip(kept, kept[1:]) if u[a] > 0]
        cols = [jstar] + cand[: max(kcap - 1, 0)]
        C = R[ns:, [ns + j for j in cols]]
        G = C.T @ C
        dn = np.sqrt(np.diag(G))
        J = [0]
        for a in range(1, len(cols)):
            ok = True
            for b in J:
                th = abs(G[a, b]) / (dn[a] * dn[b]) if dn[a] > 0 and dn[b] > 0 else 1.0
                margins.append(abs(th - step_delta))
                if not th < step_delta:
                    ok = False
            if ok:
                J.append(a)
        picked = [int(label[ns + cols[a]]) for a in J]  # original indices, in pick order
        for t, orig in enumerate(picked):  # pairwise swaps by label
            p = int(np.nonzero(label == orig)[0][0])
            q = ns + t
            if p != q:
                R[:, [p, q]] = R[:, [q, p]]
                label[[p, q]] = label[[q, p]]
        k = len(picked)
        eps_s = step_tau * mu
        lacc = k
        for l in range(k):
            col = ns + l
            if l >= 1 and l + 1 < k:
                nrm = np.linalg.norm(R[col:, col])
                margins.append(abs(nrm - eps_s) / eps_s)
                if nrm < eps_s:
                    lacc = l
                    break
            v, ht, beta = _house(R[col:, col].copy())
            R[col:, col + 1:] -= ht * np.outer(v, v @ R[col:, col + 1:])
            R[col, col] = beta
            R[col + 1:, col] = 0.0
        steps.append({"ns": ns, "k": k, "l": lacc, "dm_on": int(dm_on), "J": picked, "margin": min(margins)})
        ns += lacc
    return {"R": np.triu(R[:kmin]), "perm": label, "steps": steps, "rank": kmin if rank is None else rank}


def _clear(rec, gap):
    """The oracle's step is decided clear of both uncertainties: every
    logged relative margin above `gap` (the exact-vs-downdated norm gap), and
    every margin above the rounding uncertainty of the compared quantities
    (score >= 1, the tie test of the GPU comparison; in a roundoff-level
    trailing block the norms themselves are rounding noise)."""
    gaps = ("g_argmax", "g_cand", "g_cos", "g_break", "g_stop")
    # (no recompute score: the brute force uses exact norms, and the oracle's
    # are within the gap whether or not it recomputed them)
    scores = ("s_argmax", "s_cand", "s_order", "s_cos", "s_break", "s_stop")
    return all(float(rec[f]) > gap for f in gaps) and all(float(rec[f]) >= 1.0 for f in scores)


CASES = [
    # (name, matrix, tau, delta, k_max, share of the columns that must be compared)
    ("dense 30x20", lambda sd: inputs.random_dense(30, 20, sd), 0.5, 0.9, 4, 1.0),
    ("dense 24x24", lambda sd: inputs.random_dense(24, 24, sd), 0.9, 0.5, 8, 1.0),
    ("dense 16x28", lambda sd: inputs.random_dense(16, 28, sd), 0.3, 0.7, 5, 1.0),
    # rank 12 of 30: past it the trailing block is rounding noise, different in the two programs
    ("gap 40x30", lambda sd: inputs.from_spectrum(40, 30, inputs.sigma_gap(30, 12), sd), 0.5, 0.9, 6, 0.4),
    ("geo 36x36", lambda sd: inputs.from_spectrum(36, 36, inputs.sigma_geometric(36, 1e-10), sd), 0.15, 0.9, 8,
     1.0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_oracle_takes_the_brute_force_decisions(case):
    name, build, tau, delta, kmax, share = case
    compared = 0
    for sd in range(12):
        A = build(sd)
        o = O.qrdm(A, tau, delta, kmax)
        b = qrdm_bruteforce(A, tau, delta, kmax)
        # exact and downdated norms differ by up to about sqrt(m eps) relative
        gap = 1e-6
        ncols = 0
        for s, (rec, bs) in enumerate(zip(o["trace"], b["steps"])):
            if not _clear(rec, gap) or bs["margin"] <= gap:
                break
            k = int(rec["k"])
            assert (int(rec["ns"]), k, int(rec["l"]), int(rec["dm_on"])) == (bs["ns"], bs["k"], bs["l"], bs["dm_on"]), \
                (name, sd, s)
            assert list(o["J"][s][:k]) == bs["J"], (name, sd, s)
            ncols = int(rec["ns"]) + int(rec["l"])
        else:
            if len(o["trace"]) == len(b["steps"]):
                assert np.array_equal(o["perm"], b["perm"]), (name, sd)
                assert o["rank"] == b["rank"]
        if ncols:
            assert np.array_equal(o["perm"][:ncols], b["perm"][:ncols]), (name, sd)
            # the finished rows of R, signs included, columns matched by original
            # index: within the rounding of two different update orders
            m, n = A.shape
            Ro = np.empty((ncols, n))
            Rb = np.empty((ncols, n))
            Ro[:, o["perm"]] = np.triu(o["A"][:ncols, :])
            Rb[:, b["perm"]] = b["R"][:ncols, :]
            anorm = float(np.max(np.linalg.norm(A, axis=0)))
            tol = 1e-10 * np.abs(Rb) + 10.0 * np.sqrt(m * (np.arange(ncols)[:, None] + 1.0)) * EPS * anorm
            assert np.all(np.abs(Ro - Rb) <= tol), (name, sd, float(np.max(np.abs(Ro - Rb) / tol)))
        compared += ncols
    print(f"\n[brute force] {name}: {compared} of {12 * min(build(0).shape)} columns compared")
    assert compared >= round(share * 12 * min(build(0).shape)), compared


def test_per_step_schedule_matches_the_brute_force():
    """A per-step (tau, delta) schedule (the learned policy's form): step s
    uses row s of the schedule for its candidate threshold, its cosine test
    and its break threshold eps_s = tau_s mu."""
    rng = np.random.default_rng(7)
    compared = 0
    for sd in range(12):
        A = inputs.random_dense(30, 24, 50 + sd)
        sched = np.column_stack([rng.uniform(0.3, 1.0, 10), rng.uniform(0.3, 1.0, 10)])
        o = O.qrdm(A, 0.9, 0.9, 6, schedule=sched)
        b = qrdm_bruteforce(A, 0.9, 0.9, 6, schedule=sched)
        for s, (rec, bs) in enumerate(zip(o["trace"], b["steps"])):
            if not _clear(rec, 1e-6) or bs["margin"] <= 1e-6:
                break
            k = int(rec["k"])
            assert (k, int(rec["l"])) == (bs["k"], bs["l"]) and list(o["J"][s][:k]) == bs["J"], (sd, s)
            assert float(rec["eps_s"]) == pytest.approx((sched[s][0] if s < 10 else 0.9) * float(rec["mu"]), rel=1e-15)
            compared += 1
    assert compared >= 60, compared
