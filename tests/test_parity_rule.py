"""The GPU-vs-oracle comparison rule (tests/_parity.py), checked on the CPU.

The GPU parity tests are only as strong as ``compare``.  Here the oracle's
own output plays the GPU's part: ``compare`` must accept it unchanged, accept
it moved by half of every rounding bound, accept a divergence at an exact
tie, and accept the oracle's run on a rounding-sized perturbation of the
input (which checks the margins the oracle logs: a decision it calls clear
must not flip); and it must reject each planted mistake that a wrong kernel
could make (an R entry, a diagonal, a reflector or an htau beyond its bound,
a swapped permutation, a different pick, block size or step count with no
tie, a wrong rank, a missed stop at the rank)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._parity import EPS, SCORES, compare

# The rule's bounds, restated from its statement (tests/_parity.py docstring)
# rather than imported, so that a changed constant there fails here.


def row_err(m, ncmp, anorm):
    """e_i = sqrt(m (i + 1)) eps anorm."""
    return np.sqrt(m * (np.arange(ncmp) + 1.0)) * EPS * anorm


def rdiag_tol(d, anorm, m):
    """|R_ii| within 1e-11 relative where |R_ii| >= 1e-3 anorm, else 1e-11 |R_ii| + e_i."""
    return np.where(d >= 1e-3 * anorm, 1e-11 * d, 1e-11 * d + row_err(m, d.size, anorm))


M, N = 300, 200


def _matrix():
    """300 x 200 with a rank-100 gap: live rows 0..99, rounding noise after."""
    return inputs.from_spectrum(M, N, inputs.sigma_gap(N, N // 2), 11)


def _copy(o):
    return {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in o.items()}


@pytest.fixture(scope="module")
def case():
    A = _matrix()
    return A, O.qrdm(A, 0.5, 0.9, 16)


def _perturbed(A, o, frac, seed=0):
    """The oracle's output moved by frac of each bound of the rule, random signs."""
    rng = np.random.default_rng(seed)
    g = _copy(o)
    p = min(M, N)
    anorm = float(np.max(np.linalg.norm(A, axis=0)))
    e = row_err(M, p, anorm)
    d = np.abs(np.diag(o["A"])[:p])
    i0 = int(np.nonzero(d < 4.0 * e)[0][0])
    R = np.triu(o["A"][:p, :])
    sgn = rng.choice([-1.0, 1.0], size=R.shape)
    g["A"][:p, :] += np.triu(frac * sgn * (1e-11 * np.abs(R) + e[:, None]), 1)
    dt = np.minimum(rdiag_tol(d, anorm, M), 1e-11 * d + e)
    g["A"][np.arange(p), np.arange(p)] += frac * np.sign(np.diag(R)) * sgn[0, :p] * dt
    for i in range(i0):
        tail = rng.choice([-1.0, 1.0], size=M - i - 1)
        g["A"][i + 1:, i] += frac * tail * (3.0 * e[i] / d[i])
        g["htau"][i] += frac * rng.choice([-1.0, 1.0]) * (2.0 * e[i] / d[i])
    return g, e, d, i0


def test_accepts_the_oracle_unchanged(case):
    A, o = case
    rep = compare(A, _copy(o), o)
    assert rep["diverged_at"] is None and rep["ncmp"] == N
    assert rep["r_max_err_over_bound"] == 0.0
    assert rep["noise_onset_row"] == N // 2  # both regimes of the rule are exercised


def test_accepts_changes_within_half_of_every_bound(case):
    A, o = case
    for seed in range(3):
        g, _, _, _ = _perturbed(A, o, 0.5, seed)
        rep = compare(A, g, o)
        # (adding a step of 1e-11 |R| rounds it by up to 2e-5 of itself)
        assert 0.2 < rep["r_max_err_over_bound"] <= 0.5 * (1 + 1e-4)
        assert 0.2 < rep["v_max_err_over_bound"] <= 0.5 * (1 + 1e-4)
        assert 0.2 < rep["htau_max_err_over_bound"] <= 0.5 * (1 + 1e-4)


def test_accepts_a_divergence_at_an_exact_tie():
    """Two identical columns have equal norms at every step: a program that
    takes the other one where the oracle takes the first is as right, and
    only the rows finished before that step are compared."""
    A = _matrix()
    j1, j2 = 37, 150
    A[:, j2] = A[:, j1]
    o = O.qrdm(A, 0.5, 0.9, 16)
    sw = np.arange(N)
    sw[j1], sw[j2] = j2, j1
    g = _copy(o)
    g["perm"] = sw[o["perm"]]
    g["J"] = np.where(o["J"] >= 0, sw[np.maximum(o["J"], 0)], -1)
    rep = compare(A, g, o)
    assert rep["diverged_at"] is not None and rep["tie_score"] == 0.0
    assert 0 < rep["ncmp"] < N


PERTURBED = [
    # (name, matrix, tau, delta, k_max, decisions flip somewhere)
    ("gap256 (0.9, 0.9, 32)", lambda: inputs.from_spectrum(256, 256, inputs.sigma_gap(256, 128), 5), 0.9, 0.9, 32,
     True),
    ("gap256 (0.15, 0.9, 64)", lambda: inputs.from_spectrum(256, 256, inputs.sigma_gap(256, 128), 5), 0.15, 0.9, 64,
     True),
    ("geo 300x200 1e-15 (0.5, 0.9, 16)",
     lambda: inputs.from_spectrum(300, 200, inputs.sigma_geometric(200, 1e-15), 7), 0.5, 0.9, 16, True),
    ("geo 300x200 1e-12 (0.2, 0.95, 16)",
     lambda: inputs.from_spectrum(300, 200, inputs.sigma_geometric(200, 1e-12), 8), 0.2, 0.95, 16, False),
    ("dense 200x150 (0.9, 0.9, 32)", lambda: inputs.random_dense(200, 150, 3), 0.9, 0.9, 32, False),
    ("kahan 200 (0.15, 0.9, 64)", lambda: inputs.kahan(200), 0.15, 0.9, 64, True),
]


@pytest.mark.parametrize("case", PERTURBED, ids=lambda c: c[0])
def test_the_oracle_on_a_perturbed_input_passes_the_rule(case):
    """Soundness of the margins the oracle logs: its own run on A + E, with
    entries of E up to about eps anorm (rounding-sized), is another correct
    program's answer for A.  The rule must accept it: every step where the
    two runs decide differently must be one the oracle logged as a tie, and
    the rows before it must agree within the bounds.  Where the inputs have a
    roundoff tail or equal norms (gap, 1e-15 geometric, Kahan) the decisions
    do flip, so the tie test itself is exercised."""
    _, build, tau, delta, kmax, flips = case
    A = build()
    o = O.qrdm(A, tau, delta, kmax)
    anorm = float(np.max(np.linalg.norm(A, axis=0)))
    diverged = []
    for seed in range(2):
        rng = np.random.default_rng(seed)
        for scale in (0.25, 1.0):
            E = scale * EPS * anorm * rng.standard_normal(A.shape)
            rep = compare(A, O.qrdm(A + E, tau, delta, kmax), o)
            diverged.append(rep["diverged_at"] is not None)
            if rep["ncmp"]:
                assert rep["r_max_err_over_bound"] <= 0.5
    assert any(diverged) == flips


# Errors are planted at 1.5 times their bound: a rule loosened by a factor of
# two or more would accept them.
OVER = 1.5


def _plant(name, A, o, e, d, i0):
    g = _copy(o)
    anorm = float(np.max(np.linalg.norm(A, axis=0)))
    if name == "r_entry":  # one entry of a live row
        i, j = 10, 150
        g["A"][i, j] += OVER * (1e-11 * abs(o["A"][i, j]) + e[i])
    elif name == "r_entry_absolute":  # the smallest live entry, where the e_i term governs
        R = np.abs(np.triu(o["A"][:i0, :], 1))
        R[R == 0.0] = np.inf
        i, j = np.unravel_index(np.argmin(R), R.shape)
        assert 1e-11 * R[i, j] < 0.01 * e[i]
        g["A"][i, j] += OVER * (1e-11 * R[i, j] + e[i])
    elif name == "r_diag_relative":  # a large |R_ii|, relative bound 1e-11
        g["A"][5, 5] *= 1.0 + OVER * 1e-11
    elif name == "r_diag_relative_only":
        # |R_ii| >= 1e-3 anorm has no absolute slack: 1e-11 |R_ii| + e_i / 2
        # passes every entry bound but not the diagonal's
        assert abs(o["A"][5, 5]) >= 1e-3 * anorm
        g["A"][5, 5] += np.sign(o["A"][5, 5]) * (1e-11 * abs(o["A"][5, 5]) + 0.5 * e[5])
    elif name == "r_diag_noise_row":  # a noise row's |R_ii|
        i = i0 + 20
        g["A"][i, i] += np.sign(o["A"][i, i]) * OVER * rdiag_tol(d, anorm, M)[i]
    elif name == "r_noise_block":  # a noise-row entry beyond the size of the noise block
        i, j = i0 + 5, i0 + 40
        noise = 2.0 * float(np.max(np.linalg.norm(np.triu(o["A"][: min(M, N), :])[i0:], axis=0)))
        g["A"][i, j] += OVER * (1e-11 * abs(o["A"][i, j]) + e[i] + noise)
    elif name == "reflector_sign":
        g["A"][11:, 10] *= -1.0
    elif name == "reflector_entry":
        g["A"][60, 40] += OVER * 3.0 * e[40] / d[40]
    elif name == "htau":
        g["htau"][7] += OVER * 2.0 * e[7] / d[7]
    elif name == "perm_swap":
        g["perm"][[3, 4]] = g["perm"][[4, 3]]
    elif name == "perm_swap_tail":
        g["perm"][[N - 2, N - 1]] = g["perm"][[N - 1, N - 2]]
    elif name == "pick":  # a different column at a step with a clear margin
        s = 2
        used = set(int(x) for x in g["J"][s][: int(o["trace"]["k"][s])])
        g["J"][s][3] = next(j for j in range(N) if j not in used)
    elif name == "block_size":
        g["trace"]["k"][4] -= 1
    elif name == "panel_break":
        g["trace"]["l"][1] -= 1
    elif name == "dm_flag":
        g["trace"]["dm_on"][3] = 1 - g["trace"]["dm_on"][3]
    elif name == "one_step_short":
        g["trace"], g["J"] = g["trace"][:-1], g["J"][:-1]
    elif name == "rank":
        g["rank"] += 1
    elif name == "rank_colmax":
        g["rank_colmax"] -= 1
    else:
        raise ValueError(name)
    return g


PLANTS = ["r_entry", "r_entry_absolute", "r_diag_relative", "r_diag_relative_only", "r_diag_noise_row", "r_noise_block", "reflector_sign", "reflector_entry",
          "htau", "perm_swap", "perm_swap_tail", "pick", "block_size", "panel_break", "dm_flag", "one_step_short",
          "rank", "rank_colmax"]


@pytest.mark.parametrize("name", PLANTS)
def test_rejects_a_planted_mistake(case, name):
    A, o = case
    _, e, d, i0 = _perturbed(A, o, 0.0)
    g = _plant(name, A, o, e, d, i0)
    with pytest.raises(AssertionError):
        compare(A, g, o)


def test_a_missed_stop_at_the_rank_needs_a_tie_in_the_stopping_test(case):
    """With the stop at the rank (Sec. 3.4 criterion), a program that goes on
    where the oracle stopped is accepted only if the oracle's stopping test
    was within its rounding margin.  At the 1e-15 gap the residual norms are
    rounding noise and the test is a tie; after exactly zero residuals
    (mu = 0) it is not."""
    A, _ = case
    o = O.qrdm(A, 0.5, 0.9, 16, stop_at_rank=True)
    full = O.qrdm(A, 0.5, 0.9, 16)
    assert o["stop"] is not None and int(o["stop"]["ns"]) == o["rank"]
    assert float(o["stop"]["s_stop"]) < 1.0
    rep = compare(A, full, o)
    assert rep["diverged_at"] == len(o["trace"]) and rep["ncmp"] == o["rank"]

    rng = np.random.default_rng(4)
    Z = np.zeros((100, 60))
    live = np.sort(rng.choice(60, size=40, replace=False))
    Z[:, live] = rng.standard_normal((100, 40))
    o = O.qrdm(Z, 0.5, 0.9, 16, stop_at_rank=True)
    full = O.qrdm(Z, 0.5, 0.9, 16)
    assert o["rank"] == 40 and o["stop"] is not None and np.isinf(float(o["stop"]["s_stop"]))
    assert len(full["trace"]) > len(o["trace"])
    with pytest.raises(AssertionError):
        compare(Z, full, o)
    # and the run without the stop has no stopping record: past its last
    # step nothing may go on
    assert full["stop"] is None
    short = _copy(full)
    short["trace"], short["J"] = full["trace"][:-1], full["J"][:-1]
    with pytest.raises(AssertionError):
        compare(Z, full, short)


def _pick_at(g, o, s):
    """g with a different column picked at step s."""
    g = _copy(g)
    used = set(int(x) for x in o["J"][s][: int(o["trace"]["k"][s])])
    g["J"][s][3] = next(j for j in range(N) if j not in used)
    return g


@pytest.mark.parametrize("score,tie", [(0.9, True), (1.1, False)])
def test_a_logged_score_below_one_is_a_tie_and_above_is_not(case, score, tie):
    """The threshold of the tie test itself: a step whose smallest logged
    score (decision margin over its rounding uncertainty) is below 1 may
    diverge, one at or above 1 may not."""
    A, o = case
    o2 = _copy(o)
    # step 2's smallest score becomes `score` (the others there are far above it)
    assert min(float(o["trace"][f][2]) for f in SCORES) > 1e3
    o2["trace"]["s_order"][2] = score
    g = _pick_at(o, o, 2)
    if tie:
        assert compare(A, g, o2)["diverged_at"] == 2
    else:
        with pytest.raises(AssertionError):
            compare(A, g, o2)


@pytest.mark.parametrize("score,tie", [(0.5, True), (2.0, False)])
def test_an_earlier_recompute_near_tie_explains_a_later_divergence(case, score, tie):
    """A norm recomputed or downdated on a near-tie of the recompute test
    changes that norm within its uncertainty, so every later decision may
    differ: a divergence at step 3 is accepted when step 1 logged a recompute
    score below 1."""
    A, o = case
    o2 = _copy(o)
    o2["trace"]["s_recomp"][1] = score
    g = _pick_at(o, o, 3)
    if tie:
        assert compare(A, g, o2)["diverged_at"] == 3
    else:
        with pytest.raises(AssertionError):
            compare(A, g, o2)


def test_the_permutation_of_unfactored_columns_is_compared():
    """A wide matrix (m < n): the columns past min(m, n) are never factored,
    but their order is part of the result and must match when no decision
    differs.  Two identical tiny columns stay there; exchanging their labels
    leaves R by original column unchanged, so only the permutation check can
    see it."""
    rng = np.random.default_rng(4)
    c = 1e-8 * rng.standard_normal((80, 1))
    A = np.asfortranarray(np.hstack([inputs.from_spectrum(80, 118, inputs.sigma_geometric(80, 1e-6), 4), c, c]))
    o = O.qrdm(A, 0.5, 0.9, 16)
    g = _copy(o)
    assert compare(A, g, o)["diverged_at"] is None
    p1, p2 = (int(np.nonzero(o["perm"] == j)[0][0]) for j in (118, 119))
    assert min(p1, p2) >= 80  # both left unfactored
    g["perm"][[p1, p2]] = g["perm"][[p2, p1]]
    with pytest.raises(AssertionError):
        compare(A, g, o)


def test_the_permutation_before_a_tie_is_compared():
    """After a divergence at a tie, the permutation of the columns factored
    before it must still match."""
    A = _matrix()
    j1, j2 = 37, 150
    A[:, j2] = A[:, j1]
    o = O.qrdm(A, 0.5, 0.9, 16)
    sw = np.arange(N)
    sw[j1], sw[j2] = j2, j1
    g = _copy(o)
    g["perm"] = sw[o["perm"]]
    g["J"] = np.where(o["J"] >= 0, sw[np.maximum(o["J"], 0)], -1)
    ncmp = compare(A, g, o)["ncmp"]
    g["perm"][[0, 1]] = g["perm"][[1, 0]]
    assert ncmp > 2
    with pytest.raises(AssertionError):
        compare(A, g, o)
