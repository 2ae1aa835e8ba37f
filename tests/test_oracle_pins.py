"""Pins for the CPU oracle: each check compares it with something fixed by the
paper or by the mathematics, never with itself.

A plausible slip anywhere in the oracle (a wrong sign in the reflector, a
transposed T, an off-by-one in the panel or the downdate, a wrong comparison
in DM, a mis-tracked swap) fails at least one of these."""
from __future__ import annotations

import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._helpers import EPS, factorization_errors, form_q, golden, qrp_bruteforce, upper


# ---------------------------------------------------------------- reflector
def test_householder_golden():
    """Closed-form reflectors (Alg. 2/4 'compute the Householder reflector')."""
    g = golden("householder.json")
    for c in g["cases"]:
        beta, ht, v = O.house(c["x"])
        assert beta == pytest.approx(c["beta"], abs=1e-15)
        assert ht == pytest.approx(c["htau"], abs=1e-15)
        np.testing.assert_allclose(v, c["v"], atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_householder_reflects(seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(7 + seed)
    beta, ht, v = O.house(x)
    H = np.eye(x.size) - ht * np.outer(v, v)
    y = H @ x
    assert abs(abs(beta) - np.linalg.norm(x)) <= 4 * EPS * np.linalg.norm(x)
    assert y[0] == pytest.approx(beta, rel=1e-14)
    assert np.linalg.norm(y[1:]) <= 8 * EPS * np.linalg.norm(x)
    np.testing.assert_allclose(H.T @ H, np.eye(x.size), atol=1e-14)


# ---------------------------------------------------------------- compact WY
def test_larft_golden():
    g = golden("larft.json")
    T = O.larft(np.array(g["V"]), np.array(g["htau"]))
    np.testing.assert_allclose(T, np.array(g["T"]), atol=1e-15)


@pytest.mark.parametrize("mr,l", [(9, 1), (12, 4), (40, 7), (33, 33)])
def test_larft_equals_product_of_reflectors(mr, l):
    """I - V T V^T must equal H_1 H_2 ... H_l (Sec. 3.2, compact WY)."""
    rng = np.random.default_rng(mr * 100 + l)
    V = np.zeros((mr, l))
    ht = np.zeros(l)
    P = np.eye(mr)
    for i in range(l):
        x = rng.standard_normal(mr - i)
        _, h, v = O.house(x)
        V[i:, i] = v
        ht[i] = h
        vf = np.zeros(mr)
        vf[i:] = v
        P = P @ (np.eye(mr) - h * np.outer(vf, vf))
    Vst = V.copy()
    for i in range(l):
        Vst[: i + 1, i] = 99.0  # entries on/above the diagonal must not be read
    T = O.larft(Vst, ht)
    assert np.allclose(np.tril(T, -1), 0.0)
    np.testing.assert_allclose(np.eye(mr) - V @ T @ V.T, P, atol=1e-14)


# ---------------------------------------------------------------- cosine matrix
def test_cosine_properties():
    """Theta is symmetric, has unit diagonal, |theta| <= 1 (Sec. 2 definition),
    and equals the cosines of independently normalized columns."""
    rng = np.random.default_rng(3)
    A = np.asfortranarray(rng.standard_normal((50, 12)))
    cols = [7, 0, 3, 11, 5]
    G, Th = O.cosine(A, cols, r0=4)
    C = A[4:, cols]
    np.testing.assert_allclose(G, C.T @ C, rtol=1e-13, atol=1e-13)
    Cn = C / np.linalg.norm(C, axis=0)
    np.testing.assert_allclose(Th, Cn.T @ Cn, atol=1e-14)
    np.testing.assert_allclose(Th, Th.T, atol=0)
    np.testing.assert_allclose(np.diag(Th), 1.0, atol=1e-15)
    assert np.all(np.abs(Th) <= 1.0 + 1e-15)


# ---------------------------------------------------------------- DM decisions
def _dm_matrix(name: str) -> np.ndarray:
    g = golden("dm_first_step.json")
    if name == "pair":
        return np.asfortranarray(np.array(g["matrices"]["pair"]["columns"]).T)
    c0 = np.array([1.0, 0, 0, 0])
    c1 = 0.97 * np.array([0.95, np.sqrt(1 - 0.95 ** 2), 0, 0])
    c2 = 0.95 * np.array([0.5, 0, np.sqrt(0.75), 0])
    c3 = np.array([0, 0, 0, 0.5])
    return np.asfortranarray(np.stack([c0, c1, c2, c3], axis=1))


@pytest.mark.parametrize("case", golden("dm_first_step.json")["cases"], ids=lambda c: c["why"][:40])
def test_dm_first_step_golden(case):
    A = _dm_matrix(case["matrix"])
    r = O.qrdm(A, case["tau"], case["delta"], case["k_max"], check_last=case["check_last"], max_steps=1)
    tr = r["trace"][0]
    assert int(tr["k"]) == case["k"]
    assert int(tr["l"]) == case["l"]
    assert list(r["J"][0][: case["k"]]) == case["J"]


def dm_equality_matrix(name: str) -> np.ndarray:
    """A matrix of tests/golden/dm_equality.json, column-major."""
    g = golden("dm_equality.json")
    cols = np.array(g["matrices"][name]["columns"], dtype=np.float64)
    assert cols.shape[1] == g["rows"]
    return np.asfortranarray(cols.T)


@pytest.mark.parametrize("case", golden("dm_equality.json")["cases"], ids=lambda c: c["why"][:48])
def test_dm_equality_edges(case):
    """The equality edges of the first step, from exactly representable
    columns: u_i = tau mu is a candidate (eq. def_candidate_set, >=), a
    residual equal to eps_s does not stop the panel (eq. lenght_check, <),
    and equal-norm candidates are visited in position order (reading R4)."""
    A = dm_equality_matrix(case["matrix"])
    r = O.qrdm(A, case["tau"], case["delta"], case["k_max"], check_last=case["check_last"], max_steps=1)
    tr = r["trace"][0]
    assert int(tr["ncand_all"]) == case["ncand_all"]
    assert int(tr["k"]) == case["k"]
    assert int(tr["l"]) == case["l"]
    assert list(r["J"][0][: case["k"]]) == case["J"]
    # the exact values behind the decisions
    assert float(tr["mu"]) == float(np.max(np.linalg.norm(A, axis=0)))
    assert float(tr["eps_s"]) == case["tau"] * float(tr["mu"])


def test_dm_duplicate_columns_never_accepted():
    """|theta| = 1 for equal columns: 1 < delta fails even at delta = 1."""
    a = np.array([1.0, 2.0, -1.0, 0.5])
    A = np.asfortranarray(np.stack([a, a, 2 * a], axis=1))
    r = O.qrdm(A, 0.1, 1.0, 3, max_steps=1)
    assert int(r["trace"][0]["k"]) == 1
    assert r["J"][0][0] == 2  # largest norm


def test_argmax_tie_goes_to_lowest_position():
    a = np.array([1.0, 0.0, 0.0])
    b = np.array([0.0, 1.0, 0.0])
    A = np.asfortranarray(np.stack([0.5 * a, b, a], axis=1))
    r = O.qrdm(A, 1.0, 0.0, 1, max_steps=1)
    assert r["J"][0][0] == 1


# ---------------------------------------------------------------- k_max = 1 is QRP
@pytest.mark.parametrize("seed", range(40))
def test_kmax1_is_column_pivoting(seed):
    """k_max = 1 must be QR with column pivoting (Alg. 2), checked against a
    brute-force pivot search that recomputes every residual norm."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(4, 17))
    m = int(rng.integers(max(2, n - 3), n + 12))
    A = np.asfortranarray(rng.standard_normal((m, n)) * rng.uniform(0.1, 3.0, n)[None, :])
    order, gaps = qrp_bruteforce(A)
    if np.min(gaps[: min(m, n) - 1]) < 1e-6:
        pytest.skip("near-tie in the exact pivot order")
    r = O.qrdm(A, 0.5, 0.5, 1)
    p = min(m, n)
    assert list(r["perm"][:p]) == order[:p]
    assert np.all(r["trace"]["k"] == 1) and np.all(r["trace"]["l"] == 1)
    # R is the R factor of A[:, perm] (unique up to row signs)
    R_ref = np.linalg.qr(A[:, r["perm"]], mode="r")
    np.testing.assert_allclose(np.abs(upper(r["A"])), np.abs(R_ref[:p]), atol=1e-13 * np.linalg.norm(A))


# ---------------------------------------------------------------- the whole factorization
CASES = [
    ("gap256", 0.9, 0.9, 32),
    ("gap256", 0.15, 0.9, 64),
    ("gap256", 0.5, 0.3, 8),
    ("gap256", 1.0, 1.0, 128),
    ("dense", 0.9, 0.9, 32),
    ("tall", 0.2, 0.95, 16),
    ("wide", 0.6, 0.8, 5),
]


def _case_matrix(name):
    if name == "gap256":
        return inputs.named("gap256").build()
    if name == "dense":
        return inputs.random_dense(120, 90, 5)
    if name == "tall":
        return inputs.from_spectrum(200, 70, inputs.sigma_geometric(70, 1e-12), 7)
    if name == "wide":
        return inputs.from_spectrum(60, 150, inputs.sigma_geometric(60, 1e-10), 8)
    raise ValueError(name)


@pytest.mark.parametrize("name,tau,delta,kmax", CASES)
def test_factorization_is_a_qr_of_the_permuted_matrix(name, tau, delta, kmax):
    """A Pi = Q R with Q orthogonal to 1e-13 (the stated acceptance bound), R
    upper triangular and equal (up to row signs) to the library R of A Pi."""
    A = _case_matrix(name)
    r = O.qrdm(A, tau, delta, kmax)
    assert r["status"] == 0
    perm = r["perm"]
    assert sorted(perm.tolist()) == list(range(A.shape[1]))
    res, orth = factorization_errors(A, r["A"], r["htau"], perm)
    assert res <= 1e-13
    assert orth <= 1e-13
    p = min(A.shape)
    R_ref = np.linalg.qr(A[:, perm], mode="r")[:p]
    np.testing.assert_allclose(np.abs(upper(r["A"])), np.abs(R_ref), atol=1e-13 * np.linalg.norm(A))
    tr = r["trace"]
    assert np.all(tr["l"] >= 1) and np.all(tr["l"] <= tr["k"]) and np.all(tr["k"] <= kmax)
    assert int(tr["l"].sum()) == p
    assert np.all(np.diff(tr["ns"]) == tr["l"][:-1])


def test_rank_gap_matrix():
    """256 x 256 with sigma = 1 (128 times) then 1e-14: the column-max form of
    the criterion (no sqrt(n - n_s) factor) gives 128; the paper's criterion
    (Sec. 3.4) is conservative and approaches eps*n*||A|| from below, so it
    stops later (Sec. 5 discusses the same over-estimate)."""
    A = inputs.named("gap256").build()
    r = O.qrdm(A, 0.9, 0.9, 32)
    assert r["rank_colmax"] == 128
    assert 128 <= r["rank"] <= 256
    d = np.abs(np.diag(r["A"]))
    assert d[:128].min() > 1e-3 and d[128:].max() < 1e-12


def criterion_diagonal() -> np.ndarray:
    """100 x 100 diagonal: 50 unit columns, then 50 of norm eta = 20 eps.
    Every reflector is the identity (zero tails), every downdate exact, and
    anorm = 1, eps1 = 100 eps exactly."""
    d = np.ones(100)
    d[50:] = 20.0 * EPS
    return np.asfortranarray(np.diag(d))


def test_rank_criterion_and_dm_safeguard_on_an_exact_diagonal():
    """The paper's stopping test sqrt(n - n_s) mu <= eps n max||a_i|| (Sec.
    3.4), taken at block starts, and the DM safeguard of Sec. 4 (reading R12:
    once the test holds, single-column steps finish).  With k_max = 8 the
    blocks start at 0, 8, ..., 40, 48 (the last unit pair), 50, 58, 66, 74, 82.
    At n_s = 50 the column maximum eta = 20 eps is already below 100 eps
    (rank_colmax = 50), but sqrt(50) eta = 141 eps is not; sqrt(26) eta =
    102 eps at n_s = 74 is not either; sqrt(18) eta = 85 eps at n_s = 82 is,
    so rank = 82, and the 18 columns left go one per step with DM off."""
    A = criterion_diagonal()
    r = O.qrdm(A, 0.9, 0.9, 8)
    assert r["rank_colmax"] == 50
    assert r["rank"] == 82
    tr = r["trace"]
    ns, k, dm = tr["ns"], tr["k"], tr["dm_on"]
    assert list(ns[:12]) == [0, 8, 16, 24, 32, 40, 48, 50, 58, 66, 74, 82]
    assert list(k[:11]) == [8, 8, 8, 8, 8, 8, 2, 8, 8, 8, 8]
    assert np.all(dm[:11] == 1)
    assert len(tr) == 11 + 18 and np.all(k[11:] == 1) and np.all(dm[11:] == 0)
    assert np.array_equal(r["perm"], np.arange(100))
    assert r["stop"] is None
    # stopping at the rank: 11 steps, then the stopping test's own record at
    # n_s = 82 with mu = eta exactly
    s = O.qrdm(A, 0.9, 0.9, 8, stop_at_rank=True)
    assert s["rank"] == 82 and len(s["trace"]) == 11
    assert np.array_equal(s["trace"], tr[:11])
    st = s["stop"]
    assert int(st["k"]) == -1 and int(st["ns"]) == 82 and float(st["mu"]) == 20.0 * EPS
    assert np.all(s["A"][82:, 82:] == A[82:, 82:]) and np.all(s["htau"][82:] == 0.0)


def test_rank_criterion_counts_all_n_minus_ns_columns_on_a_wide_matrix():
    """The criterion's factor is sqrt(n - n_s), the number of columns of R22
    (Sec. 3.4), not sqrt(min(m, n) - n_s).  The diagonal above with 40 zero
    columns appended (100 x 140): eps1 = 140 eps.  At n_s = 90, sqrt(50) eta
    = 141.4 eps does not pass; at n_s = 98, sqrt(42) eta = 129.6 eps does, so
    rank = 98 (with sqrt(100 - n_s) it would already pass at n_s = 58)."""
    A = np.asfortranarray(np.hstack([criterion_diagonal(), np.zeros((100, 40))]))
    r = O.qrdm(A, 0.9, 0.9, 8)
    assert r["rank"] == 98 and r["rank_colmax"] == 50
    tr = r["trace"]
    assert list(tr["ns"]) == [0, 8, 16, 24, 32, 40, 48, 50, 58, 66, 74, 82, 90, 98, 99]
    assert list(tr["k"]) == [8, 8, 8, 8, 8, 8, 2, 8, 8, 8, 8, 8, 8, 1, 1]
    assert list(tr["dm_on"]) == [1] * 13 + [0, 0]
    assert np.array_equal(r["perm"], np.arange(140))


def test_rank_exact_integer_matrices():
    for c in golden("exact_rank.json")["cases"]:
        A = np.asfortranarray(np.array(c["columns"]).T)
        for kmax in (1, 3):
            r = O.qrdm(A, 0.5, 0.9, kmax)
            assert r["rank"] == c["rank"], (c, kmax)


@pytest.mark.parametrize("kmax", [1, 16, 32])
def test_rank_geometric_bounds(kmax):
    """Geometric spectrum.  When the criterion holds at n_s, interlacing
    (eq. interlacing2) and the column bound eq. bound_largest_sv give
    sigma_{n_s+1}(A) <= ||R22|| <= sqrt(n - n_s) mu <= eps1 max||a_i|| <= eps1 sigma_1,
    so the rank is never below #{sigma_i > eps n sigma_1} (up to roundoff in
    R22), and the column-max form never below #{sigma_i > sqrt(n) eps n sigma_1}.
    The over-estimate is bounded softly by the paper's worst case (+45 %, Sec. 5)."""
    n = 300
    s = inputs.sigma_geometric(n, 1e-15)
    A = inputs.from_spectrum(n, n, s, 11)
    nr = int(np.sum(s > 2 * EPS * n * s[0]))
    nr_cm = int(np.sum(s > 2 * np.sqrt(n) * EPS * n * s[0]))
    r = O.qrdm(A, 0.9, 0.9, kmax)
    assert r["rank"] >= nr
    assert r["rank_colmax"] >= nr_cm
    assert r["rank"] >= r["rank_colmax"]
    assert r["rank"] <= 1.45 * nr + kmax


def test_eps1_sqrt_mode_is_stricter():
    """eps*sqrt(n) < eps*n, so the criterion holds later (Sec. 3.4 choices)."""
    A = inputs.named("gap256").build()
    r0 = O.qrdm(A, 0.9, 0.9, 32, eps1_mode=0)
    r1 = O.qrdm(A, 0.9, 0.9, 32, eps1_mode=1)
    assert r1["rank"] >= r0["rank"] and r1["rank_colmax"] >= r0["rank_colmax"]


def test_stop_at_rank_leaves_trailing_block():
    A = inputs.named("gap256").build()
    full = O.qrdm(A, 0.9, 0.9, 32)
    r = O.qrdm(A, 0.9, 0.9, 32, stop_at_rank=True)
    k = r["rank"]
    assert k == full["rank"]
    assert np.all(r["htau"][k:] == 0.0)
    assert int(r["trace"]["l"].sum()) == k
    # the first k columns of A Pi are still exactly Q_1 R_11 (+ R_12 block)
    Q = form_q(r["A"], r["htau"][:k], ncols=256)
    R = np.triu(r["A"][:k, :])
    R2 = r["A"][k:, k:]
    M = Q @ np.vstack([R, np.hstack([np.zeros((256 - k, k)), R2])])
    assert np.linalg.norm(A[:, r["perm"]] - M) <= 1e-13 * np.linalg.norm(A)


# ---------------------------------------------------------------- norm downdate
@pytest.mark.parametrize("steps", [1, 2, 5])
def test_partial_norms_track_exact_trailing_norms(steps):
    """After each step u_j approximates ||A[n_s:m, j]|| for the trailing
    columns (Sec. 3.1, 3.2 downdate); the error is bounded by the cancellation
    amplification (uref/u)^2 that triggers recomputation at sqrt(eps)."""
    A = inputs.from_spectrum(160, 120, inputs.sigma_geometric(120, 1e-13), 21)
    r = O.qrdm(A, 0.5, 0.95, 16, max_steps=steps)
    ns = int(r["trace"]["ns"][-1] + r["trace"]["l"][-1])
    exact = np.linalg.norm(r["A"][ns:, ns:], axis=0)
    u = r["u"][ns:]
    amp = (r["uref"][ns:] / u) ** 2
    rel = np.abs(u - exact) / exact
    assert np.all(rel <= 1e3 * EPS * amp + 1e-14)


def test_cancellation_triggers_recompute():
    """A column almost parallel to the pivot: its downdated norm would lose
    all digits, so it must be recomputed exactly (robust downdate, Sec. 3.1)."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal(30)
    b = a + 1e-9 * rng.standard_normal(30)
    c = rng.standard_normal(30) * 0.1
    A = np.asfortranarray(np.stack([a, b, c], axis=1))
    r = O.qrdm(A, 0.99, 0.1, 1, max_steps=1)
    tr = r["trace"][0]
    assert tr["nrecomp"] >= 1
    exact = np.linalg.norm(r["A"][1:, 1:], axis=0)
    np.testing.assert_allclose(r["u"][1:], exact, rtol=1e-13)


DOWNDATE_CASES = [
    ("geo 300x300 1e-15", lambda sd: inputs.from_spectrum(300, 300, inputs.sigma_geometric(300, 1e-15), sd), 0.15,
     0.9, 16, range(4)),
    ("geo 400x250 1e-12", lambda sd: inputs.from_spectrum(400, 250, inputs.sigma_geometric(250, 1e-12), sd), 0.5,
     0.9, 32, range(2)),
    ("kahan 300", lambda sd: inputs.kahan(300), 0.15, 0.9, 16, range(1)),
]


@pytest.mark.parametrize("case", DOWNDATE_CASES, ids=lambda c: c[0])
def test_partial_norms_stay_within_the_downdate_bound(case):
    """A bound that does not use the oracle's own uref.  A partial norm
    carries an absolute error of about sqrt(m) eps uref (inner products of
    length m); the downdate amplifies it by (uref/u)^2 relative to u, and the
    recompute test (Sec. 3.1, t (u/uref)^2 > sqrt(eps) to keep a downdate)
    holds that factor below 1/sqrt(eps).  So at every block-step start each
    partial norm is within sqrt(m eps) relative of the true norm of its
    column of R22, computed here from the trailing block itself."""
    _, build, tau, delta, kmax, seeds = case
    for sd in seeds:
        A = build(sd)
        m = A.shape[0]
        for steps in (3, 6, 10, 15, 20, 30):
            r = O.qrdm(A, tau, delta, kmax, max_steps=steps)
            ns = int(r["trace"]["l"].sum())
            if ns >= min(A.shape):
                break
            true = np.linalg.norm(r["A"][ns:, ns:], axis=0)
            rel = np.abs(r["u"][ns:] - true) / true
            assert rel.max() <= np.sqrt(m * EPS), (sd, steps, ns, rel.max())
            assert np.all(r["u"][:ns] == 0.0)  # factored columns carry no partial norm


def test_recompute_test_at_its_threshold_recomputes():
    """Reading R9 (the robust downdate of Sec. 3.1): the norm is recomputed
    when t (u/uref)^2 <= sqrt(eps), equality included.  An exact case: four
    unit pivots of norms 4, 3.5, 3, 2.5 (zero tails, so every reflector is the
    identity) and a column of norm exactly 1 whose entries in the pivot rows
    are (8191, 125, 26, 9) 2^-13, with 2^-13 below them.  Their squares add up
    to 1 - 2^-26 exactly (8191^2 + 125^2 + 26^2 + 9^2 = 2^26 - 1), so
    t = 2^-26 = sqrt(eps) exactly and uref = u: the test sits on its
    threshold.  The norm is recomputed (uref reset to the new 2^-13), and the
    column beside it, untouched by the pivots, is not.  Factored columns'
    partial norms are zero afterwards."""
    A = np.zeros((6, 6))
    A[0, 0], A[1, 1], A[2, 2], A[3, 3] = 4.0, 3.5, 3.0, 2.5
    A[:5, 4] = np.array([8191.0, 125.0, 26.0, 9.0, 1.0]) * 2.0 ** -13
    A[5, 5] = 0.5
    assert np.linalg.norm(A[:, 4]) == 1.0
    r = O.qrdm(np.asfortranarray(A), 0.5, 0.9, 4, max_steps=1)
    tr = r["trace"][0]
    assert (int(tr["k"]), int(tr["l"]), int(tr["nrecomp"])) == (4, 4, 1)
    assert np.array_equal(r["perm"], np.arange(6))
    assert r["u"][4] == 2.0 ** -13 and r["uref"][4] == 2.0 ** -13
    assert r["u"][5] == 0.5 and r["uref"][5] == 0.5
    assert np.all(r["u"][:4] == 0.0)


# ---------------------------------------------------------------- theorems (SDD mode)
def _sdd_run(A, tau, kmax):
    r = O.qrdm(A, tau, 1.0, kmax, sdd=True, no_break=True)
    assert r["status"] == 0
    return r


@pytest.mark.parametrize("cos,accepted", [(0.35, True), (0.6, False)])
def test_sdd_delta_divides_tau_squared_by_the_candidate_count(cos, accepted):
    """eq. delta_max with reading R18: delta_s = min(delta, tau^2 / |I|), |I|
    the candidates other than the pivot (eq. def_candidate_set), so that the
    k - 1 <= |I| off-diagonal cosines of a row add up to less than tau^2.
    Pivot e1, candidates of norms 0.95 (cosine `cos` with the pivot) and 0.92
    (orthogonal to both), tau = 0.9: |I| = 2 and delta_s = 0.405.  A cosine of
    0.35 passes (it would not under tau^2 / (|I| + 1) = 0.27); 0.6 does not
    (it would under tau^2 / (|I| - 1) = 0.81)."""
    A = np.zeros((4, 4))
    A[0, 0] = 1.0
    A[:2, 1] = 0.95 * np.array([cos, np.sqrt(1.0 - cos * cos)])
    A[2, 2] = 0.92
    A[3, 3] = 0.1
    r = O.qrdm(np.asfortranarray(A), 0.9, 0.9, 4, sdd=True, no_break=True, max_steps=1)
    tr = r["trace"][0]
    assert int(tr["ncand"]) == 2
    assert list(r["J"][0][: int(tr["k"])]) == ([0, 1, 2] if accepted else [0, 2])


@pytest.mark.parametrize("seed", range(4))
def test_lemma1_lemma2_theorem_sdd(seed):
    """With delta <= tau^2/|I| (eq. delta_max) every DM block satisfies Lemma 1;
    Lemma 2 and the QRDM worst-case bound (Sec. 3.3) hold at every step."""
    m, n = 60, 40
    s = inputs.sigma_geometric(n, 1e-6)
    A = inputs.from_spectrum(m, n, s, 100 + seed)
    tau = 0.7
    r = _sdd_run(A, tau, 8)
    R = upper(r["A"])
    sv = np.linalg.svd(A, compute_uv=False)
    prev_sig = None
    for rec in r["trace"]:
        ns, k = int(rec["ns"]), int(rec["k"])
        if not rec["dm_on"]:
            break
        Tb = R[ns:ns + k, ns:ns + k]
        dn = np.linalg.norm(Tb, axis=0)
        Th = (Tb / dn).T @ (Tb / dn)
        gamma = min(1.0 - (np.sum(np.abs(Th[i])) - 1.0) for i in range(k))
        assert gamma > 1 - tau ** 2 - 1e-12
        c1 = abs(Tb[0, 0])
        smin_T = np.linalg.svd(Tb, compute_uv=False)[-1]
        lam = np.sqrt(max(gamma + tau ** 2 - 1, 0.0))
        assert smin_T >= lam * c1 * (1 - 1e-9)  # Lemma 1
        n1 = ns + k
        assert smin_T >= lam / np.sqrt(n - n1 + 1) * sv[n1 - 1] * (1 - 1e-9)  # Lemma 2
        sig = np.linalg.svd(R[:n1, :n1], compute_uv=False)[-1]
        if prev_sig is not None and n - n1 > 0:
            bound = sv[n1 - 1] * prev_sig / sv[0] / np.sqrt(2 * (n - n1) * n1) * lam / (k ** 2 * ns)
            assert sig >= bound * (1 - 1e-9)  # Theorem (QRDM bound)
        prev_sig = sig


def test_qrp_theorem_bound():
    """Column pivoting bound (Sec. 3.3, theorem quoted from Chandrasekaran & Ipsen)."""
    n = 40
    A = inputs.from_spectrum(50, n, inputs.sigma_geometric(n, 1e-8), 77)
    r = O.qrdm(A, 0.9, 0.9, 1)
    R = upper(r["A"])
    sv = np.linalg.svd(A, compute_uv=False)
    sig = [np.linalg.svd(R[:s, :s], compute_uv=False)[-1] for s in range(1, n + 1)]
    for s in range(1, n - 1):
        bound = sv[s] * sig[s - 1] / sv[0] / np.sqrt(2 * (n - s) * (s + 1))
        assert sig[s] >= bound * (1 - 1e-9)


# ---------------------------------------------------------------- optimality on tiny inputs
@pytest.mark.parametrize("seed", range(3))
def test_subset_optimality_tiny(seed):
    """sigma_min(R11) equals sigma_min of the chosen columns and can not exceed
    the best r-subset (eq. NPhard, interlacing eq. interlacing1)."""
    m, n, rk = 12, 10, 5
    s = np.concatenate([[1.0, 0.6, 0.3, 0.1, 0.05], np.full(5, 1e-14)])
    A = inputs.from_spectrum(m, n, s, 300 + seed)
    best = max(np.linalg.svd(A[:, list(S)], compute_uv=False)[-1] for S in itertools.combinations(range(n), rk))
    for kmax, tau in ((1, 0.9), (4, 0.5), (8, 0.15)):
        r = O.qrdm(A, tau, 0.9, kmax)
        R11 = upper(r["A"])[:rk, :rk]
        s11 = np.linalg.svd(R11, compute_uv=False)[-1]
        sS = np.linalg.svd(A[:, r["perm"][:rk]], compute_uv=False)[-1]
        assert s11 == pytest.approx(sS, rel=1e-10)
        assert s11 <= best * (1 + 1e-12)
        assert s11 <= s[rk - 1] * (1 + 1e-12)
        assert s11 >= 1e-2 * best


# ---------------------------------------------------------------- edge cases
def test_invalid_arguments():
    A = np.eye(3, order="F")
    assert O.qrdm(A, 0.0, 0.5, 4)["status"] == -5
    assert O.qrdm(A, 1.5, 0.5, 4)["status"] == -5
    assert O.qrdm(A, 0.5, -0.1, 4)["status"] == -6
    assert O.qrdm(A, 0.5, 0.5, 0)["status"] == -7


def test_nonfinite_input():
    A = np.eye(3, order="F")
    A[1, 2] = np.nan
    assert O.qrdm(A, 0.5, 0.5, 2)["status"] == 1


@pytest.mark.parametrize("m,n", [(0, 0), (0, 4), (5, 0), (1, 1), (1, 6), (6, 1)])
def test_degenerate_shapes(m, n):
    A = np.asfortranarray(np.arange(1, m * n + 1, dtype=np.float64).reshape(m, n) if m * n else np.zeros((m, n)))
    r = O.qrdm(A, 0.5, 0.5, 4)
    assert r["status"] == 0
    assert sorted(r["perm"].tolist()) == list(range(n))
    if m and n:
        res, orth = factorization_errors(A, r["A"], r["htau"], r["perm"])
        assert res <= 1e-14 and orth <= 1e-14
    assert r["rank"] == min(m, n) or (m * n == 0 and r["rank"] == 0)


def test_no_break_mode_takes_whole_block():
    A = inputs.named("gap256").build()
    r = O.qrdm(A, 0.9, 0.9, 32, no_break=True)
    assert np.all(r["trace"]["l"] == r["trace"]["k"])


def test_ls_basic_square_full_rank_is_the_linear_solve():
    A = inputs.random_dense(60, 60, 3)
    b = np.random.default_rng(4).standard_normal(60)
    x = O.ls_basic(A, b, tau=0.5, delta=0.9, k_max=8)
    ref = np.linalg.solve(A, b)
    cond = np.linalg.cond(A)
    assert np.linalg.norm(x - ref) <= 50 * cond * 2.0 ** -52 * np.linalg.norm(ref)


def test_ls_basic_tall_full_rank_is_the_least_squares_solution():
    A = inputs.random_dense(120, 40, 5)
    B = np.random.default_rng(6).standard_normal((120, 3))
    X = O.ls_basic(A, B, tau=0.15, delta=0.9, k_max=16)
    ref = np.linalg.lstsq(A, B, rcond=None)[0]
    np.testing.assert_allclose(X, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_ls_basic_rank_deficient_compatible_system_is_solved():
    """A of rank 25 (sigma 1 then 1e-15), b = A x0: the basic solution with
    r = 25 reproduces b to roundoff and has at most 25 nonzeros."""
    A = inputs.from_spectrum(90, 70, inputs.sigma_gap(70, 25, lo=1e-15), 7)
    x0 = np.random.default_rng(8).standard_normal(70)
    b = A @ x0
    x = O.ls_basic(A, b, rank=25, tau=0.9, delta=0.9, k_max=32)
    assert np.count_nonzero(x) <= 25
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_ls_basic_incompatible_rank_deficient_is_the_lstsq_on_the_pivot_columns():
    """The basic solution x = Pi [R11^-1 (Q^T b)_{1:r}; 0] is, by definition,
    the least-squares solution restricted to the r pivot columns: for an
    incompatible right-hand side it equals the library least-squares
    solution of A[:, perm[:r]] scattered back, and its residual is
    orthogonal to those columns."""
    A = inputs.from_spectrum(90, 70, inputs.sigma_gap(70, 25, lo=1e-15), 9)
    b = np.random.default_rng(10).standard_normal(90)
    f = O.qrdm(A, 0.9, 0.9, 32)
    x = O.ls_basic(A, b, rank=25, fact=f)
    sel = f["perm"][:25]
    ref = np.zeros(70)
    ref[sel] = np.linalg.lstsq(A[:, sel], b, rcond=None)[0]
    cond = np.linalg.cond(A[:, sel])
    np.testing.assert_allclose(x, ref, rtol=0, atol=100 * cond * 2.0 ** -52 * np.abs(ref).max())
    assert np.linalg.norm(A[:, sel].T @ (b - A @ x)) <= 1e-12 * np.linalg.norm(b) * np.linalg.norm(A[:, sel])


# ---------------------------------------------------------------- OpenMP build
@pytest.mark.parametrize("kind", ["gap", "geo", "kahan"])
def test_openmp_build_gives_the_same_bits(kind):
    """The OpenMP build (timed as the all-cores CPU baseline) spreads only the
    trailing update's independent column loops over threads, each column
    summed in the same order, so every output is bit-identical to the
    single-threaded build's."""
    if O.build_omp() is None:
        pytest.skip("the C compiler has no OpenMP")
    A = {"gap": lambda: inputs.from_spectrum(400, 300, inputs.sigma_gap(300, 150), 2),
         "geo": lambda: inputs.from_spectrum(350, 350, inputs.sigma_geometric(350, 1e-15), 3),
         "kahan": lambda: inputs.kahan(300)}[kind]()
    a = O.qrdm(A, 0.15, 0.9, 32)
    b = O.qrdm(A, 0.15, 0.9, 32, parallel=True)
    for key in ("A", "htau", "perm", "u", "uref", "trace", "J"):
        assert np.array_equal(a[key], b[key]), key
    assert (a["rank"], a["rank_colmax"], a["nsteps"]) == (b["rank"], b["rank_colmax"], b["nsteps"])


# ---------------------------------------------------------------- metamorphic invariances
def _clear_everywhere(o, gap=1e-6):
    tr = o["trace"]
    gaps = np.min(np.stack([tr[f] for f in ("g_argmax", "g_cand", "g_cos", "g_break", "g_stop")]), axis=0)
    return bool(np.all(gaps > gap))


@pytest.mark.parametrize("kind", ["dense", "gap", "kahan"])
def test_scaling_by_a_power_of_two_scales_r_exactly(kind):
    """Every threshold of QRDM is relative: the candidate test tau mu, the
    cosines, the break test eps_s = tau mu, the downdate's ratios and the
    stopping test against eps1 max||a_i|| (Sec. 2, 3.4, Alg. 4).  Scaling A by
    2^k is exact in binary floating point, so every decision, every reflector
    and htau are the same bits, and R is scaled exactly."""
    A = {"dense": lambda: inputs.random_dense(90, 70, 1),
         "gap": lambda: inputs.from_spectrum(120, 100, inputs.sigma_gap(100, 40), 2),
         "kahan": lambda: inputs.kahan(80)}[kind]()
    o = O.qrdm(A, 0.3, 0.8, 16)
    for c in (2.0 ** 40, 2.0 ** -30):
        s = O.qrdm(c * A, 0.3, 0.8, 16)
        assert np.array_equal(s["perm"], o["perm"]) and np.array_equal(s["J"], o["J"])
        assert (s["rank"], s["rank_colmax"]) == (o["rank"], o["rank_colmax"])
        for f in ("k", "l", "ns", "dm_on", "nrecomp"):
            assert np.array_equal(s["trace"][f], o["trace"][f]), f
        assert np.array_equal(s["htau"], o["htau"])
        R_o, R_s = np.triu(o["A"]), np.triu(s["A"])
        assert np.array_equal(R_s, c * R_o)
        assert np.array_equal(s["A"] - R_s, o["A"] - R_o)  # reflector tails


def test_a_column_permutation_of_the_input_selects_the_same_columns():
    """The decisions depend on the columns, not on where they sit (positions
    only break exact ties, absent here): factoring A[:, pi] picks the same
    original columns in the same order, and each column's R entries are the
    same bits, since every column is updated on its own."""
    A = inputs.random_dense(80, 60, 3)
    o = O.qrdm(A, 0.5, 0.9, 8)
    assert _clear_everywhere(o)
    pi = np.random.default_rng(4).permutation(60)
    b = O.qrdm(A[:, pi], 0.5, 0.9, 8)
    assert np.array_equal(pi[b["perm"]], o["perm"])
    R_o = np.empty((60, 60))
    R_b = np.empty((60, 60))
    R_o[:, o["perm"]] = np.triu(o["A"][:60])
    R_b[:, pi[b["perm"]]] = np.triu(b["A"][:60])
    assert np.array_equal(R_b, R_o)


def test_a_left_orthogonal_factor_changes_no_decision():
    """Column norms and the Gram matrix of the trailing block are invariant
    under A -> U A with U orthogonal (the appendix's invariance of singular
    values under orthogonal factors), so QRDM on U A takes the same decisions
    and gives the same |R| up to rounding (R is unique up to row signs)."""
    rng = np.random.default_rng(5)
    for A in (inputs.random_dense(70, 50, 6), inputs.from_spectrum(70, 50, inputs.sigma_geometric(50, 1e-6), 7)):
        U = inputs.haar(70, 70, rng)
        o = O.qrdm(A, 0.3, 0.8, 8)
        b = O.qrdm(U @ A, 0.3, 0.8, 8)
        assert _clear_everywhere(o)
        assert np.array_equal(b["perm"], o["perm"]) and np.array_equal(b["J"], o["J"])
        np.testing.assert_allclose(np.abs(np.triu(b["A"][:50])), np.abs(np.triu(o["A"][:50])),
                                   rtol=1e-10, atol=1e-13 * np.abs(A).max())


@pytest.mark.parametrize("kmax", [1, 8, 32])
def test_inputs_that_need_no_pivoting_give_plain_householder_qr(kmax):
    """Orthogonal columns of strictly decreasing norm: every column is a
    candidate in position order, every cosine is 0, no residual falls below
    eps_s, so the permutation is the identity and R is the plain Householder
    R of A (the library's, up to row signs): here diag(d)."""
    Q = inputs.haar(60, 40, np.random.default_rng(8))
    d = 2.0 ** (-np.arange(40) / 8.0)
    A = np.asfortranarray(Q * d)
    o = O.qrdm(A, 0.01, 0.9, kmax)
    assert np.array_equal(o["perm"], np.arange(40))
    R = np.triu(o["A"][:40])
    Rlib = np.linalg.qr(A, mode="r")
    np.testing.assert_allclose(np.abs(R), np.abs(Rlib), atol=1e-14)
    np.testing.assert_allclose(np.abs(np.diag(R)), d, rtol=1e-13)
