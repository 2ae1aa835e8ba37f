"""Batched QRDM (one persistent launch over many uneven matrices) against the
CPU oracle: every matrix of the batch is compared with the oracle's
factorization of the same matrix under the tie-aware rules of the single-
matrix parity tests (identical decisions until a logged near-tie, |R_ii| and
htau within the perturbation bound), for every tuning the autotuner may pick,
through the direct launch and the CUDA-graph launch."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._helpers import factorization_errors
from tests._parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402


def _run(hosts, tau, delta, kmax, *, tuning=None, graph=False, **kw):
    mats = [q.colmajor(A) for A in hosts]
    plan = q.BatchPlan(mats, kmax, trace=True)
    if tuning is not None:
        plan.set_tuning(*tuning)
    opts = q.make_opts(**kw)
    plan.run(tau, delta, opts, graph=graph)
    res = plan.results()
    out = []
    for i, A in enumerate(mats):
        h, p = plan.outputs(i)
        tr, J = plan.trace(i, res.steps[i])
        out.append({"A": A.cpu().numpy(), "htau": h.cpu().numpy(), "perm": p.cpu().numpy().astype(np.int64),
                    "trace": tr, "J": J.astype(np.int64), "rank": int(res.rank[i]),
                    "rank_colmax": int(res.rank_colmax[i]), "status": int(res.status[i]),
                    "nsteps": int(res.steps[i])})
    plan.close()
    return out


def _check(hosts, got, tau, delta, kmax, **kw):
    reports = []
    for A, g in zip(hosts, got):
        assert g["status"] == 0
        o = O.qrdm(A, tau, delta, kmax, **kw)
        rep = compare(A, g, o)
        reports.append(rep)
        if A.size:
            res, orth = factorization_errors(A, g["A"], g["htau"], g["perm"])
            assert res <= 1e-13 and orth <= 1e-13, (A.shape, res, orth)
    return reports


def _small_batch(count, seed, m_hi=300):
    ents = inputs.batch_entries(count, seed=seed, m_lo=16, m_hi=m_hi, n_lo=8)
    return [e.build() for e in ents]


@pytest.mark.parametrize("tau,delta,kmax", [(0.15, 0.9, 64), (0.9, 0.9, 32), (0.5, 0.5, 8), (0.15, 0.9, 1)])
def test_batched_matches_oracle_per_matrix(tau, delta, kmax):
    hosts = _small_batch(40, seed=11)
    got = _run(hosts, tau, delta, kmax)
    reps = _check(hosts, got, tau, delta, kmax)
    n_div = sum(r["diverged_at"] is not None for r in reps)
    print(f"\n[batched] tau {tau} delta {delta} kmax {kmax}: {len(reps)} matrices, {n_div} with a tie-divergence")


@pytest.mark.parametrize("tuning", [(1, 1024, 8), (1, 512, 4), (2, 512, 8), (2, 256, 4), (1, 64, 8)])
def test_every_tuning_gives_the_oracle_result(tuning):
    hosts = _small_batch(24, seed=5, m_hi=700)
    got = _run(hosts, 0.15, 0.9, 64, tuning=tuning)
    _check(hosts, got, 0.15, 0.9, 64)


def test_options_are_honoured():
    hosts = _small_batch(16, seed=3)
    for kw in ({"eps1_mode": 1}, {"stop_at_rank": True}, {"check_last": True}, {"no_break": True},
               {"sdd": True}):
        got = _run(hosts, 0.3, 0.8, 16, **kw)
        for A, g in zip(hosts, got):
            o = O.qrdm(A, 0.3, 0.8, 16, **kw)
            compare(A, g, o)


def test_edge_shapes_nonfinite_and_structured_in_one_batch():
    rng = np.random.default_rng(0)
    hosts = [
        np.zeros((0, 5)),
        np.zeros((5, 0)),
        np.asfortranarray(rng.standard_normal((1, 1))),
        np.asfortranarray(rng.standard_normal((7, 19))),                 # wide
        inputs.kahan(96),
        np.zeros((40, 30), order="F"),                                      # zero matrix
        np.asfortranarray(np.repeat(rng.standard_normal((50, 1)), 20, 1)),  # rank 1, equal norms
        inputs.random_dense(130, 129, 4),
        inputs.from_spectrum(200, 64, inputs.sigma_gap(64, 17), 9),
    ]
    bad = inputs.random_dense(33, 12, 1)
    bad[5, 7] = np.nan
    hosts_all = hosts + [bad]
    got = _run(hosts_all, 0.5, 0.9, 16)
    _check(hosts, got[:-1], 0.5, 0.9, 16)
    g = got[-1]
    assert g["status"] == 1 and g["rank"] == -1
    np.testing.assert_array_equal(np.isnan(g["A"]), np.isnan(bad))
    assert np.array_equal(g["A"][~np.isnan(bad)], bad[~np.isnan(bad)])


def test_graph_launch_replays_the_direct_launch_bit_for_bit():
    hosts = _small_batch(20, seed=8)
    direct = _run(hosts, 0.15, 0.9, 64)
    mats = [q.colmajor(A) for A in hosts]
    plan = q.BatchPlan(mats, 64)
    for rep in range(2):  # the second call replays the captured graph
        for t, A in zip(mats, hosts):
            t.copy_(torch.from_numpy(np.asfortranarray(A)).t().contiguous().t())
        plan.run(0.15, 0.9, graph=True)
        res = plan.results()
        for i, (t, d) in enumerate(zip(mats, direct)):
            assert np.array_equal(t.cpu().numpy(), d["A"]), (rep, i)
            assert np.array_equal(plan.outputs(i)[1].cpu().numpy(), d["perm"]), (rep, i)
            assert res.rank[i] == d["rank"] and res.steps[i] == d["nsteps"]
    plan.close()


def test_autotune_restores_the_inputs_and_picks_a_feasible_tuning():
    hosts = _small_batch(30, seed=2, m_hi=500)
    mats = [q.colmajor(A) for A in hosts]
    plan = q.BatchPlan(mats, 64)
    best, ms = plan.autotune(0.15, 0.9)
    assert ms > 0
    assert best == plan.tuning
    assert best["lanes_per_col"] in (4, 8) and 1 <= best["ctas_per_sm"] <= 2
    for t, A in zip(mats, hosts):
        assert np.array_equal(t.cpu().numpy(), A)
    plan.run(0.15, 0.9)
    res = plan.results()
    for i, A in enumerate(hosts):
        o = O.qrdm(A, 0.15, 0.9, 64)
        h, p = plan.outputs(i)
        g = {"A": mats[i].cpu().numpy(), "htau": h.cpu().numpy(), "perm": p.cpu().numpy().astype(np.int64),
             "rank": int(res.rank[i]), "rank_colmax": int(res.rank_colmax[i])}
        # no trace here: where the oracle logged no near-tie the permutation is exact
        if min(float(o["trace"][f].min()) for f in ("s_argmax", "s_cand", "s_order", "s_cos", "s_break",
                                                     "s_stop", "s_recomp")) >= 1.0:
            assert np.array_equal(g["perm"], o["perm"]), i
            assert g["rank"] == o["rank"]
    plan.close()


def test_tuning_feasibility_is_checked():
    mats = [q.colmajor(inputs.random_dense(64, 40, 0))]
    plan = q.BatchPlan(mats, 128)
    with pytest.raises(q.QRDMError):
        plan.set_tuning(3, 512, 8)  # more CTAs than the cap
    with pytest.raises(q.QRDMError):
        plan.set_tuning(1, 500, 8)  # not a multiple of 64
    with pytest.raises(q.QRDMError):
        plan.set_tuning(2, 1024, 8)  # two such CTAs do not fit on an SM
    plan.close()


def test_full_size_sample_of_the_uneven_batch():
    """The largest shapes of the 2000-matrix workload (m up to 1024), in a
    batch with a spread of smaller ones, every matrix against the oracle."""
    ents = inputs.batch_entries(2000, seed=0)
    big = sorted(ents, key=lambda e: e.m * e.n * min(e.m, e.n), reverse=True)[:3]
    pick = big + ents[:9]
    hosts = [e.build() for e in pick]
    got = _run(hosts, 0.15, 0.9, 64)
    reps = _check(hosts, got, 0.15, 0.9, 64)
    # the criterion never reports a rank below the spectrum's gap (it may
    # report more where roundoff in the trailing columns exceeds eps*n*||A||)
    for e, g in zip(pick, got):
        assert e.rank <= g["rank_colmax"] <= min(e.m, e.n), (e, g["rank_colmax"])
    print("\n[batched] full-size sample:", [(e.m, e.n, e.rank, g["rank"], g["rank_colmax"]) for e, g in zip(pick, got)],
          "divergences", [r["diverged_at"] for r in reps])


def test_equality_edges_in_the_batched_kernel():
    """The hand-derived equality edges of tests/golden/dm_equality.json
    (candidate u = tau mu admitted, residual = eps_s does not break, equal
    norms in position order) in the batched kernel's own selection and panel
    code: each case's first step equals the golden decisions."""
    from tests._helpers import golden
    from tests.test_oracle_pins import dm_equality_matrix

    for case in golden("dm_equality.json")["cases"]:
        A = dm_equality_matrix(case["matrix"])
        (g,) = _run([A], case["tau"], case["delta"], case["k_max"], check_last=case["check_last"])
        tr = g["trace"][0]
        assert int(tr["ncand_all"]) == case["ncand_all"], case["why"]
        assert int(tr["k"]) == case["k"] and int(tr["l"]) == case["l"], case["why"]
        assert list(g["J"][0][: case["k"]]) == case["J"], case["why"]
        _check([A], [g], case["tau"], case["delta"], case["k_max"], check_last=case["check_last"])
