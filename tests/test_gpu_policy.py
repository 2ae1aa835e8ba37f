"""The learned (tau, delta) policy on the GPU, against the oracles:

* the MLP's forward pass, loss gradient and Adam step (library kernels)
  against the numpy FP64 oracle MLP on the same BF16 weights;
* the in-kernel inference of a factorization against the oracle MLP on the
  features the kernel logged, and those features against features computed
  from the CPU oracle's partial norms;
* a factorization with the learned policy against the CPU oracle replaying
  the per-step (tau, delta) the policy chose (same tie-aware rule as the
  plain parity tests), in the single-matrix and the batched form;
* the guard, and what a trained network gains over fixed (0.9, 0.9)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._parity import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402
from paper_2106_03138_gb300 import policy as P  # noqa: E402


def _policy_with(w32: np.ndarray, **kw) -> P.Policy:
    pol = P.Policy(**kw)
    pol.load_weights(w32)
    torch.cuda.synchronize()
    # the device's BF16 copy is the oracle's rounding of the same values
    got = pol.w16.view(torch.int16).cpu().numpy().view(np.uint16)
    assert np.array_equal(got, M.bf16_bits(np.asarray(w32, np.float32)))
    return pol


def _w_bf16(w32):
    return M.bf16_round(np.asarray(w32, np.float32)).astype(np.float64)


def test_forward_gradient_and_adam_match_the_oracle():
    rng = np.random.default_rng(0)
    w32 = (rng.standard_normal(M.NPARAM) * 0.2).astype(np.float32)
    pol = _policy_with(w32)
    x = rng.standard_normal((300, 16)).astype(np.float32)
    t = rng.uniform(0, 1, (300, 2)).astype(np.float32)
    wb = _w_bf16(w32)
    y = pol.forward(x)
    yo, _ = M.forward(wb, x.astype(np.float64))
    assert np.max(np.abs(y - yo)) <= 2e-6
    L, g = pol.loss_grad(x, t)
    Lo, go = M.loss_grad(wb, x.astype(np.float64), t.astype(np.float64))
    assert L == pytest.approx(Lo, rel=2e-5)
    scale = np.max(np.abs(go))
    err = np.max(np.abs(g - go))
    assert err <= 1e-4 * scale, (err, scale)
    # one Adam step on the device against the oracle's
    lib = q.load()
    m = torch.zeros(M.NPARAM, dtype=torch.float32, device="cuda")
    v = torch.zeros_like(m)
    gd = torch.as_tensor(g, device="cuda")
    rc = lib.qrdm_mlp_adam_step(pol.w32.data_ptr(), pol.w16.data_ptr(), gd.data_ptr(), m.data_ptr(), v.data_ptr(), 1,
                                1e-3, 0.9, 0.999, 1e-8, 1e-2, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    w1o, m1o, v1o = M.adam_step(w32.astype(np.float64), g.astype(np.float64), np.zeros(M.NPARAM),
                                np.zeros(M.NPARAM), 1, 1e-3, wd=1e-2)
    np.testing.assert_allclose(pol.w32.cpu().numpy(), w1o, rtol=0, atol=2e-7)
    np.testing.assert_allclose(m.cpu().numpy(), m1o, rtol=1e-6, atol=1e-12)


def test_training_kernels_reduce_the_loss_on_a_learnable_target():
    """Targets that are a smooth function of the inputs: Adam on the
    library's kernels must fit them."""
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 1, (4096, 16)).astype(np.float32)
    T = np.stack([0.2 + 0.6 * X[:, 0] * X[:, 1], 0.5 + 0.4 * np.sin(3 * X[:, 2])], axis=1).astype(np.float32)
    pol = P.Policy(seed=7)
    L0 = pol.loss_grad(X[:1024], T[:1024])[0]
    loss = pol.train(X, T, steps=600, batch=512, lr=3e-3, seed=3)
    L1 = pol.loss_grad(X[:1024], T[:1024])[0]
    assert np.all(np.isfinite(loss))
    assert L1 < 0.2 * L0, (L0, L1)
    # deterministic: the same run twice gives the same weights
    pol2 = P.Policy(seed=7)
    pol2.train(X, T, steps=600, batch=512, lr=3e-3, seed=3)
    assert torch.equal(pol.w32, pol2.w32)


def _factor_with_policy(A, pol, tau=0.9, delta=0.9, kmax=32):
    m, n = A.shape
    dA = q.colmajor(A)
    cap = min(m, n) + 1
    fl = torch.zeros((cap, 16), dtype=torch.float32, device="cuda")
    al = torch.zeros((cap, 2), dtype=torch.float64, device="cuda")
    st = pol.struct(feat_log=fl, act_log=al)
    f = q.factor(dA, tau, delta, kmax, trace=True, policy=st)
    torch.cuda.synchronize()
    g = {"A": dA.cpu().numpy(), "htau": f.htau.cpu().numpy(), "perm": f.perm.cpu().numpy().astype(np.int64),
         "trace": f.trace, "J": f.J.astype(np.int64), "rank": f.rank, "rank_colmax": f.rank_colmax}
    return g, fl[:f.nsteps].cpu().numpy(), al[:f.nsteps].cpu().numpy()


def _random_policy(seed, tau_bias=0.0):
    """Random weights, guard off (rho_min = 0): every DM step uses the MLP."""
    rng = np.random.default_rng(seed)
    w32 = (rng.standard_normal(M.NPARAM) * 0.15).astype(np.float32)
    w32[-2] += tau_bias
    return _policy_with(w32, rho_min=0.0), w32


@pytest.mark.parametrize("seed,shape", [(1, (300, 220)), (2, (256, 256)), (3, (500, 130))])
def test_learned_factorization_replays_on_the_oracle(seed, shape):
    m, n = shape
    A = inputs.from_spectrum(m, n, inputs.sigma_rank_geometric(min(m, n), min(m, n) * 2 // 3), 40 + seed)
    pol, w32 = _random_policy(seed, tau_bias=-1.0)
    g, feats, acts = _factor_with_policy(A, pol)
    dm = g["trace"]["dm_on"] == 1
    # the kernel's (tau_s, delta_s) are the oracle MLP's on the logged features
    yo, _ = M.forward(_w_bf16(w32), feats[dm].astype(np.float64))
    to, do = M.to_tau_delta(yo, *P.TAU_RANGE, *P.DELTA_RANGE)
    assert np.max(np.abs(acts[dm, 0] - to)) <= 1e-5
    assert np.max(np.abs(acts[dm, 1] - do)) <= 1e-5
    assert np.unique(np.round(acts[dm, 0], 6)).size > 1  # the schedule really varies
    # the oracle replaying the schedule takes the same decisions
    o = O.qrdm(A, 0.9, 0.9, 32, schedule=acts)
    rep = compare(A, g, o)
    print(f"\n[policy] {shape}: {int(dm.sum())} learned steps, tau in [{acts[dm,0].min():.3f}, "
          f"{acts[dm,0].max():.3f}], diverged at {rep['diverged_at']}")


def test_logged_features_match_the_oracles_partial_norms():
    A = inputs.from_spectrum(260, 200, inputs.sigma_rank_geometric(200, 150), 9)
    pol, _ = _random_policy(4, tau_bias=-0.5)
    g, feats, acts = _factor_with_policy(A, pol)
    tr = g["trace"]
    anorm = float(np.max(np.linalg.norm(A, axis=0)))
    checked = 0
    for s in range(min(len(tr), 8)):
        if tr["dm_on"][s] != 1:
            break
        if s == 0:
            u = np.linalg.norm(A, axis=0)
        else:
            # the oracle's partial norms at the start of step s
            o = O.qrdm(A, 0.9, 0.9, 32, schedule=acts, max_steps=s)
            if o["nsteps"] != s or int(o["trace"]["ns"][-1] + o["trace"]["l"][-1]) != int(tr["ns"][s]):
                break  # the two sides diverged (a tie); stop comparing
            u = o["u"]
        ns = int(tr["ns"][s])
        jstar = ns + int(np.argmax(u[ns:]))
        prev_l = float(tr["l"][s - 1]) if s else 0.0
        prev_k = float(tr["k"][s - 1]) if s else 0.0
        prev_tau = float(acts[s - 1, 0]) if s else 0.0
        fo = M.step_features(u, ns, jstar, anorm, prev_l, prev_k, feats[s, 13], feats[s, 14], prev_tau)
        # counts at the eight thresholds: equal up to one column at a threshold tie
        assert np.max(np.abs(feats[s, :8] - fo[:8])) <= 1.0 / 128 + 1e-7, (s, feats[s, :8], fo[:8])
        np.testing.assert_allclose(feats[s, 8:13], fo[8:13], rtol=1e-5, atol=1e-6)
        assert feats[s, 15] == pytest.approx(fo[15], abs=1e-6)
        assert 0.0 <= feats[s, 13] <= feats[s, 14] <= 1.0 + 1e-6
        checked += 1
    assert checked >= 3


def test_smin_estimate_matches_the_singular_values():
    """The inverse power iteration used for label quality against the
    library SVD of the same R11 blocks."""
    rng = np.random.default_rng(8)
    mats, ranks = [], []
    for n, r in ((70, 50), (130, 128), (64, 1), (200, 150)):
        A = inputs.from_spectrum(n, n, inputs.sigma_geometric(n, 1e-8), int(rng.integers(1000)))
        Rq = np.linalg.qr(A, mode="r")
        mats.append(torch.as_tensor(np.asfortranarray(Rq), device="cuda"))
        ranks.append(r)
    est = P.smin_r11(mats, ranks, iters=60)
    for M_, r, e in zip(mats, ranks, est):
        exact = np.linalg.svd(np.triu(M_[:r, :r].cpu().numpy()), compute_uv=False)[-1]
        assert e == pytest.approx(exact, rel=0.05), (r, e, exact)


def test_guard_turns_the_policy_off():
    A = inputs.from_spectrum(300, 300, inputs.sigma_geometric(300, 1e-15), 11)
    rng = np.random.default_rng(5)
    w32 = (rng.standard_normal(M.NPARAM) * 0.01).astype(np.float32)
    w32[-2] = -30.0  # tau_s -> tau_lo for every step
    rho = 0.9
    pol = _policy_with(w32, rho_min=rho)
    g, feats, acts = _factor_with_policy(A, pol, tau=0.9, delta=0.9)
    tr = g["trace"]
    dm = np.nonzero(tr["dm_on"] == 1)[0]
    assert acts[dm[0], 0] == pytest.approx(P.TAU_RANGE[0], abs=1e-6)
    # some later DM step runs with the fixed (0.9, 0.9) again, and all after it
    fixed = np.nonzero((acts[dm, 0] == 0.9) & (acts[dm, 1] == 0.9))[0]
    assert fixed.size > 0
    k = int(fixed[0])
    assert k >= 1 and np.all(acts[dm[k:], 0] == 0.9)
    # the switch follows the first learned step whose smallest accepted pivot
    # |R_ii| is below rho times the largest partial norm left after it (the
    # next step's mu); every earlier learned step stayed above that bound
    d = np.abs(np.diag(g["A"]))
    for j in range(k):
        s = int(dm[j])
        mb = d[int(tr["ns"][s]):int(tr["ns"][s] + tr["l"][s])].min()
        bound = rho * float(tr["mu"][s + 1])
        assert (mb < bound) if j == k - 1 else (mb >= bound), (j, k, mb, bound)
    o = O.qrdm(A, 0.9, 0.9, 32, schedule=acts)
    compare(A, g, o)
    # with rho_min = 0 the policy is never switched off
    pol0 = _policy_with(w32, rho_min=0.0)
    g0, _, acts0 = _factor_with_policy(A, pol0, tau=0.9, delta=0.9)
    dm0 = np.nonzero(g0["trace"]["dm_on"] == 1)[0]
    assert np.all(np.abs(acts0[dm0, 0] - P.TAU_RANGE[0]) < 1e-6)
    assert len(acts0) < len(acts)  # the smallest tau all along takes fewer, larger blocks


def test_batched_learned_matches_oracle_replay():
    ents = inputs.batch_entries(24, seed=3, m_lo=32, m_hi=300, n_lo=16)
    hosts = [e.build() for e in ents]
    pol, _ = _random_policy(6, tau_bias=-1.0)
    mats = [q.colmajor(A) for A in hosts]
    plan = q.BatchPlan(mats, 32, trace=True, policy_logs=True)
    st = pol.struct()
    plan.run(0.9, 0.9, q.make_opts(policy=st))
    res = plan.results()
    for i, A in enumerate(hosts):
        tr, J = plan.trace(i, res.steps[i])
        f, a = plan.policy_logs(i, res.steps[i])
        h, p = plan.outputs(i)
        g = {"A": mats[i].cpu().numpy(), "htau": h.cpu().numpy(), "perm": p.cpu().numpy().astype(np.int64),
             "trace": tr, "J": J.astype(np.int64), "rank": int(res.rank[i]), "rank_colmax": int(res.rank_colmax[i])}
        o = O.qrdm(A, 0.9, 0.9, 32, schedule=a)
        compare(A, g, o)
    plan.close()


def test_trained_policy_gains_over_fixed_tau_delta():
    """Train on plain-QRDM sweeps of small generated matrices, then factor
    held-out matrices: fewer block steps than fixed (0.9, 0.9) at rank quality
    sigma_min(R11) / sigma_r within a factor 2."""
    train = P.training_entries(150, seed=21, n_lo=64, n_hi=320)
    pristine = [e.build_gpu() for e in train]
    X, T, info = P.collect(train, pristine)
    assert X.shape[0] >= 1000
    pol = P.Policy(seed=2)
    loss = pol.train(X, T, steps=1500, batch=1024, lr=2e-3)
    assert loss[-50:].mean() < loss[:50].mean()
    held = P.training_entries(60, seed=99, n_lo=64, n_hi=320)
    hp = [e.build_gpu() for e in held]
    fixed = P.run_batch(hp, held, 0.9, 0.9)
    learned = P.run_batch(hp, held, 0.9, 0.9, policy=pol)
    ratio = learned.smin / np.maximum(fixed.smin, 1e-300)
    print(f"\n[policy] samples {X.shape[0]}, labels {info['label_counts']}; held-out steps: fixed "
          f"{fixed.steps.sum()}, learned {learned.steps.sum()}; quality ratio min {ratio.min():.3f} "
          f"median {np.median(ratio):.3f}; kernel ms fixed {fixed.ms:.1f} learned {learned.ms:.1f}")
    assert learned.steps.sum() < 0.8 * fixed.steps.sum()
    assert np.mean(ratio >= 0.5) >= 0.9
