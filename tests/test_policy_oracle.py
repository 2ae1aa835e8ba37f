"""CPU pins of the learned-policy oracle (oracle/mlp_oracle.py) and of the
oracle's per-step (tau, delta) schedule: each checked against something other
than itself (finite differences, closed forms, direct counts, the plain
oracle)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2106_03138_gb300 import inputs


def _rand_w(rng, scale=0.3):
    return rng.standard_normal(M.NPARAM) * scale


def test_parameter_count_matches_the_layer_sizes():
    assert M.NPARAM == 16 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2 == 5378
    w = np.arange(M.NPARAM, dtype=np.float64)
    assert np.array_equal(M.pack(M.unpack(w)), w)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    w = _rand_w(rng)
    x = rng.standard_normal((7, 16))
    t = rng.uniform(0, 1, (7, 2))
    L, g = M.loss_grad(w, x, t)
    assert abs(L - M.loss(w, x, t)) <= 1e-15 * max(1.0, L)
    h = 1e-6
    idx = rng.choice(M.NPARAM, 300, replace=False)
    # include every bias and some weights of each layer
    idx = np.unique(np.concatenate([idx, np.arange(1024, 1088), np.arange(5184, 5248), np.arange(5376, 5378)]))
    num = np.empty(idx.size)
    for k, i in enumerate(idx):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        num[k] = (M.loss(wp, x, t) - M.loss(wm, x, t)) / (2 * h)
    err = np.abs(num - g[idx])
    assert np.max(err) <= 1e-7 * max(1.0, np.max(np.abs(g))), np.max(err)


def test_zero_network_closed_form():
    """All weights zero: y = 1/2 everywhere, L = mean sum (1/2 - t)^2 / 2, and
    only the output bias has a gradient: dL/db3_o = (1/B) sum_b (1/2 - t_bo) / 4."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 16))
    t = rng.uniform(0, 1, (5, 2))
    w = np.zeros(M.NPARAM)
    y, _ = M.forward(w, x)
    assert np.all(y == 0.5)
    L, g = M.loss_grad(w, x, t)
    assert L == pytest.approx(0.5 * np.sum((0.5 - t) ** 2) / 5, rel=1e-15)
    expect_b3 = np.sum(0.5 - t, axis=0) * 0.25 / 5
    np.testing.assert_allclose(g[-2:], expect_b3, rtol=1e-14)
    assert np.all(g[:-2] == 0.0)


def test_single_path_hand_example():
    """One live path x_0 -> h1_0 -> h2_0 -> o_0: o_0 = w3 relu(w2 relu(w1 x_0 + b1) + b2) + b3."""
    p = M.unpack(np.zeros(M.NPARAM))
    p["W1"][0, 0], p["b1"][0] = 2.0, 0.5
    p["W2"][0, 0], p["b2"][0] = -1.5, 4.0
    p["W3"][0, 0], p["b3"][0] = 0.25, -0.1
    w = M.pack(p)
    x = np.zeros((1, 16))
    x[0, 0] = 0.75
    h1 = 2.0 * 0.75 + 0.5
    h2 = max(-1.5 * h1 + 4.0, 0.0)
    o = 0.25 * h2 - 0.1
    y, _ = M.forward(w, x)
    assert y[0, 0] == pytest.approx(1 / (1 + np.exp(-o)), rel=1e-15)
    assert y[0, 1] == 0.5


def test_bf16_rounding():
    a = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 0.0, 3.0e38], dtype=np.float32)
    r = M.bf16_round(a)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties to even -> 1
    assert r[0] == 1.0 and r[1] == 1.0
    assert r[2] == np.float32(1.0 + 2.0 ** -7)
    assert r[3] == -2.5 and r[4] == 0.0
    assert np.isfinite(r[5])
    assert M.bf16_bits(np.array([1.0], np.float32))[0] == 0x3F80


def test_step_features_by_hand():
    u = np.array([0.5, 3.0, 2.9, 0.1, 2.0, 1.0])
    f = M.step_features(u, ns=1, jstar=1, anorm=4.0, prev_l=8, prev_k=16, cos_mean=0.2, cos_max=0.7, prev_tau=0.15)
    # the other trailing norms relative to mu = 3: 0.967, 0.033, 0.667, 0.333
    counts = [1, 1, 1, 2, 2, 3, 3, 3]  # >= .95, .9, .75, .6, .45, .3, .15, .05 (times mu)
    assert np.allclose(f[:8], np.array(counts) / 128.0)
    assert f[8] == pytest.approx(5 / 6)
    assert f[9] == pytest.approx(np.log2(5) / 16)
    assert f[10] == pytest.approx(np.log10(0.75) / 16)
    assert f[11] == pytest.approx(8 / 64) and f[12] == pytest.approx(0.5)
    assert (f[13], f[14], f[15]) == (0.2, 0.7, 0.15)


def test_step_features_do_not_depend_on_the_matrix_scale():
    """Every feature is relative (norms against mu, mu against max||a_i||),
    so scaling the norms by 2^k (exact in floating point) leaves all 16
    features the same bits: the policy cannot react to the scale of A."""
    rng = np.random.default_rng(9)
    for _ in range(50):
        n = int(rng.integers(5, 300))
        u = np.abs(rng.standard_normal(n)) * np.exp(rng.uniform(-20, 20, size=n))
        ns = int(rng.integers(0, n - 1))
        jstar = ns + int(np.argmax(u[ns:]))
        anorm = float(u.max()) * float(rng.uniform(1.0, 3.0))
        args = dict(prev_l=5, prev_k=9, cos_mean=0.1, cos_max=0.4, prev_tau=0.6)
        f = M.step_features(u, ns, jstar, anorm, **args)
        for c in (2.0 ** 30, 2.0 ** -40):
            g = M.step_features(c * u, ns, jstar, c * anorm, **args)
            assert np.array_equal(f, g)


def test_step_feature_counts_at_their_thresholds():
    """The candidate-count features count u >= t mu with t the FP32 value of
    each threshold (the kernel compares against FP32 constants): a norm equal
    to float32(t) mu is counted; the double t itself is no threshold
    (float32(0.95) < 0.95, float32(0.15) > 0.15 ...), and equality counts."""
    mu = 1.0
    ts32 = [float(np.float32(t)) for t in M.THRESH]
    # one norm sitting exactly on each FP32 threshold, plus the argmax
    u = np.array([mu] + ts32)
    f = M.step_features(u, ns=0, jstar=0, anorm=1.0, prev_l=0, prev_k=0, cos_mean=0.0, cos_max=0.0, prev_tau=0.0)
    # threshold b counts the norms >= ts32[b]: those of thresholds 0..b
    assert list(np.round(f[:8] * 128).astype(int)) == list(range(1, 9))
    # a norm just below float32(0.95) mu is not counted at 0.95
    u2 = np.array([mu, float(np.nextafter(np.float64(ts32[0]), 0.0))])
    f2 = M.step_features(u2, ns=0, jstar=0, anorm=1.0, prev_l=0, prev_k=0, cos_mean=0.0, cos_max=0.0, prev_tau=0.0)
    assert f2[0] == 0.0 and f2[1] == 1 / 128


def test_outputs_map_to_tau_then_delta():
    """Output 0 of the MLP is tau and output 1 is delta, each mapped
    linearly onto its range (0 -> lower end, 1 -> upper end)."""
    t, d = M.to_tau_delta(np.array([1.0, 0.0]), 0.5, 1.0, 0.3, 0.9)
    assert (t, d) == (1.0, 0.3)
    t, d = M.to_tau_delta(np.array([0.25, 0.5]), 0.2, 1.0, 0.4, 1.0)
    assert t == pytest.approx(0.4) and d == pytest.approx(0.7)


def test_constant_schedule_reproduces_the_plain_oracle_bit_for_bit():
    A = inputs.from_spectrum(120, 90, inputs.sigma_geometric(90, 1e-12), 3)
    plain = O.qrdm(A, 0.3, 0.8, 16)
    sched = np.tile([0.3, 0.8], (plain["nsteps"] + 5, 1))
    got = O.qrdm(A, 0.9, 0.1, 16, schedule=sched)
    assert np.array_equal(got["A"], plain["A"])
    assert np.array_equal(got["perm"], plain["perm"])
    assert got["rank"] == plain["rank"]


def test_schedule_sets_each_steps_threshold():
    """The first step's candidate count equals the number of columns whose
    norm is at least tau_0 times the largest (eq. def_candidate_set)."""
    A = inputs.from_spectrum(100, 80, inputs.sigma_geometric(80, 1e-10), 5)
    norms = np.linalg.norm(A, axis=0)
    for tau0 in (0.2, 0.6, 0.95):
        o = O.qrdm(A, 0.9, 0.9, 64, schedule=[[tau0, 0.9]])
        mu = norms.max()
        expect = int(np.count_nonzero(norms >= tau0 * mu)) - 1
        assert o["trace"]["ncand_all"][0] == expect
        assert o["trace"]["eps_s"][0] == pytest.approx(tau0 * o["trace"]["mu"][0], rel=1e-15)


def test_adam_first_step_is_a_signed_step_of_size_lr():
    """Bias correction makes the first Adam step lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    w = rng.standard_normal(M.NPARAM)
    g = rng.standard_normal(M.NPARAM)
    w1, m1, v1 = M.adam_step(w, g, np.zeros_like(w), np.zeros_like(w), 1, 1e-2, eps=1e-8)
    np.testing.assert_allclose(w - w1, 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # weight decay acts on weights only, never on biases
    w2, _, _ = M.adam_step(w, np.zeros_like(w), np.zeros_like(w), np.zeros_like(w), 1, 1e-2, wd=0.5)
    d = w - w2
    assert d[1024] == 0.0 and d[5377] == 0.0 and d[0] == pytest.approx(1e-2 * 0.5 * w[0])
