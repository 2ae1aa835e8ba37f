"""CPU models of three reformulations the kernels use, each checked against
the plain form it replaces.  The kernels are checked against the oracle on
the GPU; these tests pin the equivalence argument itself, which is what lets
the reformulated kernels keep the plain forms' decisions:

* the greedy DM pick (Alg. 1 loop) from a bit matrix of all pairwise cosine
  tests equals the loop that tests each candidate against the accepted set;
* the pairwise swaps of Sec. 4 simulated with an inverse map equal the
  simulation that searches the current position of each selected column;
* a transposed lane tree (each level keeps half of a lane's values) adds the
  same pairs as one xor lane tree per value, so every sum has the same bits;
* the trailing update's W = T^T V^T A, formed without T by forward
  substitution with S = V^T V (W_t = htau_t (P_t - sum_{q<t} S_qt W_q)),
  makes A - V W equal the reflectors applied one after another;
* the argmax, the candidate test u >= tau mu and the candidate order taken on
  the raw bits of the partial norms read as signed 64-bit integers (integer
  compares instead of FP64 ones) equal the same decisions on the values.
  This holds for non-negative doubles.  The partial norms are never negative
  and never -0.0: they are square roots of sums of squares, 0.0 for factored
  columns, or u sqrt(t) with u > 0 and t clamped to +0.0 or more (1 - q is
  +0.0 when q = 1 in round-to-nearest).
"""
from __future__ import annotations

import numpy as np


def _theta_ok(g, d, a, b, delta):
    """|theta_ab| < delta with the kernels' operand order: |G_ab| (d_a d_b);
    a zero column counts as |theta| = 1."""
    rr = d[a] * d[b]
    th = abs(g[a, b]) * rr if rr > 0.0 else 1.0
    return th < delta


def _pick_plain(g, d, delta):
    J = [0]
    for a in range(1, len(d)):
        if all(_theta_ok(g, d, a, b, delta) for b in J):
            J.append(a)
    return J


def _pick_bits(g, d, delta):
    kc = len(d)
    cmp = [0] * kc  # bit b of cmp[a], b < a: the test passes
    for a in range(kc):
        for b in range(a):
            if _theta_ok(g, d, a, b, delta):
                cmp[a] |= 1 << b
    jm, J = 1, [0]
    for a in range(1, kc):
        if jm & ~cmp[a] == 0:
            jm |= 1 << a
            J.append(a)
    return J


def test_greedy_pick_from_the_bit_matrix_equals_the_plain_loop():
    rng = np.random.default_rng(5)
    for trial in range(300):
        kc = int(rng.integers(1, 70))
        m = int(rng.integers(2, 12))
        C = rng.standard_normal((m, kc))
        if trial % 5 == 0:  # repeated and zero columns
            C[:, rng.integers(0, kc, size=kc // 3)] = C[:, [0]]
            C[:, rng.integers(0, kc)] = 0.0
        g = C.T @ C
        dg = np.sqrt(np.diag(g))
        d = np.where(dg > 0.0, 1.0 / np.where(dg > 0.0, dg, 1.0), 0.0)
        delta = float(rng.choice([0.0, 0.3, 0.6, 0.9, 1.0]))
        if trial % 7 == 0 and kc > 2:  # a pair exactly at the threshold
            delta = float(abs(g[1, 2]) * (d[1] * d[2]))
        assert _pick_bits(g, d, delta) == _pick_plain(g, d, delta)


def _swaps_search(ns, k, pos_of_J):
    """Entries: ns + t for t < k, then the positions of the J_t outside the
    block in t order; for each t, find the entry currently holding J_t's
    starting position and swap it with entry t."""
    pos = [ns + t for t in range(k)] + [p for p in pos_of_J if p >= ns + k]
    cont = list(pos)
    for t, orig in enumerate(pos_of_J):
        e = cont.index(orig)
        cont[t], cont[e] = cont[e], cont[t]
    return [(pos[e], cont[e]) for e in range(len(pos)) if cont[e] != pos[e]]


def _swaps_inverse(ns, k, pos_of_J):
    pos = [ns + t for t in range(k)]
    eid = []
    for p in pos_of_J:
        if p >= ns + k:
            eid.append(len(pos))
            pos.append(p)
        else:
            eid.append(p - ns)
    cid = list(range(len(pos)))
    inv = list(range(len(pos)))
    for t in range(k):
        e = inv[eid[t]]
        if e != t:
            ct, ce = cid[t], cid[e]
            cid[t], cid[e] = ce, ct
            inv[ce], inv[ct] = t, e
    return [(pos[e], pos[cid[e]]) for e in range(len(pos)) if pos[cid[e]] != pos[e]]


def test_swap_simulation_with_an_inverse_map_equals_the_search():
    rng = np.random.default_rng(9)
    for _ in range(500):
        n = int(rng.integers(2, 200))
        ns = int(rng.integers(0, n - 1))
        kmax = min(n - ns, 64)
        k = int(rng.integers(1, kmax + 1))
        pos_of_J = [int(x) for x in rng.choice(np.arange(ns, n), size=k, replace=False)]
        pos_of_J.sort(key=lambda _: rng.random())  # any candidate order
        moves = _swaps_inverse(ns, k, pos_of_J)
        assert moves == _swaps_search(ns, k, pos_of_J)
        # the moves are a permutation of the touched positions that puts J_t at ns + t
        final = {p: p for p in set(p for mv in moves for p in mv)}
        for dst, src in moves:
            final[dst] = src
        for t, p in enumerate(pos_of_J):
            assert final.get(ns + t, ns + t) == p


def _xor_tree(vals, offsets):
    """One value per lane; at each level lane L adds lane L ^ o's value to its own."""
    v = list(vals)
    for o in offsets:
        v = [v[L] + v[L ^ o] for L in range(len(v))]
    return v


def _transposed_tree(lanes, offsets):
    """lanes[L] holds K values; at the level of offset o a lane keeps the upper
    half of its values when bit o is set (else the lower half) and adds its
    partner's copy of the same values; once one value is left, plain levels."""
    cur = [list(x) for x in lanes]
    for o in offsets:
        h = len(cur[0]) // 2
        if h == 0:
            cur = [[cur[L][0] + cur[L ^ o][0]] for L in range(len(cur))]
            continue
        nxt = []
        for L in range(len(cur)):
            up = (L & o) != 0
            P = L ^ o
            nxt.append([(cur[L][i + h] if up else cur[L][i]) + (cur[P][i + h] if up else cur[P][i]) for i in range(h)])
        cur = nxt
    return cur


def test_transposed_lane_tree_adds_the_same_pairs_as_the_xor_tree():
    rng = np.random.default_rng(3)
    # (lanes, values per lane, offsets): the panel's cluster sums (16 lanes per
    # half, 8 values), a pair of columns over 32 lanes, a full 32-value transpose
    for nl, K, offs in ((16, 8, (8, 4, 2, 1)), (32, 2, (16, 8, 4, 2, 1)), (32, 32, (16, 8, 4, 2, 1))):
        for _ in range(50):
            x = rng.standard_normal((nl, K)) * np.exp(rng.uniform(-30, 30, size=(nl, K)))
            got = _transposed_tree([list(r) for r in x], offs)
            for L in range(nl):
                # the value a lane ends with: index from its bits, high level first
                idx, h = 0, K
                for o in offs:
                    h //= 2
                    if h >= 1 and (L & o):
                        idx += h
                ref = _xor_tree(list(x[:, idx]), offs)[L]
                assert got[L][0] == ref  # bit for bit


def _keys(u):
    return np.asarray(u, dtype=np.float64).view(np.int64)


def test_integer_keys_of_non_negative_doubles_order_like_the_values():
    rng = np.random.default_rng(12)
    tiny = np.nextafter(0.0, 1.0)
    edges = np.array([0.0, tiny, 2 * tiny, np.finfo(np.float64).tiny, 1.0, np.nextafter(1.0, 2.0),
                      np.nextafter(1.0, 0.0), 20 * 2.0 ** -52, np.finfo(np.float64).max])
    for trial in range(400):
        n = int(rng.integers(1, 300))
        u = np.abs(rng.standard_normal(n)) * np.exp(rng.uniform(-700, 700, size=n))  # finite values
        if trial % 3 == 0:
            u[rng.integers(0, n, size=n // 4 + 1)] = rng.choice(edges)
        if trial % 4 == 0:  # exact ties, and zero columns
            u[rng.integers(0, n, size=n // 3 + 1)] = u[0]
            u[rng.integers(0, n)] = 0.0
        assert np.all(u >= 0.0) and not np.any(np.signbit(u))
        k = _keys(u)
        # argmax, ties to the lowest position
        assert int(np.argmax(k)) == int(np.argmax(u))
        # the candidate test u >= thr, thr = tau mu, with the key of thr
        for tau in (0.0, 0.15, 0.5, 0.9, 1.0, float(rng.uniform())):
            thr = tau * float(u.max())
            assert np.array_equal(k >= _keys([thr])[0], u >= thr)
        # the order by (u descending, position ascending)
        pos = np.arange(n)
        assert np.array_equal(np.lexsort((pos, -k)), np.lexsort((pos, -u)))


def test_negative_zero_would_break_the_keys():
    """Why the partial norms must never be -0.0: its key is the smallest
    integer, so it would sort below +0.0, where the values tie."""
    assert _keys([-0.0])[0] < _keys([0.0])[0]
    assert -0.0 == 0.0


def test_w_by_forward_substitution_applies_the_block_reflector():
    """Sec. 3.2: H_1 ... H_l = I - V T V^T, so the trailing update is
    A - V (T^T V^T A).  The kernels never form T: with S = V^T V,
    T^-1 = strict_upper(S) + diag(1/htau), and W solves (T^-1)^T W = V^T A
    column by column.  Checked against the reflectors applied one by one,
    including a reflector with a zero tail (htau = 0, H = I)."""
    rng = np.random.default_rng(11)
    for m, l, n2 in ((50, 6, 20), (33, 16, 7), (9, 1, 4), (64, 32, 5)):
        h, tau = np.linalg.qr(rng.standard_normal((m, l)), mode="raw")
        V = np.tril(h.T, -1)[:, :l] + np.eye(m, l)
        htau = tau.copy()
        if l > 2:  # a zero tail: H_2 = I
            V[3:, 2] = 0.0
            htau[2] = 0.0
        A = rng.standard_normal((m, n2))
        P = V.T @ A
        S = V.T @ V
        W = np.zeros((l, n2))
        for t in range(l):
            W[t] = htau[t] * (P[t] - S[:t, t] @ W[:t])
        ref = A.copy()
        for i in range(l):  # H_1 first, then H_2, ...
            v = V[:, i]
            ref -= htau[i] * np.outer(v, v @ ref)
        np.testing.assert_allclose(A - V @ W, ref, atol=1e-13 * np.abs(A).max())
        if l > 2:
            assert np.all(W[2] == 0.0)
