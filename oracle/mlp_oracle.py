"""Oracle for the learned (tau, delta) policy: a plain numpy FP64 restatement
of the 16 -> 64 -> 64 -> 2 MLP (ReLU hidden layers, sigmoid outputs), its
loss, its gradient, and the step features computed from partial norms.

THIS IS TEST INFRASTRUCTURE: only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it.  It shares no code with the CUDA
library.

Parameter layout (a flat vector of 5378 values, row-major):
W1[16][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2].
Loss over a batch of B samples: L = (1/B) sum_b sum_o (y_bo - t_bo)^2 / 2.
The paper has no learned component; the policy is this library's addition,
so these definitions are the specification the kernels are checked against.
"""
from __future__ import annotations

import numpy as np

NFEAT, HIDDEN, NOUT = 16, 64, 2
SIZES = (("W1", (NFEAT, HIDDEN)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
         ("W3", (HIDDEN, NOUT)), ("b3", (NOUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
THRESH = (0.95, 0.9, 0.75, 0.6, 0.45, 0.3, 0.15, 0.05)


def unpack(w: np.ndarray) -> dict:
    w = np.asarray(w, dtype=np.float64).ravel()
    if w.size != NPARAM:
        raise ValueError(f"expected {NPARAM} parameters")
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = w[o:o + k].reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16_round(a: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32.
    bfloat16 keeps the top 16 bits of the IEEE-754 binary32 pattern."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """The 16-bit patterns of bf16_round(a) (what a bfloat16 array stores)."""
    return (bf16_round(a).view(np.uint32) >> 16).astype(np.uint16)


def forward(w: np.ndarray, x: np.ndarray):
    """Returns (y, cache): y = sigmoid(relu(relu(x W1 + b1) W2 + b2) W3 + b3)."""
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ p["W3"] + p["b3"]
    y = 1.0 / (1.0 + np.exp(-o))
    return y, (x, a1, h1, a2, h2, o, y)


def loss(w: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(w, x)
    return float(0.5 * np.sum((y - np.asarray(t, dtype=np.float64)) ** 2) / x.shape[0])


def loss_grad(w: np.ndarray, x: np.ndarray, t: np.ndarray):
    """(L, dL/dw) by the chain rule, layer by layer."""
    p = unpack(w)
    y, (x, a1, h1, a2, h2, o, y) = forward(w, x)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    L = float(0.5 * np.sum((y - t) ** 2) / B)
    d3 = (y - t) * y * (1.0 - y) / B          # dL/do
    g = {"W3": h2.T @ d3, "b3": d3.sum(axis=0)}
    d2 = (d3 @ p["W3"].T) * (a2 > 0.0)        # dL/da2
    g["W2"] = h1.T @ d2
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"].T) * (a1 > 0.0)        # dL/da1
    g["W1"] = x.T @ d1
    g["b1"] = d1.sum(axis=0)
    return L, pack(g)


def adam_step(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One Adam step (Kingma & Ba 2015) with decoupled weight decay (not on
    biases); returns (w, m, v)."""
    w, g, m, v = (np.asarray(a, dtype=np.float64) for a in (w, g, m, v))
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    decay = np.full(w.shape, wd)
    o = 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        if name.startswith("b"):
            decay[o:o + k] = 0.0
        o += k
    return w - lr * (mhat / (np.sqrt(vhat) + eps) + decay * w), m, v


def to_tau_delta(y: np.ndarray, tau_lo, tau_hi, delta_lo, delta_hi):
    y = np.asarray(y, dtype=np.float64)
    return tau_lo + (tau_hi - tau_lo) * y[..., 0], delta_lo + (delta_hi - delta_lo) * y[..., 1]


def step_features(u: np.ndarray, ns: int, jstar: int, anorm: float, prev_l: float, prev_k: float,
                  cos_mean: float, cos_max: float, prev_tau: float) -> np.ndarray:
    """The 16 features of a DM step from the partial norms u at its start
    (mu = u[jstar], the largest of u[ns:])."""
    u = np.asarray(u, dtype=np.float64)
    n = u.shape[0]
    mu = float(u[jstar])
    rest = np.delete(u[ns:], jstar - ns)
    f = np.zeros(NFEAT)
    for b, tb in enumerate(THRESH):
        thr = float(np.float32(tb)) * mu
        c = int(np.count_nonzero(rest >= thr))
        f[b] = min(c, 128) / 128.0
    nrem = n - ns
    f[8] = nrem / max(n, 1)
    f[9] = np.log2(nrem) / 16.0
    r = mu / anorm if (anorm > 0 and mu > 0) else 1e-30
    f[10] = np.log10(max(r, 1e-30)) / 16.0
    f[11] = min(prev_l / 64.0, 1.0)
    f[12] = prev_l / prev_k if prev_k > 0 else 1.0
    f[13] = cos_mean
    f[14] = cos_max
    f[15] = prev_tau
    return f
