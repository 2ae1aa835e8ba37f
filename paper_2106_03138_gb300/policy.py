"""Learned per-step (tau, delta) for QRDM.

The paper fixes (tau, delta) for a whole factorization and studies the choice
empirically (Sec. 5).  This module learns a per-step choice:

* **Training data** come from plain QRDM runs (the batched kernel) on
  generated matrices, one run per point of a (tau, delta) grid.  Each run
  logs, per block step, the 16 features of include/qrdm.h (qrdm_policy).
* **Labels.** The factorization is split into four phases by n_s / min(m, n).
  For each matrix and phase the label is the grid point with the largest mean
  block size l in that phase among the points whose rank quality
  sigma_min(R11) / sigma_r is at least QUALITY_FACTOR (0.9) times that of the
  fixed (0.9, 0.9) run.  Every logged step of every run gets the label of its matrix and
  phase.
* **Training** runs the library's own kernels (qrdm_mlp_train: forward,
  backward and Adam on the GPU) on BF16 weights with FP32 accumulation.
* **Use.** ``Policy.struct()`` is the qrdm_policy passed to ``factor`` or
  ``BatchPlan.run``.  The kernels predict (tau_s, delta_s) at every DM step,
  and a guard falls back to the fixed (tau, delta) for the rest of a
  factorization when a learned step accepted a pivot below rho_min times the
  largest partial norm left after it (an approximate column-pivoting order).

Argument marshalling and bookkeeping only; every numeric step runs in the
library's kernels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import _binding as _b
from . import inputs

GRID_TAU = (0.1, 0.15, 0.25, 0.4, 0.6, 0.9)
GRID_DELTA = (0.5, 0.7, 0.9)
TAU_RANGE = (0.05, 1.0)
DELTA_RANGE = (0.3, 1.0)
RHO_MIN = 0.5
REFERENCE = (0.9, 0.9)
NPHASE = 4
QUALITY_FACTOR = 0.9


@dataclass(frozen=True)
class TrainEntry:
    """A square training matrix: order n, spectrum recipe kind, rank, seed."""

    n: int
    kind: int  # 0: geometric 1 -> 1e-12 over the rank then 1e-15; 1: geometric 1 -> 1e-15; 2: gap 1 then 1e-14
    rank: int
    seed: int

    def sigma(self) -> np.ndarray:
        if self.kind == 0:
            return inputs.sigma_rank_geometric(self.n, self.rank)
        if self.kind == 1:
            return inputs.sigma_geometric(self.n, 1e-15)
        return inputs.sigma_gap(self.n, self.rank)

    def build_gpu(self, device="cuda"):
        return inputs.from_spectrum_gpu(self.n, self.n, self.sigma(), self.seed, device=device)


def training_entries(count: int, seed: int, n_lo: int = 64, n_hi: int = 768) -> list:
    """n log-uniform in [n_lo, n_hi]; the three spectrum recipes in turn;
    rank ~ U[n/4, n] (kind 0) or U[n/4, 3n/4] (kind 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = i % 3
        if kind == 0:
            r = int(rng.integers(max(1, n // 4), n + 1))
        elif kind == 1:
            r = n
        else:
            r = int(rng.integers(max(1, n // 4), max(2, 3 * n // 4) + 1))
        out.append(TrainEntry(n, kind, r, seed * 1_000_003 + i))
    return out


def normalize(tau, delta, tau_range=TAU_RANGE, delta_range=DELTA_RANGE) -> np.ndarray:
    """(tau, delta) -> the MLP's sigmoid targets in [0, 1]^2."""
    t = (np.asarray(tau, np.float64) - tau_range[0]) / (tau_range[1] - tau_range[0])
    d = (np.asarray(delta, np.float64) - delta_range[0]) / (delta_range[1] - delta_range[0])
    return np.stack([t, d], axis=-1)


class Policy:
    """The MLP's weights on the device: FP32 master copy and BF16 working copy."""

    def __init__(self, device="cuda", seed: int = 0, tau_range=TAU_RANGE, delta_range=DELTA_RANGE,
                 rho_min: float = RHO_MIN):
        import torch

        self._torch = torch
        self.device = torch.device(device)
        self.w32 = torch.zeros(_b.QRDM_POLICY_NPARAM, dtype=torch.float32, device=self.device)
        self.w16 = torch.zeros(_b.QRDM_POLICY_NPARAM, dtype=torch.bfloat16, device=self.device)
        self.adam = torch.zeros(2 * _b.QRDM_POLICY_NPARAM, dtype=torch.float32, device=self.device)
        self.tau_range, self.delta_range, self.rho_min = tau_range, delta_range, float(rho_min)
        self.steps_done = 0
        self._check(_b.load().qrdm_mlp_init(self.w32.data_ptr(), self.w16.data_ptr(), seed, self._s()),
                    "qrdm_mlp_init")

    def _s(self):
        return self._torch.cuda.current_stream(self.device).cuda_stream

    @staticmethod
    def _check(rc, where):
        if rc != 0:
            from . import QRDMError

            raise QRDMError(rc, where)

    def load_weights(self, w32: np.ndarray) -> None:
        """Set the master weights (QRDM_POLICY_NPARAM floats) and refresh BF16."""
        self.w32.copy_(self._torch.from_numpy(np.asarray(w32, dtype=np.float32)))
        self._check(_b.load().qrdm_mlp_to_bf16(self.w32.data_ptr(), self.w16.data_ptr(), self._s()),
                    "qrdm_mlp_to_bf16")

    @classmethod
    def load(cls, path: str, device="cuda") -> "Policy":
        """A policy from the weights train_policy stored (FP32 master copy and
        the output ranges it was trained for)."""
        import json

        with np.load(path) as z:
            w = z["w32"]
            meta = json.loads(str(z["summary"]))
        pol = cls(device=device, tau_range=tuple(meta.get("tau_range", TAU_RANGE)),
                  delta_range=tuple(meta.get("delta_range", DELTA_RANGE)), rho_min=meta.get("rho_min", RHO_MIN))
        pol.load_weights(w)
        return pol

    def struct(self, *, weights: bool = True, feat_log=None, act_log=None) -> _b.qrdm_policy:
        """qrdm_policy for the C calls (keep the returned object alive)."""
        p = _b.qrdm_policy()
        p.d_weights = self.w16.data_ptr() if weights else None
        if feat_log is not None:
            p.d_feat_log = feat_log.data_ptr()
            p.d_act_log = act_log.data_ptr()
            p.log_cap = feat_log.shape[0]
        p.tau_lo, p.tau_hi = self.tau_range
        p.delta_lo, p.delta_hi = self.delta_range
        p.rho_min = self.rho_min
        return p

    def forward(self, x) -> np.ndarray:
        """y = sigmoid outputs for features x (N x 16), through qrdm_mlp_forward."""
        torch = self._torch
        xd = torch.as_tensor(np.asarray(x, np.float32), device=self.device).contiguous()
        n = xd.shape[0]
        y = torch.empty((n, 2), dtype=torch.float32, device=self.device)
        ws = torch.empty(_b.qrdm_mlp_workspace_size(n) // 4 + 1, dtype=torch.float32, device=self.device)
        self._check(_b.load().qrdm_mlp_forward(self.w16.data_ptr(), xd.data_ptr(), n, y.data_ptr(), ws.data_ptr(),
                                               ws.numel() * 4, self._s()), "qrdm_mlp_forward")
        return y.cpu().numpy()

    def loss_grad(self, x, t):
        """(L, dL/dw) on a batch through qrdm_mlp_loss_grad."""
        torch = self._torch
        xd = torch.as_tensor(np.asarray(x, np.float32), device=self.device).contiguous()
        td = torch.as_tensor(np.asarray(t, np.float32), device=self.device).contiguous()
        n = xd.shape[0]
        g = torch.empty(_b.QRDM_POLICY_NPARAM, dtype=torch.float32, device=self.device)
        L = torch.empty(1, dtype=torch.float32, device=self.device)
        ws = torch.empty(_b.qrdm_mlp_workspace_size(n) // 4 + 1, dtype=torch.float32, device=self.device)
        self._check(_b.load().qrdm_mlp_loss_grad(self.w16.data_ptr(), xd.data_ptr(), td.data_ptr(), n, g.data_ptr(),
                                                 L.data_ptr(), ws.data_ptr(), ws.numel() * 4, self._s()),
                    "qrdm_mlp_loss_grad")
        return float(L.item()), g.cpu().numpy()

    def train(self, X, T, *, steps: int = 2000, batch: int = 1024, lr: float = 2e-3, weight_decay: float = 1e-4,
              seed: int = 1) -> np.ndarray:
        """Minibatch Adam on (X, T) with the library's training kernels;
        returns the per-step loss."""
        torch = self._torch
        xd = torch.as_tensor(np.asarray(X, np.float32), device=self.device).contiguous()
        td = torch.as_tensor(np.asarray(T, np.float32), device=self.device).contiguous()
        loss = torch.zeros(max(steps, 1), dtype=torch.float32, device=self.device)
        ws = torch.empty(_b.qrdm_mlp_workspace_size(batch) // 4 + 1, dtype=torch.float32, device=self.device)
        self._check(_b.load().qrdm_mlp_train(self.w32.data_ptr(), self.w16.data_ptr(), self.adam.data_ptr(),
                                             xd.data_ptr(), td.data_ptr(), xd.shape[0], batch, steps, lr,
                                             weight_decay, seed, loss.data_ptr(), ws.data_ptr(), ws.numel() * 4,
                                             self._s()), "qrdm_mlp_train")
        self.steps_done += steps
        return loss[:steps].cpu().numpy()


def smin_r11(mats, ranks, iters: int = 30, seed: int = 0) -> np.ndarray:
    """sigma_min of each factored matrix's leading R11 (ranks[i] x ranks[i]),
    by inverse power iteration on (R11^T R11)^{-1}: each iteration is two
    triangular solves; the Rayleigh quotient after `iters` steps estimates
    1 / sigma_min^2 from below.  The R11 are padded with identity blocks to
    sizes that are multiples of 64 and solved in batches of equal size.
    Evaluation of the training labels only (the factorization is done)."""
    import torch

    out = np.ones(len(mats))
    groups = {}
    for i, (A, r) in enumerate(zip(mats, ranks)):
        if r > 0:
            groups.setdefault(-(-int(r) // 64) * 64, []).append(i)
    g = torch.Generator(device=mats[0].device if mats else "cpu")
    g.manual_seed(seed)
    for size, idx in groups.items():
        R = torch.eye(size, dtype=torch.float64, device=mats[idx[0]].device).repeat(len(idx), 1, 1)
        for b, i in enumerate(idx):
            r = int(ranks[i])
            R[b, :r, :r] = torch.triu(mats[i][:r, :r])
        x = torch.randn((len(idx), size, 1), dtype=torch.float64, device=R.device, generator=g)
        x = x / torch.linalg.vector_norm(x, dim=1, keepdim=True)
        lam = None
        for _ in range(iters):
            y = torch.linalg.solve_triangular(R.transpose(1, 2), x, upper=False)
            z = torch.linalg.solve_triangular(R, y, upper=True)
            lam = (x * z).sum(dim=(1, 2))
            x = z / torch.linalg.vector_norm(z, dim=1, keepdim=True)
        sm = (1.0 / torch.sqrt(lam)).cpu().numpy()
        for b, i in enumerate(idx):
            out[i] = sm[b]
    return out


def _quality(A_fact, sigma: np.ndarray, r: int) -> float:
    """min_{i<r} |R_ii| / sigma_i of a factored matrix (device tensor)."""
    import torch

    if r <= 0:
        return 1.0
    d = torch.diagonal(A_fact)[:r].abs().cpu().numpy()
    return float(np.min(d / sigma[:r]))


@dataclass
class SweepResult:
    tau: float
    delta: float
    steps: np.ndarray      # per matrix
    quality: np.ndarray    # per matrix: min_{i<r} |R_ii| / sigma_i
    rank_colmax: np.ndarray
    ms: float
    traces: list = field(default_factory=list)  # per matrix: (ns, k, l, dm_on) arrays
    feats: list = field(default_factory=list)   # per matrix: (steps x 16) features
    smin: np.ndarray | None = None              # per matrix: sigma_min(R11) / sigma_r


def run_batch(pristine, entries, tau, delta, k_max=64, policy: Policy | None = None, logs=False, stream=None):
    """Factor copies of `pristine` with the batched kernel at (tau, delta)
    (and the policy's MLP if given); returns a SweepResult."""
    import torch

    from . import BatchPlan, make_opts

    work = [p.clone() for p in pristine]
    plan = BatchPlan(work, k_max, trace=logs, policy_logs=logs or policy is not None, stream=stream)
    pol = None
    if policy is not None:
        pol = policy.struct()
    elif logs:
        pol = _features_only_struct()  # log the features, keep (tau, delta) fixed
    opts = make_opts(policy=pol) if pol is not None else None
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.run(tau, delta, opts)
    e1.record()
    e1.synchronize()
    res = plan.results()
    out = SweepResult(tau, delta, res.steps.copy(), np.zeros(len(work)), res.rank_colmax.copy(), e0.elapsed_time(e1))
    qranks = [_quality_rank(e, int(res.rank_colmax[i])) for i, e in enumerate(entries)]
    sm = smin_r11(work, qranks)
    out.smin = np.array([sm[i] / e.sigma()[qranks[i] - 1] if qranks[i] > 0 else 1.0 for i, e in enumerate(entries)])
    for i, (A, e) in enumerate(zip(work, entries)):
        out.quality[i] = _quality(A, e.sigma(), qranks[i])
        if logs:
            tr, _ = plan.trace(i, res.steps[i])
            out.traces.append((tr["ns"].copy(), tr["k"].copy(), tr["l"].copy(), tr["dm_on"].copy()))
            f, _a = plan.policy_logs(i, res.steps[i])
            out.feats.append(f)
    plan.close()
    del work
    return out


def _features_only_struct() -> _b.qrdm_policy:
    p = _b.qrdm_policy()
    p.tau_lo, p.tau_hi = TAU_RANGE
    p.delta_lo, p.delta_hi = DELTA_RANGE
    p.rho_min = RHO_MIN
    return p


def _quality_rank(e, rank_colmax: int) -> int:
    """The rank over which quality is measured: the spectrum's gap where it
    has one, else the rank the criterion found."""
    return min(e.rank, rank_colmax) if e.kind != 1 else rank_colmax


# the grid of the large training run (train_policy): finer near the
# reference, where a 4096^2 sweep showed the quality cliff (tau 0.6 is 1.85x
# faster than 0.9 and still within 2x quality on most matrices)
GRID_TAU_FINE = (0.25, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9)


def collect(entries, pristine, k_max=64, stream=None, quality_factor: float = QUALITY_FACTOR,
            grid_tau=GRID_TAU, grid_delta=GRID_DELTA, tau_range=TAU_RANGE) -> tuple[np.ndarray, np.ndarray, dict]:
    """Sweep the (tau, delta) grid with plain QRDM and build (X, T).  A grid
    point is admissible for a matrix when its sigma_min(R11) / sigma_r is at
    least quality_factor times the fixed (0.9, 0.9) run's.  Returns (X, T,
    info) with T the normalized label (tau*, delta*)."""
    sweeps = {}
    for tau in grid_tau:
        for delta in grid_delta:
            sweeps[(tau, delta)] = run_batch(pristine, entries, tau, delta, k_max, logs=True, stream=stream)
    ref = sweeps[REFERENCE]
    X, T = [], []
    label_hist = {}
    for i, e in enumerate(entries):
        kmin = e.n
        qref = ref.smin[i]
        best = {}
        for q in range(NPHASE):
            cand = []
            for g, sw in sweeps.items():
                if not (sw.smin[i] >= quality_factor * qref):
                    continue
                ns, k, l, dm = sw.traces[i]
                ph = np.minimum((NPHASE * ns) // max(kmin, 1), NPHASE - 1)
                sel = (dm == 1) & (ph == q)
                if not np.any(sel):
                    continue
                cand.append((float(np.mean(l[sel])), g[0], g[1]))
            if cand:
                cand.sort(key=lambda c: (-c[0], -c[1], -c[2]))
                best[q] = (cand[0][1], cand[0][2])
        for g, sw in sweeps.items():
            ns, k, l, dm = sw.traces[i]
            f = sw.feats[i]
            ph = np.minimum((NPHASE * ns) // max(kmin, 1), NPHASE - 1)
            for s in range(len(ns)):
                if dm[s] != 1 or int(ph[s]) not in best:
                    continue
                tau_l, delta_l = best[int(ph[s])]
                X.append(f[s])
                T.append(normalize(tau_l, delta_l, tau_range=tau_range))
                label_hist[(tau_l, delta_l)] = label_hist.get((tau_l, delta_l), 0) + 1
    info = {"grid": [list(g) for g in sweeps], "sweep_ms": {f"{g[0]},{g[1]}": sw.ms for g, sw in sweeps.items()},
            "label_counts": {f"{k[0]},{k[1]}": v for k, v in sorted(label_hist.items())},
            "samples": len(X)}
    return np.asarray(X, np.float32), np.asarray(T, np.float32), info
