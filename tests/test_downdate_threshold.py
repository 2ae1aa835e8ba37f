"""The partial-norm downdate under a reduced-precision trailing update, as a
CPU model (the reading behind the recomputation threshold of opts.precision
1-3).

Sec. 3.1 downdates a column's norm after each step:
  t = max(0, 1 - sum(r / u)^2),  u <- u sqrt(t),
with r the entries the step moved into R. It recomputes the norm when
t (u / uref)^2 falls to a threshold, uref being the last recomputed norm.
The downdate is exact only if the remaining entries are an exact orthogonal
image of the column. An update with unit roundoff u_upd adds noise of about
u_upd times the column's size to them at every step.

The model follows a set of columns through a run. Each step moves a share of the
remaining norm into R, and the kept part gets noise of that size. At the
gap, the whole remaining signal goes, leaving only noise. The tracked norm is
compared with the true norm of what is actually left.
  * With sqrt(eps) as the threshold and u_upd = 2^-21 or 2^-16 (the
    tensor-core forms), the tracked norm stays orders of magnitude above the
    true noise-level norm. That is the stale norm that made those forms take
    30 extra single-column steps on the GPU.
  * With sqrt(u_upd), the downdate is trusted only while its relative error
    is at most about sqrt(u_upd), and the tracked norm follows the true one."""
from __future__ import annotations

import numpy as np

EPS = 2.0**-52


def _run(thr, u_upd, steps=40, m=2000, cols=200, gap_step=30, seed=0):
    """Track `cols` columns through a run.  Returns the worst ratio, after the
    gap, between the largest tracked norm (the mu of the rank criterion and
    of the candidate threshold) and the largest true norm, and the number of
    recomputations."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((m, cols))
    x /= np.linalg.norm(x, axis=0)
    u = np.linalg.norm(x, axis=0)
    uref = u.copy()
    recomputes = 0
    worst = 1.0
    for s in range(steps):
        # the step moves part of every column into R (an orthogonal
        # transformation would rotate first; the model takes the rotated
        # columns as given); at the gap the whole signal goes
        frac = 1.0 if s == gap_step else 0.3
        r = np.sqrt(frac) * np.linalg.norm(x, axis=0)
        keep = np.sqrt(1.0 - frac) * x
        # the reduced-precision update perturbs what it keeps by about u_upd
        # times the size of the column it transformed
        noise = rng.standard_normal((m, cols))
        noise *= u_upd * np.linalg.norm(x, axis=0) / np.linalg.norm(noise, axis=0)
        x = keep + noise
        true = np.linalg.norm(x, axis=0)
        t = np.maximum(0.0, 1.0 - (r / u) ** 2)
        rec = t * (u / uref) ** 2 <= thr
        recomputes += int(rec.sum())
        u = np.where(rec, true, u * np.sqrt(t))
        uref = np.where(rec, true, uref)
        if s >= gap_step:
            ratio = u.max() / true.max()
            worst = max(worst, ratio, 1.0 / ratio)
    return worst, recomputes


def test_fp64_threshold_leaves_stale_norms_after_the_gap():
    for u_upd in (2.0**-21, 2.0**-16):
        worst, _ = _run(np.sqrt(EPS), u_upd)
        assert worst > 1e3, (u_upd, worst)
    # FP32 noise (2^-24) still cancels deeply enough at the gap for sqrt(eps)
    # to fire, as the FP32 form did on the GPU before the threshold changed
    worst, _ = _run(np.sqrt(EPS), 2.0**-24)
    assert worst < 1.0 + 1e-6, worst


def test_update_precision_threshold_tracks_the_true_norm():
    for u_upd in (2.0**-24, 2.0**-21, 2.0**-16):
        worst, rec = _run(np.sqrt(u_upd), u_upd)
        assert worst < 1.0 + 10 * np.sqrt(u_upd), (u_upd, worst)
        assert rec >= 1


def test_exact_update_needs_no_recomputation_before_the_gap():
    """Without noise (an FP64 update, modelled as exact) the downdate is exact
    to rounding and the sqrt(eps) threshold never fires before a gap."""
    worst, rec = _run(np.sqrt(EPS), 0.0, gap_step=1000, steps=40)
    assert worst == 1.0 and rec == 0
