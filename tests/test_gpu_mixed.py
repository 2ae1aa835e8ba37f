"""The reduced-precision forms against the FP64 oracle and the plain FP64
form. In every form the panel, norms and rank stay FP64:
  precision=1: FP32-class trailing update and candidate Gram (FP32 from FP64
    storage, CUDA cores);
  precision=2: split-BF16x3 on the tensor cores (tcgen05), one merged
    trailing update per step, the Gram on the tensor cores too;
  precision=3: the same with 3xTF32.

Results are not expected to match the FP64 oracle digit for digit. Each case
reports its error against the oracle and checks the bounds of its precision
class: residual and R error 1e-5 for FP32 and 3xTF32, 5e-5 for BF16x3. It
also checks the rank quality the FP64 form reaches:
  ||Q^T Q - I|| <= 1e-13 (the reflectors themselves are FP64);
  the precision-aware criterion finds the gap rank;
  sigma_min(R11) / sigma_r(A) within 2x of the plain FP64 form (the
  acceptance for the variants).
precision=4, the merged structure in FP64, must reproduce the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03138_gb300 import inputs
from tests._helpers import factorization_errors, upper

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402

CASES = [
    # name, m, n, sigma builder, numerical rank (gap position)
    ("gapgeo1024", 1024, 1024, lambda p: inputs.sigma_gap_geometric(p, 512), 512),
    ("gapgeo2048x1024", 2048, 1024, lambda p: inputs.sigma_gap_geometric(p, 600), 600),
    ("gap768", 768, 768, lambda p: inputs.sigma_gap(p, 300), 300),
]


def _gpu(A, precision):
    dA = q.colmajor(A)
    f = q.factor(dA, 0.15, 0.9, 64, precision=precision, trace=True)
    torch.cuda.synchronize()
    return dA.cpu().numpy(), f.htau.cpu().numpy(), f.perm.cpu().numpy().astype(np.int64), f


# precision -> (residual, R error / ||A||, rel |R_ii| error) bounds of its class
BOUNDS = {1: (1e-5, 1e-5, 1e-3), 2: (5e-5, 5e-5, 5e-3), 3: (1e-5, 1e-5, 1e-3)}


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("name,m,n,sig,r", CASES, ids=[c[0] for c in CASES])
def test_mixed_precision_against_oracle_and_plain(name, m, n, sig, r, precision):
    s = sig(min(m, n))
    A = inputs.from_spectrum(m, n, s, 1234)
    o = O.qrdm(A, 0.15, 0.9, 64)
    A64, h64, p64, f64 = _gpu(A, 0)
    A32, h32, p32, f32 = _gpu(A, precision)
    res32, orth32 = factorization_errors(A, A32, h32, p32)
    res64, orth64 = factorization_errors(A, A64, h64, p64)
    bres, berr, brel = BOUNDS[precision]
    assert res64 <= 1e-13 and orth64 <= 1e-13
    assert res32 <= bres, res32
    assert orth32 <= 1e-13, orth32
    # the precision-aware criterion finds the gap within one block (the test
    # runs at block starts and approaches eps1 ||A|| from below, Sec. 3.4/5)
    assert r <= f32.rank_colmax <= r + 64, (f32.rank, f32.rank_colmax, r)
    assert f32.rank >= f32.rank_colmax
    # rank quality against the plain FP64 form
    s11_32 = np.linalg.svd(upper(A32)[:r, :r], compute_uv=False)[-1]
    s11_64 = np.linalg.svd(upper(A64)[:r, :r], compute_uv=False)[-1]
    q32, q64 = s11_32 / s[r - 1], s11_64 / s[r - 1]
    assert q32 >= 0.5 * q64, (q32, q64)
    # per-result error: R of the mixed form against the FP64 R of the same
    # permuted matrix A Pi_32 (a library QR, rows normalized to |R|)
    R32 = upper(A32)
    Rref = np.linalg.qr(A[:, p32], mode="r")[: min(m, n)]
    anorm = np.linalg.norm(A, 2)
    err_R = float(np.max(np.abs(np.abs(R32) - np.abs(Rref)))) / anorm
    d32, dref = np.abs(np.diag(R32))[:r], np.abs(np.diag(Rref))[:r]
    rel = float(np.max(np.abs(d32 - dref) / dref))
    same = 0
    for st in range(min(len(f32.trace), len(o["trace"]))):
        if f32.trace["k"][st] != o["trace"]["k"][st] or f32.trace["l"][st] != o["trace"]["l"][st]:
            break
        same += 1
    print(f"\n[precision {precision}] {name}: residual {res32:.2e} (fp64 {res64:.2e}), orth {orth32:.1e}, "
          f"rank {f32.rank}/{f32.rank_colmax} (oracle {o['rank']}/{o['rank_colmax']}, gap {r}), "
          f"sigma_min(R11)/sigma_r {q32:.3f} (fp64 {q64:.3f}), max |R - R64(A Pi)| / ||A|| {err_R:.2e}, "
          f"max rel err |R_ii| (i < r) {rel:.2e}, steps identical to the oracle {same}")
    assert err_R <= berr
    assert rel <= brel


def test_tensor_core_forms_refuse_blocks_beyond_64():
    A = inputs.random_dense(100, 80, 0)
    for precision in (2, 3):
        with pytest.raises(q.QRDMError) as ei:
            q.factor(q.colmajor(A), 0.15, 0.9, 128, precision=precision)
        assert ei.value.code == q.QRDM_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", [2, 3])
def test_tensor_core_forms_through_the_least_squares_refinement(precision):
    m, n = 1500, 1100
    A = inputs.from_spectrum(m, n, np.geomspace(1.0, 1e-3, n), 17)
    x0 = np.random.default_rng(3).standard_normal(n)
    b = A @ x0
    dA = q.colmajor(A)
    f = q.factor(dA, 0.15, 0.9, 64, precision=precision)
    X, res = q.ls_solve(q.colmajor(A), f, torch.as_tensor(b, device="cuda"), refine=6)
    nb = np.linalg.norm(b)
    print(f"\n[precision {precision} ls] residual per iteration:", (res[:, 0] / nb).tolist())
    assert res[-1, 0] / nb <= 1e-14
    assert np.linalg.norm(X.cpu().numpy() - x0) / np.linalg.norm(x0) <= 1e-12


@pytest.mark.parametrize("shape,tau,delta,kmax", [((256, 256), 0.15, 0.9, 64), ((300, 257), 0.9, 0.9, 32),
                                                   ((700, 130), 0.2, 0.95, 16), ((1024, 1024), 0.15, 0.9, 64)])
def test_merged_fp64_form_matches_the_oracle(shape, tau, delta, kmax):
    """precision=4: the merged per-step trailing update (the structure of the
    tensor-core forms: panel-only sub-panel updates, one update with the full
    compact-WY T of the step) in FP64: the oracle's decisions and R."""
    from tests._parity import compare

    m, n = shape
    A = inputs.from_spectrum(m, n, inputs.sigma_geometric(min(m, n), 1e-12), 5 + m)
    dA = q.colmajor(A)
    f = q.factor(dA, tau, delta, kmax, precision=4, trace=True)
    torch.cuda.synchronize()
    g = {"A": dA.cpu().numpy(), "htau": f.htau.cpu().numpy(), "perm": f.perm.cpu().numpy().astype(np.int64),
         "trace": f.trace, "J": f.J.astype(np.int64), "rank": f.rank, "rank_colmax": f.rank_colmax}
    o = O.qrdm(A, tau, delta, kmax)
    rep = compare(A, g, o)
    res, orth = factorization_errors(A, g["A"], g["htau"], g["perm"])
    assert res <= 1e-13 and orth <= 1e-13, (res, orth)
    print(f"\n[precision 4] {shape}: residual {res:.2e}, diverged at {rep['diverged_at']}")


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("m,n,lda,kmax", [(515, 301, 515, 64), (640, 384, 640, 63), (515, 301, 517, 63)])
def test_tensor_core_forms_unaligned_storage(m, n, lda, kmax, precision):
    """An odd leading dimension (the W pass then reads A in 8-byte units) and
    an even one with odd panel starts (k_max = 63: 16-byte units from the even
    row ns - 1): each gives a factorization of the precision class."""
    A = inputs.from_spectrum(m, n, np.geomspace(1.0, 1e-3, min(m, n)), 23 + m)
    buf = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    buf[:, :m] = torch.as_tensor(A.T, device="cuda")
    dA = buf.t()[:m, :]  # column-major view, stride(1) = lda
    f = q.factor(dA, 0.15, 0.9, kmax, precision=precision, trace=True)
    torch.cuda.synchronize()
    Ag = dA.cpu().numpy()
    res, orth = factorization_errors(A, Ag, f.htau.cpu().numpy(), f.perm.cpu().numpy().astype(np.int64))
    odd_starts = int(np.sum(np.asarray(f.trace["ns"]) % 2))
    print(f"\n[precision {precision}] {m}x{n} lda {lda} k_max {kmax}: residual {res:.2e}, orth {orth:.1e}, "
          f"steps {f.nsteps}, odd panel starts {odd_starts}")
    assert res <= BOUNDS[precision][0], res
    assert orth <= 1e-13, orth


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("kmax", [2, 3, 16])
def test_tensor_core_forms_small_blocks(kmax, precision):
    """Blocks of a few columns: the W pass's segment partials must fit the
    workspace whatever k_max is (their region is sized for the tensor-core
    forms, not from k_max)."""
    m, n, r = 600, 400, 150
    A = inputs.from_spectrum(m, n, inputs.sigma_gap(n, r), 77)
    dA = q.colmajor(A)
    f = q.factor(dA, 0.15, 0.9, kmax, precision=precision)
    torch.cuda.synchronize()
    res, orth = factorization_errors(A, dA.cpu().numpy(), f.htau.cpu().numpy(), f.perm.cpu().numpy().astype(np.int64))
    print(f"\n[precision {precision}] k_max {kmax}: residual {res:.2e}, orth {orth:.1e}, rank_colmax {f.rank_colmax}, "
          f"steps {f.nsteps}")
    assert res <= BOUNDS[precision][0], res
    assert orth <= 1e-13, orth
    assert r <= f.rank_colmax <= r + kmax, (f.rank_colmax, r)
