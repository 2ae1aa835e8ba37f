"""qrdm_factor_noalloc: the factorization for callers that cannot allocate
device memory (it works in a fixed scratch array inside the library's device
image).  Called through the C ABI, it must give what qrdm_factor gives on the
same input, on consecutive calls that share the scratch; shapes too large for
the scratch must be refused before any work.

Kept in its own file, collected last, so a run that stops at the first
failure has run every other test first."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2106_03138_gb300 import inputs
from tests._parity import rdiag_tol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2106_03138_gb300 as q  # noqa: E402
from paper_2106_03138_gb300 import _binding as b  # noqa: E402


def _reference(A, tau, delta, kmax):
    dA = q.colmajor(A)
    f = q.factor(dA, tau, delta, kmax)
    torch.cuda.synchronize()
    return dA.cpu().numpy(), f.htau.cpu().numpy(), f.perm.cpu().numpy(), f.rank, f.rank_colmax


@pytest.mark.parametrize("shape,kmax", [((600, 450), 32), ((1024, 1024), 64)])
def test_noalloc_matches_qrdm_factor_on_consecutive_calls(shape, kmax):
    m, n = shape
    A = inputs.from_spectrum(m, n, inputs.sigma_geometric(min(m, n), 1e-13), 77)
    tau, delta = 0.15, 0.9
    need = b.qrdm_workspace_size(m, n, kmax)
    assert need <= b.QRDM_NOALLOC_SCRATCH_BYTES
    Aref, href, pref, rank, rank_cm = _reference(A, tau, delta, kmax)
    anorm = float(np.max(np.linalg.norm(A, axis=0)))
    tol = rdiag_tol(np.diag(Aref), anorm, m)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        dA = q.colmajor(A)
        htau = torch.empty(min(m, n), dtype=torch.float64, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        rc, info = b.qrdm_factor_noalloc(dA.data_ptr(), m, n, dA.stride(1), tau, delta, kmax, htau.data_ptr(),
                                         perm.data_ptr(), None, stream)
        torch.cuda.synchronize()
        assert rc == 0, (call, rc, b.qrdm_strerror(rc))
        got = dA.cpu().numpy()
        assert np.array_equal(perm.cpu().numpy(), pref), call
        assert info.rank == rank and info.rank_colmax == rank_cm
        assert np.all(np.abs(np.abs(np.diag(got)) - np.abs(np.diag(Aref))) <= tol), call
        assert np.max(np.abs(got - Aref)) <= 1e-12 * anorm, call
        np.testing.assert_allclose(htau.cpu().numpy(), href, rtol=0, atol=1e-12)


def test_noalloc_refuses_shapes_beyond_the_scratch():
    m, n, kmax = 64, 65536, 128
    assert b.qrdm_workspace_size(m, n, kmax) > b.QRDM_NOALLOC_SCRATCH_BYTES
    # real buffers, so that nothing could go out of bounds even if it ran
    dA = torch.zeros((m, n), dtype=torch.float64, device="cuda").t().contiguous().t()
    htau = torch.zeros(m, dtype=torch.float64, device="cuda")
    perm = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    rc, _ = b.qrdm_factor_noalloc(dA.data_ptr(), m, n, m, 0.5, 0.5, kmax, htau.data_ptr(), perm.data_ptr(), None,
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == b.QRDM_ERR_WORKSPACE
    assert torch.all(perm == -7)


def test_noalloc_empty_matrix_writes_identity_permutation():
    perm = torch.full((5,), -1, dtype=torch.int32, device="cuda")
    rc, info = b.qrdm_factor_noalloc(0, 0, 5, 1, 0.5, 0.5, 4, 0, perm.data_ptr(), None,
                                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0 and info.rank == 0
    assert perm.cpu().tolist() == [0, 1, 2, 3, 4]
