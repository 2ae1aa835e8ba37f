"""GB300-native QRDM: rank-revealing Householder QR with Deviation Maximization
pivoting (Dessole & Marcuzzi, 2021), as hand-written sm_103a CUDA kernels
behind the C ABI of include/qrdm.h.

``factor`` is a convenience wrapper: it allocates the outputs and the
workspace with PyTorch (device memory and the current stream only) and calls
``qrdm_factor`` through ctypes.  The factorization itself runs entirely in the
library's kernels; there is no CPU path.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ._binding import (  # noqa: F401
    EXPORTS,
    QRDM_ERR_CHECKED,
    QRDM_ERR_CUDA,
    QRDM_ERR_INTERNAL,
    QRDM_ERR_TIMEOUT,
    QRDM_FAIL_CHECK,
    QRDM_FAIL_GRID_BARRIER,
    QRDM_FAIL_MMA_WAIT,
    QRDM_FAIL_PIVOT_RANGE,
    QRDM_ERR_NONFINITE,
    QRDM_ERR_UNSUPPORTED,
    QRDM_ERR_WORKSPACE,
    QRDM_KMAX_LIMIT,
    QRDM_OK,
    load,
    qrdm_factor,
    qrdm_info,
    KERNEL_NAMES,
    qrdm_opts,
    qrdm_policy,
    qrdm_profile,
    qrdm_step_record,
    qrdm_strerror,
    qrdm_workspace_size,
)
from .batched import BatchPlan, BatchResult  # noqa: F401,E402

TRACE_DTYPE = np.dtype([("ns", np.int64), ("jstar", np.int64), ("ncand_all", np.int64), ("ncand", np.int64),
                        ("k", np.int64), ("l", np.int64), ("dm_on", np.int64), ("nrecomp", np.int64),
                        ("mu", np.float64), ("eps_s", np.float64)])


class QRDMError(RuntimeError):
    """A nonzero return code; ``info`` (a qrdm_info, when the call returns
    one) carries the device-side failure record (fail_code, fail_cta,
    fail_step, fail_ns, fail_value)."""

    def __init__(self, code: int, where: str = "qrdm_factor", info=None):
        self.code = code
        self.info = info
        msg = f"{where} failed: {code} ({qrdm_strerror(code)})"
        if info is not None and getattr(info, "fail_code", 0):
            msg += (f" [fail_code {info.fail_code}, cta {info.fail_cta}, step {info.fail_step}, "
                    f"ns {info.fail_ns}, value {info.fail_value}]")
        super().__init__(msg)


@dataclass
class Factorization:
    A: object          # torch tensor (m x n, column-major): R above, reflector tails below the diagonal
    htau: object       # torch float64 (min(m, n),)
    perm: object       # torch int32 (n,)
    rank: int
    rank_colmax: int
    nsteps: int
    launches: int = 0
    trace: np.ndarray | None = None   # TRACE_DTYPE records, one per block step
    J: np.ndarray | None = None       # (nsteps, k_max) original indices of the picked columns


def make_opts(eps1_mode=0, stop_at_rank=False, check_last=False, no_break=False, sdd=False, max_steps=0,
              profile: qrdm_profile | None = None, precision: int = 0,
              policy: qrdm_policy | None = None, checked: bool = False, wait_limit_us: int = 0,
              test_fault: int = 0) -> qrdm_opts:
    import ctypes

    o = qrdm_opts()
    if profile is not None:
        o.profile = ctypes.pointer(profile)
    if policy is not None:
        o.policy = ctypes.pointer(policy)
    o.eps1_mode = int(eps1_mode)
    o.stop_at_rank = int(bool(stop_at_rank))
    o.check_last = int(bool(check_last))
    o.no_break = int(bool(no_break))
    o.sdd = int(bool(sdd))
    o.max_steps = int(max_steps)
    o.precision = int(precision)
    o.checked = int(bool(checked))
    o.wait_limit_us = int(wait_limit_us)
    o.test_fault = int(test_fault)
    return o


def colmajor(A, device="cuda"):
    """A column-major (Fortran-order) float64 CUDA tensor holding A."""
    import torch

    if isinstance(A, np.ndarray):
        t = torch.from_numpy(np.asfortranarray(A, dtype=np.float64))
    else:
        t = A
    t = t.to(device=device, dtype=torch.float64)
    if t.dim() != 2:
        raise ValueError("A must be 2-D")
    m, n = t.shape
    if (m > 1 and t.stride(0) != 1) or (n > 1 and t.stride(1) < max(1, m)):
        t = t.t().contiguous().t()
    return t


def factor(A, tau: float = 0.9, delta: float = 0.9, k_max: int = 32, *, eps1_mode: int = 0,
           stop_at_rank: bool = False, check_last: bool = False, no_break: bool = False, sdd: bool = False,
           max_steps: int = 0, trace: bool = False, workspace=None, out_htau=None, out_perm=None,
           stream=None, profile: qrdm_profile | None = None, precision: int = 0,
           policy: qrdm_policy | None = None, checked: bool = False, wait_limit_us: int = 0,
           test_fault: int = 0) -> Factorization:
    """Factor A Pi = Q R in place.  ``A`` is a CUDA float64 tensor with
    stride(0) == 1 (column-major, lda = stride(1)).  ``precision`` selects the
    arithmetic of the trailing update: 0 FP64, 1 FP32 on the CUDA cores, 2
    split-BF16x3 and 3 3xTF32 on the tensor cores, 4 the tensor-core forms'
    merged update in FP64 (include/qrdm.h states each)."""
    import torch

    if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2):
        raise ValueError("A must be a 2-D float64 CUDA tensor")
    m, n = A.shape
    if m > 1 and A.stride(0) != 1:
        raise ValueError("A must be column-major (stride(0) == 1)")
    lda = A.stride(1) if n > 1 else max(m, 1)
    if m * n and lda < max(m, 1):
        raise ValueError("A's column stride is smaller than its row count")
    kmin = min(m, n)
    dev = A.device
    htau = out_htau if out_htau is not None else torch.empty(max(kmin, 1), dtype=torch.float64, device=dev)
    perm = out_perm if out_perm is not None else torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    wbytes = qrdm_workspace_size(m, n, k_max)
    if workspace is None:
        workspace = torch.empty(wbytes, dtype=torch.uint8, device=dev)
    tr = trJ = None
    cap = 0
    if trace:
        cap = max(kmin, 1) + 1
        tr = torch.zeros(cap * TRACE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        trJ = torch.empty(cap * k_max, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    opts = make_opts(eps1_mode, stop_at_rank, check_last, no_break, sdd, max_steps, profile, precision, policy,
                     checked, wait_limit_us, test_fault)
    rc, info = qrdm_factor(A.data_ptr() if m * n else 0, m, n, lda, float(tau), float(delta), int(k_max),
                           htau.data_ptr(), perm.data_ptr(), opts, workspace.data_ptr(), workspace.numel(),
                           s.cuda_stream, tr.data_ptr() if tr is not None else 0,
                           trJ.data_ptr() if trJ is not None else 0, cap)
    if rc != 0:
        raise QRDMError(rc, info=info)
    out = Factorization(A=A, htau=htau[:kmin], perm=perm[:n], rank=int(info.rank), rank_colmax=int(info.rank_colmax),
                        nsteps=int(info.nsteps), launches=int(info.launches))
    if trace:
        ns = min(out.nsteps, cap)
        out.trace = np.frombuffer(tr.cpu().numpy().tobytes(), dtype=TRACE_DTYPE)[:ns].copy()
        out.J = trJ.cpu().numpy().reshape(cap, k_max)[:ns].copy()
    return out


def ls_solve(A_orig, f: Factorization, b, rank: int | None = None, refine: int = 0, stream=None):
    """Basic least-squares solution of min ||A x - b|| from a factorization
    ``f`` of A (``factor``), with ``refine`` FP64 refinement iterations on the
    original matrix ``A_orig`` (column-major float64 CUDA tensor, unchanged).
    ``b``: CUDA float64 (m,) or (m, nrhs).  Returns (x, residual norms per
    iteration as a numpy array (refine + 1, nrhs), or None without A_orig)."""
    import ctypes

    import torch

    from . import _binding as _b

    QR = f.A
    m, n = QR.shape
    r = f.rank if rank is None else int(rank)
    vec = b.dim() == 1
    B = (b[:, None] if vec else b).to(torch.float64)
    B = B.t().contiguous().t() if B.shape[1] > 1 else B.contiguous()
    nrhs = B.shape[1]
    X = torch.zeros((nrhs, n), dtype=torch.float64, device=QR.device).t()
    sz = ctypes.c_size_t(0)
    rc = _b.load().qrdm_ls_workspace_size(m, n, r, nrhs, ctypes.byref(sz))
    if rc != 0:
        raise QRDMError(rc, "qrdm_ls_workspace_size")
    ws = torch.empty(max(int(sz.value), 16), dtype=torch.uint8, device=QR.device)
    resid = np.zeros((refine + 1, nrhs)) if A_orig is not None else None
    s = stream if stream is not None else torch.cuda.current_stream(QR.device)
    lda = A_orig.stride(1) if A_orig is not None and n > 1 else max(m, 1)
    rc = _b.load().qrdm_ls_solve(A_orig.data_ptr() if A_orig is not None else None, lda, QR.data_ptr(),
                                 QR.stride(1) if n > 1 else max(m, 1), m, n, f.htau.data_ptr(), f.perm.data_ptr(),
                                 r, B.data_ptr(), B.stride(1) if nrhs > 1 else max(m, 1), nrhs, X.data_ptr(),
                                 X.stride(1) if nrhs > 1 else max(n, 1), int(refine),
                                 resid.ctypes.data if resid is not None else None, ws.data_ptr(), ws.numel(),
                                 s.cuda_stream)
    if rc != 0:
        raise QRDMError(rc, "qrdm_ls_solve")
    return (X[:, 0] if vec else X), resid


def qp3_factor(A, nb: int = 32, *, eps1_mode: int = 0, workspace=None, stream=None) -> Factorization:
    """Comparator: blocked QR with column pivoting (lazy updates, block nb)
    of the column-major float64 CUDA tensor A, in place (see
    qrdm_qp3_factor in include/qrdm.h)."""
    import ctypes

    import torch

    from . import _binding as _b

    if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2):
        raise ValueError("A must be a 2-D float64 CUDA tensor")
    m, n = A.shape
    if m * n and m > 1 and A.stride(0) != 1:
        raise ValueError("A must be column-major (stride(0) == 1)")
    lda = A.stride(1) if (n > 1 and m * n) else max(m, 1)
    kmin = min(m, n)
    htau = torch.empty(max(kmin, 1), dtype=torch.float64, device=A.device)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    sz = ctypes.c_size_t(0)
    rc = _b.load().qrdm_qp3_workspace_size(m, n, nb, ctypes.byref(sz))
    if rc != 0:
        raise QRDMError(rc, "qrdm_qp3_workspace_size")
    if workspace is None or workspace.numel() < sz.value:
        workspace = torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=A.device)
    info = qrdm_info()
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    rc = _b.load().qrdm_qp3_factor(A.data_ptr() if m * n else None, m, n, lda, nb, htau.data_ptr(), perm.data_ptr(),
                                   ctypes.byref(info), int(eps1_mode), workspace.data_ptr(), workspace.numel(),
                                   s.cuda_stream)
    if rc != 0:
        raise QRDMError(rc, "qrdm_qp3_factor")
    return Factorization(A=A, htau=htau[:kmin], perm=perm[:n], rank=int(info.rank),
                         rank_colmax=int(info.rank_colmax), nsteps=int(info.nsteps), launches=int(info.launches))
