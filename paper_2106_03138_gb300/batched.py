"""Batched QRDM: many independent matrices factored by one persistent kernel
(the ``qrdm_batch_*`` entry points of include/qrdm.h).

``BatchPlan`` owns the plan handle, the workspace and the per-matrix outputs
(PyTorch device memory).  The matrices themselves are the caller's
column-major float64 CUDA tensors and are factored in place, as with
``factor``.  Argument marshalling only: every step runs in the library's
kernel.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import _binding as _b


@dataclass
class BatchResult:
    rank: np.ndarray         # int64 (count,)
    rank_colmax: np.ndarray  # int64 (count,)
    status: np.ndarray       # int32 (count,): 0 ok, 1 non-finite input (matrix untouched)
    steps: np.ndarray        # int64 (count,) block steps


class BatchPlan:
    """A list of column-major float64 CUDA matrices factored together.

    ``k_max`` caps every block; ``trace`` allocates a per-matrix step trace
    (as ``factor(trace=True)`` does).  The plan may be run many times; each
    run factors the tensors as they are at that moment."""

    def __init__(self, mats, k_max: int, *, trace: bool = False, policy_logs: bool = False, stream=None):
        import torch

        from . import QRDMError

        self._torch = torch
        self.mats = list(mats)
        self.k_max = int(k_max)
        dev = self.mats[0].device if self.mats else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.htau, self.perm, self._trace, self._traceJ, self._cap = [], [], [], [], []
        self._flog, self._alog = [], []
        descs = []
        for A in self.mats:
            if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 2):
                raise ValueError("every matrix must be a 2-D float64 CUDA tensor")
            m, n = A.shape
            if m * n and m > 1 and A.stride(0) != 1:
                raise ValueError("matrices must be column-major (stride(0) == 1)")
            lda = A.stride(1) if (n > 1 and m * n) else max(m, 1)
            if m * n and lda < max(m, 1):
                raise ValueError("a matrix's column stride is smaller than its row count")
            kmin = min(m, n)
            h = torch.empty(max(kmin, 1), dtype=torch.float64, device=dev)
            p = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
            self.htau.append(h)
            self.perm.append(p)
            d = _b.qrdm_batch_matrix(A.data_ptr() if m * n else None, m, n, lda, h.data_ptr(), p.data_ptr(),
                                     None, None, 0, None, None, 0)
            if trace:
                from . import TRACE_DTYPE

                cap = max(kmin, 1) + 1
                tr = torch.zeros(cap * TRACE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
                tj = torch.empty(cap * self.k_max, dtype=torch.int32, device=dev)
                d.d_trace, d.d_trace_J, d.trace_cap = tr.data_ptr(), tj.data_ptr(), cap
                self._trace.append(tr)
                self._traceJ.append(tj)
                self._cap.append(cap)
            if policy_logs:
                lcap = max(kmin, 1) + 1
                fl = torch.zeros((lcap, _b.QRDM_POLICY_NFEAT), dtype=torch.float32, device=dev)
                al = torch.zeros((lcap, 2), dtype=torch.float64, device=dev)
                d.d_feat_log, d.d_act_log, d.log_cap = fl.data_ptr(), al.data_ptr(), lcap
                self._flog.append(fl)
                self._alog.append(al)
            descs.append(d)
        rc, self._h = _b.qrdm_batch_plan_create(descs, self.k_max)
        if rc != 0:
            raise QRDMError(rc, "qrdm_batch_plan_create")
        rc, nbytes = _b.qrdm_batch_workspace_size(self._h)
        if rc != 0:
            raise QRDMError(rc, "qrdm_batch_workspace_size")
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        rc = _b.qrdm_batch_bind(self._h, self.workspace.data_ptr(), self.workspace.numel(), self._stream(stream))
        if rc != 0:
            raise QRDMError(rc, "qrdm_batch_bind")

    def _stream(self, stream):
        s = stream if stream is not None else self._torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def close(self):
        if getattr(self, "_h", 0):
            _b.qrdm_batch_plan_destroy(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def tuning(self) -> dict:
        rc, t = _b.qrdm_batch_get_tuning(self._h)
        return t.as_dict()

    def set_tuning(self, ctas_per_sm: int, rows_per_pass: int, lanes_per_col: int) -> None:
        from . import QRDMError

        rc = _b.qrdm_batch_set_tuning(self._h, _b.qrdm_batch_tuning(ctas_per_sm, rows_per_pass, lanes_per_col, 0))
        if rc != 0:
            raise QRDMError(rc, "qrdm_batch_set_tuning")

    def autotune(self, tau: float, delta: float, opts=None, stream=None) -> tuple[dict, float]:
        """Time every feasible tuning on these matrices (restored afterwards)."""
        from . import QRDMError

        rc, t, ms = _b.qrdm_batch_autotune(self._h, float(tau), float(delta), opts, self._stream(stream))
        if rc != 0:
            raise QRDMError(rc, "qrdm_batch_autotune")
        return t.as_dict(), ms

    def run(self, tau: float, delta: float, opts=None, *, graph: bool = False, stream=None) -> None:
        """Enqueue the factorization (no host synchronization unless ``opts``
        carries a profile)."""
        from . import QRDMError

        fn = _b.qrdm_factor_batched_graph if graph else _b.qrdm_factor_batched
        rc = fn(self._h, float(tau), float(delta), opts, self._stream(stream))
        if rc != 0:
            raise QRDMError(rc, "qrdm_factor_batched_graph" if graph else "qrdm_factor_batched")

    def results(self, stream=None) -> BatchResult:
        from . import QRDMError

        c = len(self.mats)
        r = BatchResult(np.zeros(c, np.int64), np.zeros(c, np.int64), np.zeros(c, np.int32), np.zeros(c, np.int64))
        rc = _b.qrdm_batch_results(self._h, r.rank.ctypes.data, r.rank_colmax.ctypes.data, r.status.ctypes.data,
                                   r.steps.ctypes.data, self._stream(stream))
        if rc != 0:
            raise QRDMError(rc, "qrdm_batch_results")
        return r

    def trace(self, i: int, nsteps: int):
        """(records, J) of matrix i's first ``nsteps`` block steps."""
        from . import TRACE_DTYPE

        cap = self._cap[i]
        ns = min(int(nsteps), cap)
        tr = np.frombuffer(self._trace[i].cpu().numpy().tobytes(), dtype=TRACE_DTYPE)[:ns].copy()
        J = self._traceJ[i].cpu().numpy().reshape(cap, self.k_max)[:ns].copy()
        return tr, J

    def policy_logs(self, i: int, nsteps: int):
        """(features [nsteps x 16], (tau_s, delta_s) [nsteps x 2]) of matrix i
        (rows of single-column steps after the stopping criterion are zero in
        the features)."""
        ns = min(int(nsteps), self._flog[i].shape[0])
        return self._flog[i][:ns].cpu().numpy(), self._alog[i][:ns].cpu().numpy()

    def outputs(self, i: int):
        """(htau, perm) views of matrix i."""
        m, n = self.mats[i].shape
        return self.htau[i][: min(m, n)], self.perm[i][:n]
