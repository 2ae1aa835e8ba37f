"""ctypes binding of libqrdm.so: the C ABI of include/qrdm.h, same names.

Argument marshalling only.  Every step of the factorization runs in the
library's CUDA kernels; nothing here computes.  There is no fallback: if the
library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_i32, c_i64, c_f64, c_p, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t

QRDM_OK = 0
QRDM_ERR_CUDA = 1
QRDM_ERR_NONFINITE = 2
QRDM_ERR_WORKSPACE = 3
QRDM_ERR_UNSUPPORTED = 4
QRDM_ERR_INTERNAL = 5
QRDM_ERR_TIMEOUT = 6
QRDM_ERR_CHECKED = 7
QRDM_FAIL_NONE = 0
QRDM_FAIL_GRID_BARRIER = 1
QRDM_FAIL_PIVOT_RANGE = 2
QRDM_FAIL_MMA_WAIT = 4
QRDM_FAIL_CHECK = 8
QRDM_KMAX_LIMIT = 128


KERNEL_NAMES = ("k_colnorm_init", "k_select", "k_gram", "k_gram_reduce", "k_pick", "k_permute", "k_panel",
                "k_trail_w", "k_trail_wreduce", "k_trail_update", "k_downdate", "k_step_end", "k_qrp_tail",
                "k_tc_vtv+k_tc_tbuild", "k_tc_vimg", "k_tc_wsum", "k_tc_w", "k_tc_update")


class qrdm_profile(ctypes.Structure):
    _fields_ = [("ms", c_f64 * 24), ("flops", c_f64 * 24), ("launches", c_i64 * 24)]


class qrdm_policy(ctypes.Structure):
    _fields_ = [("d_weights", c_p), ("d_feat_log", c_p), ("d_act_log", c_p), ("log_cap", c_i64),
                ("tau_lo", c_f64), ("tau_hi", c_f64), ("delta_lo", c_f64), ("delta_hi", c_f64), ("rho_min", c_f64)]


QRDM_POLICY_NFEAT = 16
QRDM_POLICY_HIDDEN = 64
QRDM_POLICY_NPARAM = 5378


class qrdm_opts(ctypes.Structure):
    _fields_ = [("eps1_mode", c_i32), ("stop_at_rank", c_i32), ("check_last", c_i32), ("no_break", c_i32),
                ("sdd", c_i32), ("max_steps", c_i32), ("precision", c_i32), ("checked", c_i32),
                ("profile", ctypes.POINTER(qrdm_profile)), ("policy", ctypes.POINTER(qrdm_policy)),
                ("wait_limit_us", c_i64), ("test_fault", c_i32), ("reserved2", c_i32)]


class qrdm_info(ctypes.Structure):
    _fields_ = [("rank", c_i64), ("rank_colmax", c_i64), ("nsteps", c_i64), ("launches", c_i64),
                ("cuda_error", c_i32), ("fail_code", c_i32), ("fail_cta", c_i32), ("reserved", c_i32),
                ("fail_step", c_i64), ("fail_ns", c_i64), ("fail_value", c_i64)]


class qrdm_step_record(ctypes.Structure):
    _fields_ = [("ns", c_i64), ("jstar", c_i64), ("ncand_all", c_i64), ("ncand", c_i64), ("k", c_i64), ("l", c_i64),
                ("dm_on", c_i64), ("nrecomp", c_i64), ("mu", c_f64), ("eps_s", c_f64)]


class qrdm_batch_matrix(ctypes.Structure):
    _fields_ = [("dA", c_p), ("m", c_i64), ("n", c_i64), ("lda", c_i64), ("d_htau", c_p), ("d_perm", c_p),
                ("d_trace", c_p), ("d_trace_J", c_p), ("trace_cap", c_i64), ("d_feat_log", c_p), ("d_act_log", c_p),
                ("log_cap", c_i64)]


class qrdm_batch_tuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", c_i32), ("rows_per_pass", c_i32), ("lanes_per_col", c_i32), ("reserved", c_i32)]

    def as_dict(self) -> dict:
        return {"ctas_per_sm": int(self.ctas_per_sm), "rows_per_pass": int(self.rows_per_pass),
                "lanes_per_col": int(self.lanes_per_col)}


QRDM_BATCH_MAX_CTAS_PER_SM = 2

# every symbol declared in include/qrdm.h
EXPORTS = ("qrdm_workspace_size", "qrdm_factor", "qrdm_factor_noalloc", "qrdm_strerror", "qrdm_last_cuda_error",
           "qrdm_version", "qrdm_batch_plan_create", "qrdm_batch_plan_destroy", "qrdm_batch_workspace_size",
           "qrdm_batch_bind", "qrdm_batch_get_tuning", "qrdm_batch_set_tuning", "qrdm_batch_autotune",
           "qrdm_factor_batched", "qrdm_factor_batched_graph", "qrdm_batch_results", "qrdm_mlp_workspace_size",
           "qrdm_mlp_init", "qrdm_mlp_to_bf16", "qrdm_mlp_forward", "qrdm_mlp_loss_grad", "qrdm_mlp_adam_step",
           "qrdm_mlp_train", "qrdm_ls_workspace_size", "qrdm_ls_solve", "qrdm_qp3_workspace_size",
           "qrdm_qp3_factor", "qrdm_fp64_probe")
QRDM_NOALLOC_SCRATCH_BYTES = 32 << 20

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libqrdm.so (building it first if needed).  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"libqrdm.so not built ({_build.LIB}); run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        lib.qrdm_workspace_size.restype = ctypes.c_int
        lib.qrdm_workspace_size.argtypes = [c_i64, c_i64, c_i32, ctypes.POINTER(c_sz)]
        lib.qrdm_factor.restype = ctypes.c_int
        lib.qrdm_factor.argtypes = [c_p, c_i64, c_i64, c_i64, c_f64, c_f64, c_i32, c_p, c_p, ctypes.POINTER(qrdm_info),
                                    ctypes.POINTER(qrdm_opts), c_p, c_sz, c_p, c_p, c_p, c_i64]
        lib.qrdm_factor_noalloc.restype = ctypes.c_int
        lib.qrdm_factor_noalloc.argtypes = [c_p, c_i64, c_i64, c_i64, c_f64, c_f64, c_i32, c_p, c_p,
                                            ctypes.POINTER(qrdm_info), ctypes.POINTER(qrdm_opts), c_p, c_p, c_p,
                                            c_i64]
        lib.qrdm_fp64_probe.restype = ctypes.c_int
        lib.qrdm_fp64_probe.argtypes = [c_i32, c_i32, c_i32, c_p, c_sz, ctypes.POINTER(c_f64),
                                        ctypes.POINTER(ctypes.c_float), c_p]
        lib.qrdm_strerror.restype = ctypes.c_char_p
        lib.qrdm_strerror.argtypes = [ctypes.c_int]
        lib.qrdm_last_cuda_error.restype = ctypes.c_int
        lib.qrdm_last_cuda_error.argtypes = []
        lib.qrdm_version.restype = ctypes.c_int
        lib.qrdm_version.argtypes = []
        P = ctypes.POINTER
        lib.qrdm_batch_plan_create.restype = ctypes.c_int
        lib.qrdm_batch_plan_create.argtypes = [c_i64, P(qrdm_batch_matrix), c_i32, P(c_p)]
        lib.qrdm_batch_plan_destroy.restype = None
        lib.qrdm_batch_plan_destroy.argtypes = [c_p]
        lib.qrdm_batch_workspace_size.restype = ctypes.c_int
        lib.qrdm_batch_workspace_size.argtypes = [c_p, P(c_sz)]
        lib.qrdm_batch_bind.restype = ctypes.c_int
        lib.qrdm_batch_bind.argtypes = [c_p, c_p, c_sz, c_p]
        lib.qrdm_batch_get_tuning.restype = ctypes.c_int
        lib.qrdm_batch_get_tuning.argtypes = [c_p, P(qrdm_batch_tuning)]
        lib.qrdm_batch_set_tuning.restype = ctypes.c_int
        lib.qrdm_batch_set_tuning.argtypes = [c_p, P(qrdm_batch_tuning)]
        lib.qrdm_batch_autotune.restype = ctypes.c_int
        lib.qrdm_batch_autotune.argtypes = [c_p, c_f64, c_f64, P(qrdm_opts), c_p, P(qrdm_batch_tuning),
                                            P(c_f64)]
        lib.qrdm_factor_batched.restype = ctypes.c_int
        lib.qrdm_factor_batched.argtypes = [c_p, c_f64, c_f64, P(qrdm_opts), c_p]
        lib.qrdm_factor_batched_graph.restype = ctypes.c_int
        lib.qrdm_factor_batched_graph.argtypes = [c_p, c_f64, c_f64, P(qrdm_opts), c_p]
        lib.qrdm_batch_results.restype = ctypes.c_int
        lib.qrdm_batch_results.argtypes = [c_p, c_p, c_p, c_p, c_p, c_p]
        f32, u64 = ctypes.c_float, ctypes.c_uint64
        for name, args in (("qrdm_mlp_workspace_size", [c_i64, P(c_sz)]),
                           ("qrdm_mlp_init", [c_p, c_p, u64, c_p]),
                           ("qrdm_mlp_to_bf16", [c_p, c_p, c_p]),
                           ("qrdm_mlp_forward", [c_p, c_p, c_i64, c_p, c_p, c_sz, c_p]),
                           ("qrdm_mlp_loss_grad", [c_p, c_p, c_p, c_i64, c_p, c_p, c_p, c_sz, c_p]),
                           ("qrdm_mlp_adam_step", [c_p, c_p, c_p, c_p, c_p, c_i64, f32, f32, f32, f32, f32, c_p]),
                           ("qrdm_mlp_train", [c_p, c_p, c_p, c_p, c_p, c_i64, c_i64, c_i64, f32, f32, u64, c_p,
                                               c_p, c_sz, c_p])):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        lib.qrdm_qp3_workspace_size.restype = ctypes.c_int
        lib.qrdm_qp3_workspace_size.argtypes = [c_i64, c_i64, c_i32, P(c_sz)]
        lib.qrdm_qp3_factor.restype = ctypes.c_int
        lib.qrdm_qp3_factor.argtypes = [c_p, c_i64, c_i64, c_i64, c_i32, c_p, c_p, P(qrdm_info), c_i32, c_p, c_sz,
                                        c_p]
        lib.qrdm_ls_workspace_size.restype = ctypes.c_int
        lib.qrdm_ls_workspace_size.argtypes = [c_i64, c_i64, c_i64, c_i64, P(c_sz)]
        lib.qrdm_ls_solve.restype = ctypes.c_int
        lib.qrdm_ls_solve.argtypes = [c_p, c_i64, c_p, c_i64, c_i64, c_i64, c_p, c_p, c_i64, c_p, c_i64, c_i64, c_p,
                                      c_i64, ctypes.c_int32, c_p, c_p, c_sz, c_p]
        _lib = lib
        return lib


def qrdm_workspace_size(m: int, n: int, k_max: int) -> int:
    out = c_sz(0)
    rc = load().qrdm_workspace_size(m, n, k_max, ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"qrdm_workspace_size: invalid argument {-rc}")
    return int(out.value)


def qrdm_strerror(code: int) -> str:
    return load().qrdm_strerror(code).decode()


def qrdm_factor(dA: int, m: int, n: int, lda: int, tau: float, delta: float, k_max: int, d_htau: int, d_perm: int,
                opts: qrdm_opts | None, d_work: int, work_bytes: int, stream: int, d_trace: int = 0,
                d_trace_J: int = 0, trace_cap: int = 0) -> tuple[int, qrdm_info]:
    """Direct call of the C entry point (device addresses as ints)."""
    info = qrdm_info()
    rc = load().qrdm_factor(dA, m, n, lda, tau, delta, k_max, d_htau, d_perm, ctypes.byref(info),
                            ctypes.byref(opts) if opts is not None else None, d_work, work_bytes, stream,
                            d_trace or None, d_trace_J or None, trace_cap)
    return rc, info


def qrdm_factor_noalloc(dA: int, m: int, n: int, lda: int, tau: float, delta: float, k_max: int, d_htau: int,
                        d_perm: int, opts: qrdm_opts | None, stream: int, d_trace: int = 0, d_trace_J: int = 0,
                        trace_cap: int = 0) -> tuple[int, qrdm_info]:
    """Direct call of the allocation-free entry point (fixed device scratch)."""
    info = qrdm_info()
    rc = load().qrdm_factor_noalloc(dA, m, n, lda, tau, delta, k_max, d_htau, d_perm, ctypes.byref(info),
                                    ctypes.byref(opts) if opts is not None else None, stream, d_trace or None,
                                    d_trace_J or None, trace_cap)
    return rc, info


def _opts_ref(opts):
    return ctypes.byref(opts) if opts is not None else None


def qrdm_batch_plan_create(mats, k_max: int) -> tuple[int, int]:
    """mats: sequence of qrdm_batch_matrix.  Returns (rc, plan handle or 0)."""
    arr = (qrdm_batch_matrix * max(len(mats), 1))(*mats)
    h = c_p(0)
    rc = load().qrdm_batch_plan_create(len(mats), arr, k_max, ctypes.byref(h))
    return rc, int(h.value or 0)


def qrdm_batch_plan_destroy(plan: int) -> None:
    load().qrdm_batch_plan_destroy(plan or None)


def qrdm_batch_workspace_size(plan: int) -> tuple[int, int]:
    out = c_sz(0)
    rc = load().qrdm_batch_workspace_size(plan or None, ctypes.byref(out))
    return rc, int(out.value)


def qrdm_batch_bind(plan: int, d_work: int, work_bytes: int, stream: int) -> int:
    return load().qrdm_batch_bind(plan or None, d_work or None, work_bytes, stream or None)


def qrdm_batch_get_tuning(plan: int) -> tuple[int, qrdm_batch_tuning]:
    t = qrdm_batch_tuning()
    rc = load().qrdm_batch_get_tuning(plan or None, ctypes.byref(t))
    return rc, t


def qrdm_batch_set_tuning(plan: int, tuning: qrdm_batch_tuning) -> int:
    return load().qrdm_batch_set_tuning(plan or None, ctypes.byref(tuning))


def qrdm_batch_autotune(plan: int, tau: float, delta: float, opts, stream: int) -> tuple[int, qrdm_batch_tuning, float]:
    t = qrdm_batch_tuning()
    ms = c_f64(0.0)
    rc = load().qrdm_batch_autotune(plan or None, tau, delta, _opts_ref(opts), stream or None, ctypes.byref(t),
                                    ctypes.byref(ms))
    return rc, t, float(ms.value)


def qrdm_factor_batched(plan: int, tau: float, delta: float, opts, stream: int) -> int:
    return load().qrdm_factor_batched(plan or None, tau, delta, _opts_ref(opts), stream or None)


def qrdm_factor_batched_graph(plan: int, tau: float, delta: float, opts, stream: int) -> int:
    return load().qrdm_factor_batched_graph(plan or None, tau, delta, _opts_ref(opts), stream or None)


def qrdm_batch_results(plan: int, h_rank: int, h_rank_colmax: int, h_status: int, h_steps: int, stream: int) -> int:
    return load().qrdm_batch_results(plan or None, h_rank or None, h_rank_colmax or None, h_status or None,
                                     h_steps or None, stream or None)


def qrdm_mlp_workspace_size(batch: int) -> int:
    out = c_sz(0)
    rc = load().qrdm_mlp_workspace_size(batch, ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"qrdm_mlp_workspace_size: invalid argument {-rc}")
    return int(out.value)


def qrdm_fp64_probe(which: int, blocks: int, iters: int, d_out: int, out_bytes: int, stream: int) -> tuple[int, float, float]:
    """FP64 rate probe: (rc, flops, ms) of one timed launch (include/qrdm.h)."""
    fl = c_f64(0.0)
    ms = ctypes.c_float(0.0)
    rc = load().qrdm_fp64_probe(which, blocks, iters, d_out, out_bytes, ctypes.byref(fl), ctypes.byref(ms), stream)
    return rc, float(fl.value), float(ms.value)
