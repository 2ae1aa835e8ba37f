"""ctypes wrapper around the plain C QRDM oracle (qrdm_oracle.c).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the product path never does.

The oracle is a slow, single-threaded FP64 restatement of QRDM2 (Algorithm 4)
with Deviation Maximization (Algorithm 1) and the implementation choices of
Sec. 4; the readings it takes where the paper is silent are listed in the C
file's header.  Every function here is pinned by tests against values fixed
by the paper or the mathematics (see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qrdm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_LIB_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

EPS = 2.0 ** -52

STEP_DTYPE = np.dtype(
    [
        ("ns", np.int64),
        ("jstar", np.int64),
        ("ncand_all", np.int64),
        ("ncand", np.int64),
        ("k", np.int64),
        ("l", np.int64),
        ("dm_on", np.int64),
        ("nrecomp", np.int64),
        ("mu", np.float64),
        ("eps_s", np.float64),
        ("s_argmax", np.float64),
        ("s_cand", np.float64),
        ("s_order", np.float64),
        ("s_cos", np.float64),
        ("s_break", np.float64),
        ("s_stop", np.float64),
        ("s_recomp", np.float64),
        ("g_argmax", np.float64),
        ("g_cand", np.float64),
        ("g_cos", np.float64),
        ("g_break", np.float64),
        ("g_stop", np.float64),
    ]
)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, plain C)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False) -> str | None:
    """The same source with OpenMP on (the trailing update's column loops run
    on all host cores, with bit-identical results): oracle/_build/
    liboracle_omp.so, or None when the compiler has no OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_OMP) and os.path.getmtime(_LIB_OMP) >= os.path.getmtime(_SRC):
        return _LIB_OMP
    tmp = _LIB_OMP + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp,
           _SRC, "-lm"]
    if subprocess.run(cmd, capture_output=True).returncode != 0:
        return None
    os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _declare(lib):
    i64, f64, p = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.oq_qrdm.restype = ctypes.c_int
    lib.oq_qrdm.argtypes = [i64, i64, p, i64, f64, f64, i64, i64, i64, i64, i64, i64, i64, p, p, p, p, p, p,
                            p, i64, p, p]
    lib.oq_step_size.restype = i64
    assert lib.oq_step_size() == STEP_DTYPE.itemsize, "oracle trace layout mismatch"


def _load_omp():
    """The OpenMP build (None if unavailable)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            path = build_omp()
            if path is None:
                return None
            lib = ctypes.CDLL(path)
            _declare(lib)
            _lib_omp = lib
    return _lib_omp


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, f64, p = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.oq_qrdm.restype = ctypes.c_int
            lib.oq_qrdm.argtypes = [i64, i64, p, i64, f64, f64, i64, i64, i64, i64, i64, i64, i64, p, p, p, p, p, p,
                                    p, i64, p, p]
            lib.oq_qrdm_sched.restype = ctypes.c_int
            lib.oq_qrdm_sched.argtypes = [i64, i64, p, i64, f64, f64, i64, i64, i64, i64, i64, i64, i64, p, p, p, p, p,
                                          p, p, i64, p, p, p, p, i64]
            lib.oq_house.restype = None
            lib.oq_house.argtypes = [i64, p, p, p]
            lib.oq_larft.restype = None
            lib.oq_larft.argtypes = [i64, i64, p, i64, p, p, i64]
            lib.oq_cosine.restype = None
            lib.oq_cosine.argtypes = [i64, i64, p, i64, i64, p, p, p]
            lib.oq_step_size.restype = i64
            assert lib.oq_step_size() == STEP_DTYPE.itemsize, "oracle trace layout mismatch"
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def house(x):
    """Householder reflector of x: returns (beta, htau, v) with v[0] = 1."""
    lib = _load()
    x = np.array(x, dtype=np.float64)
    beta = np.zeros(1)
    ht = np.zeros(1)
    lib.oq_house(x.shape[0], _ptr(x), _ptr(beta), _ptr(ht))
    v = x.copy()
    v[0] = 1.0
    return float(beta[0]), float(ht[0]), v


def larft(V: np.ndarray, htau: np.ndarray) -> np.ndarray:
    """T (l x l, upper) with H_1 ... H_l = I - V T V^T; V unit lower trapezoidal."""
    lib = _load()
    V = np.asfortranarray(V, dtype=np.float64)
    mr, l = V.shape
    ht = np.ascontiguousarray(htau, dtype=np.float64)
    T = np.zeros((l, l), order="F")
    lib.oq_larft(mr, l, _ptr(V), max(mr, 1), _ptr(ht), _ptr(T), max(l, 1))
    return T


def cosine(A: np.ndarray, cols, r0: int = 0):
    """(G, Theta) for columns ``cols`` of A over rows r0..m-1."""
    lib = _load()
    A = np.asfortranarray(A, dtype=np.float64)
    m = A.shape[0]
    c = np.ascontiguousarray(cols, dtype=np.int64)
    kc = c.shape[0]
    G = np.zeros((kc, kc), order="F")
    Th = np.zeros((kc, kc), order="F")
    lib.oq_cosine(m, r0, _ptr(A), max(m, 1), kc, _ptr(c), _ptr(G), _ptr(Th))
    return G, Th


def qrdm(A: np.ndarray, tau: float = 0.9, delta: float = 0.9, k_max: int = 32, *, eps1_mode: int = 0,
         stop_at_rank: bool = False, check_last: bool = False, no_break: bool = False, sdd: bool = False,
         max_steps: int = 0, trace_cap: int | None = None, schedule=None, parallel: bool = False) -> dict:
    """Factor A Pi = Q R by QRDM2.  ``parallel``: run the OpenMP build (all
    host cores on the trailing update, identical results).  Returns a dict:

    ``A`` (R above the diagonal, reflector tails below), ``htau``, ``perm``,
    ``rank``, ``rank_colmax``, ``u``/``uref`` (partial norms at exit),
    ``trace`` (one record per block step, STEP_DTYPE), ``J`` (per step, the
    original indices of the selected columns, -1 padded), ``status``, and
    ``stop``: with ``stop_at_rank``, the record of the stopping test that
    ended the run (its margin ``s_stop``; ``k`` = -1), else None.
    """
    lib = _load()
    if parallel:
        if schedule is not None:
            raise ValueError("the OpenMP build takes no schedule")
        lib = _load_omp()
        if lib is None:
            raise RuntimeError("the oracle's OpenMP build is unavailable (no OpenMP in the C compiler)")
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = A.shape
    kmin = min(m, n)
    htau = np.zeros(max(kmin, 1))
    perm = np.zeros(max(n, 1), dtype=np.int64)
    rank = np.zeros(1, dtype=np.int64)
    rank_cm = np.zeros(1, dtype=np.int64)
    u = np.zeros(max(n, 1))
    uref = np.zeros(max(n, 1))
    cap = trace_cap if trace_cap is not None else max(kmin, 1)
    trace = np.zeros(cap, dtype=STEP_DTYPE)
    J = np.full((cap, k_max), -1, dtype=np.int64)
    nsteps = np.zeros(1, dtype=np.int64)
    if schedule is None:
        st = lib.oq_qrdm(m, n, _ptr(A), max(m, 1), float(tau), float(delta), int(k_max), int(eps1_mode),
                         int(stop_at_rank), int(check_last), int(no_break), int(sdd), int(max_steps), _ptr(htau),
                         _ptr(perm), _ptr(rank), _ptr(rank_cm), _ptr(u), _ptr(uref), _ptr(trace), cap, _ptr(J),
                         _ptr(nsteps))
    else:
        # per-step (tau, delta): schedule is an (S, 2) array
        sch = np.ascontiguousarray(np.asarray(schedule, dtype=np.float64).reshape(-1, 2))
        ts = np.ascontiguousarray(sch[:, 0])
        ds = np.ascontiguousarray(sch[:, 1])
        st = lib.oq_qrdm_sched(m, n, _ptr(A), max(m, 1), float(tau), float(delta), int(k_max), int(eps1_mode),
                               int(stop_at_rank), int(check_last), int(no_break), int(sdd), int(max_steps),
                               _ptr(htau), _ptr(perm), _ptr(rank), _ptr(rank_cm), _ptr(u), _ptr(uref), _ptr(trace),
                               cap, _ptr(J), _ptr(nsteps), _ptr(ts), _ptr(ds), int(sch.shape[0]))
    ns = int(nsteps[0])
    return {
        "status": int(st),
        "A": A,
        "htau": htau[:kmin],
        "perm": perm[:n],
        "rank": int(rank[0]),
        "rank_colmax": int(rank_cm[0]),
        "u": u[:n],
        "uref": uref[:n],
        "trace": trace[:min(ns, cap)],
        # the stopping test's record when the stop at the rank ended the run
        "stop": trace[ns].copy() if (ns < cap and int(trace[ns]["k"]) == -1) else None,
        "J": J[:min(ns, cap)],
        "nsteps": ns,
    }



def ls_basic(A: np.ndarray, b: np.ndarray, rank: int | None = None, fact: dict | None = None, **qrdm_kwargs):
    """Basic least-squares solution from the oracle's QRDM factorization:
    x = Pi [R11^{-1} (Q^T b)_{1:r}; 0], Q^T b by the reflectors H_1..H_r
    (H_j = I - htau_j v_j v_j^T, v_j(j) = 1, v_j below the diagonal of the
    factored matrix), R11 the leading r x r block.  ``fact``: a result of
    ``qrdm`` to reuse; ``rank`` defaults to its numerical rank."""
    import scipy.linalg

    A = np.asarray(A, dtype=np.float64)
    f = fact if fact is not None else qrdm(A, **qrdm_kwargs)
    F, htau, perm = f["A"], f["htau"], f["perm"]
    m, n = A.shape
    r = f["rank"] if rank is None else int(rank)
    y = np.array(b, dtype=np.float64).reshape(m, -1).copy()
    for j in range(r):
        v = np.concatenate([[1.0], F[j + 1:, j]])
        y[j:] -= htau[j] * np.outer(v, v @ y[j:])
    z = scipy.linalg.solve_triangular(np.triu(F[:r, :r]), y[:r], lower=False)
    x = np.zeros((n, y.shape[1]))
    x[perm[:r]] = z
    return x.reshape((n,) + np.shape(b)[1:])
