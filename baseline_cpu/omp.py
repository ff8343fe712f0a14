"""The paper's multi-threaded CPU method (Sec. 4.1 mixed parallel strategy, Algorithm 1; OpenMP, plain C).

A context implementation: the benchmark times it on the host's cores beside the GPU path, and the test-suite
checks that it returns exactly the oracle's recovery.  It shares no code with the oracle (oracle/) or with the GPU
library; nothing on the GPU path calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "pdgrass_omp.c")
_LIB = os.path.join(_DIR, "libpdgrass_omp.so")
_lock = threading.Lock()
_lib = None

OK, UNDER_BUDGET = 0, 1


def build(force: bool = False) -> str:
    """Compile with gcc and OpenMP (no FMA contraction: one rounding per operation)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            L.omp_recover.restype = ctypes.c_int
            L.omp_recover.argtypes = [i64, P, P, P, P, f64, i32, i32, i64, i32, i64, P, P, i64, P]
            _lib = L
    return _lib


def recover(g, alpha: float, c: int = 2, score_mode: int = 0, k_override: int = -1, threads: int = 0,
            cutoff: int = -1):
    """Returns (status, ids[int32], scores[float64]): the first k recovered edges in recovery order.
    threads: OpenMP threads (0: the default); cutoff: subtask size from which inner parallelism is used
    (-1: min(1e5, 10 % of the off-tree edges))."""
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.float64)
    par = np.ascontiguousarray(g.parent, dtype=np.int32)
    m = int(rp[-1]) // 2
    cap = max(m - g.n + 1, 1)
    ids = np.zeros(cap, dtype=np.int32)
    sc = np.zeros(cap, dtype=np.float64)
    cnt = ctypes.c_int64(0)
    st = lib().omp_recover(int(g.n), rp.ctypes.data, col.ctypes.data, w.ctypes.data, par.ctypes.data, float(alpha),
                           int(c), int(score_mode), int(k_override), int(threads), int(cutoff), ids.ctypes.data,
                           sc.ctypes.data, cap, ctypes.byref(cnt))
    if st < 0:
        raise RuntimeError(f"omp_recover failed with status {st}")
    k = int(cnt.value)
    return st, ids[:k].copy(), sc[:k].copy()
