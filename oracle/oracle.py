"""ctypes wrapper around the plain C oracle (pdgrass_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdgrass_oracle.c")
_LIB = os.path.join(_HERE, "libpdgrass_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
UNDER_BUDGET = 1
SCORE_STRETCH = 0
SCORE_RESISTANCE = 1
METHOD_WALK = 0
METHOD_DISTS = 1
TREE_MAX_WEIGHT = 0
TREE_FEGRASS = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
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
            L.orc_exact_sum.restype = f64
            L.orc_exact_sum.argtypes = [P, i64]
            L.orc_offtree_scores.restype = ctypes.c_int
            L.orc_offtree_scores.argtypes = [i64, P, P, P, P, i32, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, P]
            L.orc_spanning_tree.restype = ctypes.c_int
            L.orc_spanning_tree.argtypes = [i64, P, P, P, ctypes.c_int, P]
            L.orc_recover.restype = ctypes.c_int
            L.orc_recover.argtypes = [i64, P, P, P, P, f64, i32, ctypes.c_int, i64, P, P, i64, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _graph_arrays(g):
    return (np.ascontiguousarray(g.row_ptr, dtype=np.int64), np.ascontiguousarray(g.col, dtype=np.int32),
            np.ascontiguousarray(g.w, dtype=np.float64), np.ascontiguousarray(g.parent, dtype=np.int32))


def exact_sum(xs) -> float:
    a = np.ascontiguousarray(xs, dtype=np.float64)
    return float(lib().orc_exact_sum(_p(a), a.shape[0]))


def offtree_scores(g, c: int = 2, score_mode: int = SCORE_STRETCH, method: int = METHOD_WALK) -> dict:
    """Per off-tree edge (canonical id order): u, v, id, lca, resistance, score, beta.
    method: METHOD_WALK (path walk, the definition) or METHOD_DISTS (Algorithm 1)."""
    rp, col, w, par = _graph_arrays(g)
    E = max(int(rp[-1]) // 2 - g.n + 1, 1)
    out = {k: np.zeros(E, dtype=np.int32) for k in ("u", "v", "id", "lca", "beta")}
    out["resistance"] = np.zeros(E, dtype=np.float64)
    out["score"] = np.zeros(E, dtype=np.float64)
    n_off = np.zeros(1, dtype=np.int64)
    st = lib().orc_offtree_scores(g.n, _p(rp), _p(col), _p(w), _p(par), c, score_mode, method, _p(n_off),
                                  _p(out["u"]), _p(out["v"]), _p(out["id"]), _p(out["lca"]),
                                  _p(out["resistance"]), _p(out["score"]), _p(out["beta"]))
    if st != OK:
        raise RuntimeError(f"oracle offtree_scores failed: {st}")
    k = int(n_off[0])
    return {key: val[:k] for key, val in out.items()}


def recover(g, alpha: float, c: int = 2, score_mode: int = SCORE_STRETCH, k_override: int = -1,
            full_count: bool = False):
    """Returns (status, ids[int32], scores[float64], full_pass_count or None)."""
    rp, col, w, par = _graph_arrays(g)
    m = int(rp[-1]) // 2
    cap = max(m - g.n + 1, 1)
    ids = np.zeros(cap, dtype=np.int32)
    sc = np.zeros(cap, dtype=np.float64)
    cnt = np.zeros(1, dtype=np.int64)
    full = np.zeros(1, dtype=np.int64)
    st = lib().orc_recover(g.n, _p(rp), _p(col), _p(w), _p(par), float(alpha), int(c), int(score_mode),
                           int(k_override), _p(ids), _p(sc), cap, _p(cnt),
                           _p(full) if full_count else None)
    if st < 0:
        raise RuntimeError(f"oracle recover failed: {st}")
    k = int(cnt[0])
    return st, ids[:k].copy(), sc[:k].copy(), (int(full[0]) if full_count else None)


def spanning_tree(g, kind: int = TREE_MAX_WEIGHT) -> np.ndarray:
    """Parent array of the maximum spanning forest for (key desc, id asc), key = w (TREE_MAX_WEIGHT) or the
    effective weight of Eq. weff (TREE_FEGRASS), each component rooted at its maximum-degree vertex."""
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.float64)
    parent = np.zeros(g.n, dtype=np.int32)
    st = lib().orc_spanning_tree(g.n, _p(rp), _p(col), _p(w), int(kind), _p(parent))
    if st != OK:
        raise ValueError(f"oracle spanning_tree failed: {st}")
    return parent
