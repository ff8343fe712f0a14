"""The oracle's pins catch plausible mistakes.  Each case copies oracle/pdgrass_oracle.c, plants one mistake (a
dropped factor, a flipped tie order, a min turned into a max, a missing orientation, an off-by-one neighbourhood, a
rounding direction, a reversed sort), compiles the copy on the CPU and checks that the same independent statements
the pins use (the brute-force restatement in tests/bruteforce.py, scipy's spanning trees) reject it."""
from __future__ import annotations

import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2508_20403_gb300 import workloads as W
from tests import bruteforce as BF
from tests.helpers import random_small_graph
from tests.test_oracle_tree import _brute_force_tree, _edges, _weff_keys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pdgrass_oracle.c")

MUTANTS = {
    "score drops the weight": [("? R : w * R;", "? R : R;")],
    "ties prefer the larger id": [("return (a->id < b->id) ? -1 : (a->id > b->id);",
                                   "return (a->id > b->id) ? -1 : (a->id < b->id);")],
    "beta takes the larger side": [("int64_t bs = hu < hv ? hu : hv;", "int64_t bs = hu > hv ? hu : hv;")],
    "similarity ignores the crossed orientation": [
        ("int sim = (stamp_u[uu] == pos && stamp_v[vv] == pos) || (stamp_v[uu] == pos && stamp_u[vv] == pos);",
         "int sim = (stamp_u[uu] == pos && stamp_v[vv] == pos);")],
    "neighbourhoods one hop too wide": [("bfs_stamp(&t, o.u[i], b, stamp_u", "bfs_stamp(&t, o.u[i], b + 1, stamp_u"),
                                        ("bfs_stamp(&t, o.v[i], b, stamp_v", "bfs_stamp(&t, o.v[i], b + 1, stamp_v")],
    "budget rounds up": [("double kd = floor(alpha * (double)n);", "double kd = ceil(alpha * (double)n);")],
    "marked edges are still recovered": [("if (marked[pos]) continue; /* the \"continue\" branch */",
                                          "if (0) continue;")],
    "Kruskal takes the lightest edge first": [("if (x->key > y->key) return -1;\n  if (x->key < y->key) return 1;",
                                              "if (x->key < y->key) return -1;\n  if (x->key > y->key) return 1;")],
    "effective weight uses the smaller degree": [("log((double)(du > dv ? du : dv))", "log((double)(du < dv ? du : dv))")],
}


def _build(tmp_path, name, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, (name, old)
        src = src.replace(old, new)
    cfile = tmp_path / "mutant.c"
    cfile.write_text(src)
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(cfile),
                           "-lm"])
    L = ctypes.CDLL(str(so))
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.orc_recover.restype = ctypes.c_int
    L.orc_recover.argtypes = [i64, P, P, P, P, f64, i32, ctypes.c_int, i64, P, P, i64, P, P]
    L.orc_spanning_tree.restype = ctypes.c_int
    L.orc_spanning_tree.argtypes = [i64, P, P, P, ctypes.c_int, P]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _recover(L, g, alpha, c, k_override=-1):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.float64)
    par = np.ascontiguousarray(g.parent, dtype=np.int32)
    cap = max(g.m, 1)
    ids = np.zeros(cap, dtype=np.int32)
    sc = np.zeros(cap, dtype=np.float64)
    cnt = np.zeros(1, dtype=np.int64)
    st = L.orc_recover(g.n, _p(rp), _p(col), _p(w), _p(par), float(alpha), int(c), 0, int(k_override), _p(ids),
                       _p(sc), cap, _p(cnt), None)
    return ids[: int(cnt[0])].tolist() if st >= 0 else None


def _tree(L, g, kind):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.w, dtype=np.float64)
    par = np.zeros(g.n, dtype=np.int32)
    st = L.orc_spanning_tree(g.n, _p(rp), _p(col), _p(w), int(kind), _p(par))
    return par if st == 0 else None


def _caught(L):
    """True as soon as one independent statement disagrees with the (mutated) oracle."""
    rng = np.random.default_rng(2024)
    for _ in range(60):
        g = random_small_graph(rng, n_lo=4, n_hi=14, tree="mixed")
        c = int(rng.integers(1, 4))
        k = int(rng.integers(1, g.m + 1))
        if _recover(L, g, 0.0, c, k_override=k) != BF.greedy(g, k, c)[0]:
            return True
        alpha = float(rng.uniform(0.05, 0.6))
        if _recover(L, g, alpha, c) != BF.greedy(g, BF.budget(g.n, alpha), c)[0]:
            return True
    for _ in range(30):
        g = random_small_graph(rng, n_lo=3, n_hi=7)
        eu, ev, ew = _edges(g)
        if len(eu) > 12:
            continue
        if not np.array_equal(_tree(L, g, 0), _brute_force_tree(g, ew)):
            return True
        if not np.array_equal(_tree(L, g, 1), _brute_force_tree(g, _weff_keys(g, eu, ev, ew))):
            return True
    return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert _caught(_build(tmp_path, name, MUTANTS[name])), name


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no gcc")
def test_unmutated_copy_passes(tmp_path):
    assert not _caught(_build(tmp_path, "none", []))


PCG_MUTANTS = {
    "beta inverted": ("p = z + (rz_new / rz) * p", "p = z + (rz / rz_new) * p"),
    "step length from r.r": ("a = rz / (p @ Ap)", "a = (r @ r) / (p @ Ap)"),
    "stopping on the squared residual": ("rel = np.linalg.norm(r) / nb", "rel = (np.linalg.norm(r) / nb) ** 2"),
    "preconditioner ignores the recovered edges": ("LP = sparsifier_laplacian(g, edge_ids)",
                                                   "LP = sparsifier_laplacian(g, edge_ids[:0])"),
}


def _pcg_module(edit):
    import importlib.util
    import sys
    import types

    src = open(os.path.join(ROOT, "oracle", "pcg.py")).read()
    if edit:
        assert edit[0] in src, edit
        src = src.replace(edit[0], edit[1])
    mod = types.ModuleType("pcg_mutant")
    exec(compile(src, "pcg_mutant", "exec"), mod.__dict__)
    return mod


def _pcg_caught(PCm):
    """The pins' statements: scipy's own CG with the same exact preconditioner, and one iteration for L_P = L_G."""
    import scipy.sparse.linalg as spla

    from oracle import oracle as O

    g = W.grid_graph(30, seed=4)
    _, ids, _, _ = O.recover(g, 0.05, c=2)
    b = np.random.default_rng(1).standard_normal(g.n)
    it, _ = PCm.pcg_quality(g, ids, b, tol=1e-6)
    LG = PCm.laplacian_from_csr(g.n, g.row_ptr, g.col, g.w)
    from oracle import pcg as PC

    LP = PC.sparsifier_laplacian(g, ids)
    root = int(np.flatnonzero(g.parent < 0)[0])
    keep = np.flatnonzero(np.arange(g.n) != root)
    lu = spla.splu(LP[keep][:, keep].tocsc())

    def apply(r):
        z = np.zeros(g.n)
        z[keep] = lu.solve(np.asarray(r).ravel()[keep])
        return z - z.mean()

    count = [0]
    bc = b - b.mean()
    spla.cg(LG, bc, rtol=1e-6, atol=0.0, M=spla.LinearOperator((g.n, g.n), matvec=apply), maxiter=2000,
            callback=lambda xk: count.__setitem__(0, count[0] + 1))
    if abs(count[0] - it) > 1:
        return True
    off = O.offtree_scores(g, c=0)["id"]
    it_exact, _ = PCm.pcg_quality(g, off, b, tol=1e-8)
    return it_exact != 1


@pytest.mark.parametrize("name", sorted(PCG_MUTANTS))
def test_planted_pcg_mistake_is_caught(name):
    assert _pcg_caught(_pcg_module(PCG_MUTANTS[name])), name


def test_unmutated_pcg_passes():
    assert not _pcg_caught(_pcg_module(None))
