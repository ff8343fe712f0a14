"""Pins of the oracle's PCG sparsifier-quality measure (Sec. 5 evaluation) against independent statements:
scipy's own conjugate gradients with the same preconditioner, the exact preconditioner (one iteration), and the
finite-termination bound by the number of distinct generalised eigenvalues on tiny graphs."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import oracle as O
from oracle import pcg as PC
from paper_2508_20403_gb300 import workloads as W
from tests import bruteforce as BF
from tests.helpers import random_small_graph


def _rhs(n, seed=0):
    return np.random.default_rng(seed).standard_normal(n)


def test_exact_preconditioner_converges_in_one_iteration():
    g = W.grid_graph(30)
    off = O.offtree_scores(g, c=0)["id"]
    it, rel = PC.pcg_quality(g, off, _rhs(g.n), tol=1e-8)
    assert it == 1 and rel <= 1e-8


@pytest.mark.parametrize("alpha", [0.02, 0.10])
def test_matches_scipy_cg(alpha):
    g = W.grid_graph(60, seed=4)
    _, ids, _, _ = O.recover(g, alpha, c=2)
    b = _rhs(g.n, 1)
    it, rel = PC.pcg_quality(g, ids, b, tol=1e-3)
    # scipy's CG with the same preconditioner and stopping rule
    LG = PC.laplacian_from_csr(g.n, g.row_ptr, g.col, g.w)
    LP = PC.sparsifier_laplacian(g, ids)
    root = int(np.flatnonzero(g.parent < 0)[0])
    keep = np.flatnonzero(np.arange(g.n) != root)
    lu = spla.splu(LP[keep][:, keep].tocsc())

    def apply(r):
        z = np.zeros(g.n)
        z[keep] = lu.solve(np.asarray(r).ravel()[keep])
        return z - z.mean()

    M = spla.LinearOperator((g.n, g.n), matvec=apply)
    count = [0]
    bc = b - b.mean()
    x, info = spla.cg(LG, bc, rtol=1e-3, atol=0.0, M=M, maxiter=1000, callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert info == 0
    assert abs(count[0] - it) <= 1
    assert np.linalg.norm(bc - LG @ x) / np.linalg.norm(bc) <= 1e-3


def test_iterations_bounded_by_distinct_eigenvalues():
    rng = np.random.default_rng(9)
    for _ in range(15):
        g = random_small_graph(rng, n_lo=4, n_hi=12, tree="max")
        off = O.offtree_scores(g, c=0)["id"]
        ids = off[: max(0, len(off) // 3)]
        it, rel = PC.pcg_quality(g, ids, _rhs(g.n, 3), tol=1e-9, max_iter=200)
        eu, ev, ew = PC.canonical_edges(g.n, g.row_ptr, g.col, g.w)
        LG = BF.laplacian(g.n, list(zip(eu, ev, ew)))
        LP = PC.sparsifier_laplacian(g, ids).toarray()
        ev_ = BF.generalized_eigs(LG, LP)
        distinct = len(np.unique(np.round(ev_, 6)))
        assert it <= distinct + 1, (it, distinct)


def test_recovered_edges_precondition_better_than_random():
    """The method's point (Sec. 5): the recovered (spectrally critical) edges give fewer PCG iterations than as
    many random off-tree edges, and a larger budget gives fewer iterations than a smaller one."""
    g = W.grid_graph(100)
    b = _rhs(g.n, 2)
    its = {}
    for alpha in (0.02, 0.10):
        _, ids, _, _ = O.recover(g, alpha, c=2)
        its[alpha], _ = PC.pcg_quality(g, ids, b)
        off = O.offtree_scores(g, c=0)["id"]
        rnd = np.random.default_rng(5).choice(off, size=len(ids), replace=False)
        it_rnd, _ = PC.pcg_quality(g, rnd, b)
        assert its[alpha] < it_rnd
    assert its[0.10] <= its[0.02]


def test_rank_k_update_terminates_in_k_plus_one_iterations():
    """L_G = L_P + (the k edges the preconditioner leaves out): the generalised spectrum is 1 plus at most k other
    values, so exact-arithmetic CG stops after at most k + 1 iterations (checked with k = 1, 2, 3 missing edges)."""
    g = W.grid_graph(12, seed=6)
    off = O.offtree_scores(g, c=0)["id"]
    b = _rhs(g.n, 7)
    for missing in (1, 2, 3):
        it, rel = PC.pcg_quality(g, off[missing:], b, tol=1e-10, max_iter=50)
        assert it <= missing + 1 and rel <= 1e-10, (missing, it, rel)


@pytest.mark.parametrize("alpha", [0.0, 0.05])
def test_trace_preconditioner_solves_the_sparsifier_system(alpha):
    """The z that pcg_trace reports is a solution of L_P z = b' with mean zero (the preconditioner's definition):
    checked by a product with a Laplacian assembled independently from the CSR and the parent array, and the
    residual history ends with the returned residual."""
    g = W.grid_graph(40, seed=5)
    ids = O.recover(g, alpha, c=2)[1] if alpha > 0 else np.zeros(0, dtype=np.int32)
    b = _rhs(g.n, 3)
    it, rel, hist, z0 = PC.pcg_trace(g, ids, b, tol=1e-3)
    bb = b - b.mean()
    # L_P from an edge list: the tree edges (v, parent v) plus the listed off-tree edges
    eu, ev, ew = g.edges()
    wmap = {(int(a), int(c)): float(x) for a, c, x in zip(eu, ev, ew)}
    LPz = np.zeros(g.n)
    pairs = [(min(v, int(g.parent[v])), max(v, int(g.parent[v]))) for v in range(g.n) if g.parent[v] >= 0]
    pairs += [(int(eu[i]), int(ev[i])) for i in ids]
    for a, c in pairs:
        f = wmap[(a, c)] * (z0[a] - z0[c])
        LPz[a] += f
        LPz[c] -= f
    assert np.abs(LPz - bb).max() <= 1e-9 * np.abs(bb).max()
    assert abs(z0.mean()) <= 1e-12 * np.abs(z0).max()
    assert len(hist) == it and hist[-1] == rel
