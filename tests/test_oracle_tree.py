"""Pins of the oracle's spanning-tree generation (Sec. 2.2 feGRASS first step, Eq. weff) against independent
statements: scipy's minimum spanning tree over edge ranks, brute force over all spanning trees of tiny graphs,
and BFS distances from scipy."""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from oracle import oracle as O
from paper_2508_20403_gb300 import workloads as W
from tests.helpers import random_small_graph


def _edges(g):
    eu, ev, ew = [], [], []
    for u in range(g.n):
        for p in range(g.row_ptr[u], g.row_ptr[u + 1]):
            if g.col[p] > u:
                eu.append(u)
                ev.append(int(g.col[p]))
                ew.append(float(g.w[p]))
    return np.array(eu, dtype=np.int32), np.array(ev, dtype=np.int32), np.array(ew)


def _deg(g):
    return np.diff(g.row_ptr)


def _root_of(g, comp_vertices):
    deg = _deg(g)
    return min(comp_vertices, key=lambda v: (-deg[v], v))


def _weff_keys(g, eu, ev, ew):
    """Eq. weff written out: (w * log(max degree)) / (d(u) + d(v)), d = BFS hops from the max-degree vertex."""
    deg = _deg(g)
    root = _root_of(g, range(g.n))
    a = sp.csr_matrix((np.ones(len(g.col)), g.col, g.row_ptr), shape=(g.n, g.n))
    d = csg.shortest_path(a, unweighted=True, indices=root)
    keys = []
    for u, v, w in zip(eu, ev, ew):
        num = w * math.log(float(max(deg[u], deg[v])))
        keys.append(num / float(int(d[u]) + int(d[v])))
    return np.array(keys)


def _rooted_parent(g, n, tree_edges):
    """Parent array of a forest: each component rooted at its max-degree vertex (ties: smaller id)."""
    adj = [[] for _ in range(n)]
    for u, v in tree_edges:
        adj[u].append(v)
        adj[v].append(u)
    parent = -np.ones(n, dtype=np.int32)
    seen = np.zeros(n, dtype=bool)
    for s in range(n):
        if seen[s]:
            continue
        comp, stack = [], [s]
        seen[s] = True
        while stack:
            x = stack.pop()
            comp.append(x)
            for y in adj[x]:
                if not seen[y]:
                    seen[y] = True
                    stack.append(y)
        root = _root_of(g, comp)
        done = {root}
        frontier = [root]
        while frontier:
            nxt = []
            for x in frontier:
                for y in adj[x]:
                    if y not in done:
                        done.add(y)
                        parent[y] = x
                        nxt.append(y)
            frontier = nxt
    return parent


def _brute_force_tree(g, keys):
    """Among all spanning trees, the one with the smallest sum of ranks in (key desc, id asc): with distinct
    ranks that is the unique maximum spanning tree of the strict order."""
    eu, ev, _ = _edges(g)
    m = len(eu)
    order = sorted(range(m), key=lambda e: (-keys[e], e))
    rank = np.empty(m, dtype=np.int64)
    rank[order] = np.arange(m)
    best, best_sum = None, None
    for sub in itertools.combinations(range(m), g.n - 1):
        up = list(range(g.n))

        def find(x):
            while up[x] != x:
                x = up[x]
            return x

        ok = True
        for e in sub:
            a, b = find(int(eu[e])), find(int(ev[e]))
            if a == b:
                ok = False
                break
            up[a] = b
        if not ok:
            continue
        s = int(rank[list(sub)].sum())
        if best_sum is None or s < best_sum:
            best, best_sum = sub, s
    return _rooted_parent(g, g.n, [(int(eu[e]), int(ev[e])) for e in best])


@pytest.mark.parametrize("make", [lambda: W.grid_graph(25), lambda: W.mesh3d_graph(12), lambda: W.rmat_graph(10, seed=3),
                                  lambda: W.delaunay_graph(400, np.random.default_rng(5))])
def test_max_weight_tree_equals_scipy_kruskal(make):
    """The workload generator builds its tree with scipy's minimum spanning tree over the (w desc, id asc) ranks
    and roots it at the max-degree vertex: an independent statement of the same tree."""
    g = make()
    eu, ev, ew = _edges(g)
    assert np.array_equal(O.spanning_tree(g, O.TREE_MAX_WEIGHT), W.max_spanning_tree_parent(g.n, eu, ev, ew))


def test_max_weight_tree_with_ties_equals_scipy_kruskal():
    rng = np.random.default_rng(11)
    for _ in range(30):
        g = random_small_graph(rng, n_lo=2, n_hi=60, weights="ties")
        eu, ev, ew = _edges(g)
        assert np.array_equal(O.spanning_tree(g), W.max_spanning_tree_parent(g.n, eu, ev, ew))


@pytest.mark.parametrize("seed", range(3))
def test_trees_brute_force_tiny(seed):
    rng = np.random.default_rng(200 + seed)
    for _ in range(25):
        g = random_small_graph(rng, n_lo=2, n_hi=7)
        if len(_edges(g)[0]) > 12:
            continue
        eu, ev, ew = _edges(g)
        assert np.array_equal(O.spanning_tree(g, O.TREE_MAX_WEIGHT), _brute_force_tree(g, ew))
        assert np.array_equal(O.spanning_tree(g, O.TREE_FEGRASS), _brute_force_tree(g, _weff_keys(g, eu, ev, ew)))


def test_fegrass_tree_equals_kruskal_on_weff_keys():
    """On larger graphs: the scipy tree over the Eq. weff keys (computed here with scipy BFS and math.log)."""
    for g in (W.grid_graph(30), W.mesh3d_graph(10), W.rmat_graph(10, seed=3)):
        eu, ev, ew = _edges(g)
        keys = _weff_keys(g, eu, ev, ew)
        assert np.array_equal(O.spanning_tree(g, O.TREE_FEGRASS), W.max_spanning_tree_parent(g.n, eu, ev, keys))


def test_tree_invariants_and_disconnected():
    g = W.grid_graph(20)
    for kind in (O.TREE_MAX_WEIGHT, O.TREE_FEGRASS):
        p = O.spanning_tree(g, kind)
        assert (p < 0).sum() == 1 and p[_root_of(g, range(g.n))] == -1
        deg = _deg(g)
        for v in range(g.n):  # every link is an edge of G
            if p[v] >= 0:
                assert p[v] in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
    # two disjoint grids: a forest with one root per component; the effective weight needs a connected graph
    pk = W.pack_graphs([W.grid_graph(5), W.grid_graph(6)])
    two = W.Graph(n=int(pk.vtx_ptr[-1]), row_ptr=pk.row_ptr, col=pk.col, w=pk.w, parent=pk.parent, name="2grids")
    p = O.spanning_tree(two, O.TREE_MAX_WEIGHT)
    assert (p < 0).sum() == 2
    with pytest.raises(ValueError):
        O.spanning_tree(two, O.TREE_FEGRASS)


@pytest.mark.parametrize("n", [5, 6, 7, 8, 11, 12])
def test_fegrass_cycle_closed_form(n):
    """Cycle C_n with unit weights: every degree is 2 (L = log 2), the root is vertex 0 (ties: smaller id) and
    d(i) = min(i, n - i), so W_eff(i, i+1) = log 2 / (d(i) + d(i+1)) is smallest on the edges farthest from 0; the
    tree drops the one of those with the largest canonical id (ties go to the smaller id) and hangs the two arcs
    of the cycle from vertex 0."""
    eu = np.array([min(i, (i + 1) % n) for i in range(n)], dtype=np.int32)
    ev = np.array([max(i, (i + 1) % n) for i in range(n)], dtype=np.int32)
    rp, col, w = W.csr_from_edges(n, eu, ev, np.ones(n))
    g = W.Graph(n=n, row_ptr=rp, col=col, w=w, parent=-np.ones(n, dtype=np.int32), name=f"cycle{n}")
    d = [min(i, n - i) for i in range(n)]
    # canonical ids: edges sorted by (u, v)
    edges = sorted(zip(eu.tolist(), ev.tolist()))
    sums = [d[a] + d[b] for a, b in edges]
    far = max(sums)
    dropped = max(i for i, s in enumerate(sums) if s == far)
    keep = [e for i, e in enumerate(edges) if i != dropped]
    want = _rooted_parent(g, n, keep)
    assert want[0] == -1
    assert np.array_equal(O.spanning_tree(g, O.TREE_FEGRASS), want)
