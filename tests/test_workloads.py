"""The seeded input generators: the same graphs whatever the number of worker processes (the bench generates with
a spawn pool, the tests mostly without), valid symmetric CSR, and a spanning tree of each graph."""
from __future__ import annotations

import numpy as np

from paper_2508_20403_gb300 import workloads as W


def _same(a, b):
    return (a.n == b.n and np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
            and np.array_equal(a.w, b.w) and np.array_equal(a.parent, b.parent))


def test_worker_count_does_not_change_the_graphs():
    assert _same(W.rmat_graph(12, seed=5, workers=0), W.rmat_graph(12, seed=5, workers=2))
    one = W.batch_graphs(6, workers=0, n_hi=5e3)
    two = W.batch_graphs(6, workers=2, n_hi=5e3)
    assert all(_same(a, b) for a, b in zip(one, two))


def _check_graph(g):
    rp, col, w = g.row_ptr, g.col, g.w
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(col)
    for u in range(g.n):
        row = col[rp[u]:rp[u + 1]]
        assert np.all(np.diff(row) > 0) and not np.any(row == u)
        for p in range(rp[u], rp[u + 1]):  # symmetric, bitwise equal weights
            v = col[p]
            q = rp[v] + np.searchsorted(col[rp[v]:rp[v + 1]], u)
            assert col[q] == u and w[q] == w[p]
    roots = np.flatnonzero(g.parent < 0)
    assert len(roots) == 1
    for v in range(g.n):  # parent links are edges
        if g.parent[v] >= 0:
            assert g.parent[v] in col[rp[v]:rp[v + 1]]


def test_generated_graphs_are_valid():
    for g in (W.grid_graph(15), W.mesh3d_graph(6), W.rmat_graph(9, seed=1),
              W.delaunay_graph(300, np.random.default_rng(3)), W.batch_member(2, n_hi=3e3), W.serve_member(1)):
        if g.n <= 5000:
            _check_graph(g)


def test_seeds_reproduce():
    assert _same(W.grid_graph(20), W.grid_graph(20))
    assert not np.array_equal(W.grid_graph(20, seed=1).w, W.grid_graph(20, seed=2).w)


def test_pack_into_preallocated_buffers():
    """The serving workers pack each batch straight into larger pinned staging arrays: the first N+1 / nnz / N
    entries must equal a fresh pack, and the disjoint union must keep every graph's CSR, weights and tree."""
    graphs = [W.grid_graph(7), W.rmat_graph(8, seed=3), W.grid_graph(4)]
    N, nnz = W.packed_sizes(graphs)
    ref = W.pack_graphs(graphs)
    assert (N, nnz) == (ref.row_ptr.size - 1, ref.col.size)
    bufs = (np.full(N + 17, -7, dtype=np.int64), np.full(nnz + 5, -7, dtype=np.int32),
            np.full(nnz + 5, np.nan), np.full(N + 3, -7, dtype=np.int32))
    pk = W.pack_graphs(graphs, out=bufs)
    for a, b in ((pk.row_ptr, ref.row_ptr), (pk.col, ref.col), (pk.w, ref.w), (pk.parent, ref.parent)):
        assert np.array_equal(a, b)
    assert np.shares_memory(pk.col, bufs[1]) and bufs[1][nnz] == -7  # written in place, nothing past the end
    for i, g in enumerate(graphs):
        v0, v1 = int(pk.vtx_ptr[i]), int(pk.vtx_ptr[i + 1])
        e0 = int(pk.row_ptr[v0])
        assert np.array_equal(pk.row_ptr[v0:v1 + 1] - e0, g.row_ptr)
        assert np.array_equal(pk.col[e0:e0 + 2 * g.m] - v0, g.col)
        par = pk.parent[v0:v1]
        assert np.array_equal(np.where(par < 0, -1, par - v0), g.parent)
