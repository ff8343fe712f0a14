"""Seeded synthetic workloads for off-tree edge recovery.

This module only *generates inputs*: a weighted undirected graph in CSR form
and a spanning tree given as a parent array.  It holds none of the recovery
method's arithmetic (no resistance, LCA, similarity or budget logic), so both
the CPU oracle and the CUDA path may consume what it produces.

Shapes follow the paper's workload classes (Sec. 5, "Datasets"): uniform
finite-element meshes and census graphs (|E|/|V| of 2-3), skewed social
graphs (R-MAT stands in for com-Youtube), 2D triangulations (Delaunay stands
in for the NACA/M6/NLR meshes).  Unweighted graphs get weights drawn
uniformly from [1, 10] as in the paper.

The spanning tree is the maximum-weight spanning tree (Kruskal, weight
descending, ties broken by the smaller canonical edge id), rooted at the
vertex of maximum degree (ties to the smallest id), the root rule of the
effective-weight tree in Sec. 2.2.

Canonical undirected edge ids: edge {u, v} with u < v gets the rank of the
CSR entry (u, v) among all entries with row < col, in row-major order.
Generators draw weights in that order, so edge id i owns the i-th draw.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

SEED_BASE = 20250828


@dataclasses.dataclass
class Graph:
    """A weighted undirected graph in symmetric CSR plus a spanning tree."""

    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[2m], neighbours sorted ascending within a row
    w: np.ndarray  # float64[2m], symmetric
    parent: np.ndarray  # int32[n], -1 at the root
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1]) // 2

    @property
    def n_offtree(self) -> int:
        return self.m - self.n + 1

    def edges(self):
        """Canonical edge list (u < v) in edge-id order: (u, v, w)."""
        rows = np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_ptr))
        sel = rows < self.col
        return rows[sel], self.col[sel], self.w[sel]

    def nbytes(self) -> int:
        return self.row_ptr.nbytes + self.col.nbytes + self.w.nbytes + self.parent.nbytes


def _canonical(n: int, eu: np.ndarray, ev: np.ndarray):
    """Orient u < v, drop self loops and duplicates, sort by (u, v)."""
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    lo = np.minimum(eu, ev)
    hi = np.maximum(eu, ev)
    keep = lo != hi
    key = np.sort(lo[keep] * n + hi[keep])
    if key.shape[0]:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    return (key // n).astype(np.int32), (key % n).astype(np.int32)


def csr_from_edges(n: int, eu: np.ndarray, ev: np.ndarray, ew: np.ndarray):
    """Symmetric CSR from canonical edges (eu < ev, sorted by (eu, ev))."""
    m = eu.shape[0]
    rows = np.concatenate([eu, ev]).astype(np.int64)
    cols = np.concatenate([ev, eu]).astype(np.int64)
    ws = np.concatenate([ew, ew])
    order = np.argsort(rows * n + cols, kind="stable")
    cols = cols[order].astype(np.int32)
    ws = np.ascontiguousarray(ws[order], dtype=np.float64)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    assert row_ptr[-1] == 2 * m
    return row_ptr, cols, ws


def max_spanning_tree_parent(n: int, eu: np.ndarray, ev: np.ndarray, ew: np.ndarray) -> np.ndarray:
    """Kruskal maximum-weight spanning tree (ties -> smaller edge id), as a
    parent array rooted at the max-degree vertex (ties -> smaller id).

    Kruskal's order is made explicit by replacing each weight with its rank in
    (weight descending, id ascending); with distinct keys the minimum spanning
    tree over ranks is unique and equals Kruskal's tree for that order.
    """
    m = eu.shape[0]
    order = np.lexsort((np.arange(m), -ew))  # primary: -w, secondary: id
    rank = np.empty(m, dtype=np.float64)
    rank[order] = np.arange(1, m + 1, dtype=np.float64)
    a = sp.csr_matrix((rank, (eu, ev)), shape=(n, n))
    t = csg.minimum_spanning_tree(a).tocoo()
    if t.nnz != n - 1:
        raise ValueError("graph is not connected")
    deg = np.bincount(eu, minlength=n) + np.bincount(ev, minlength=n)
    root = int(np.argmax(deg))
    tu = t.row.astype(np.int32)
    tv = t.col.astype(np.int32)
    tsym = sp.csr_matrix((np.ones(2 * (n - 1)), (np.concatenate([tu, tv]), np.concatenate([tv, tu]))), shape=(n, n))
    _, pred = csg.breadth_first_order(tsym, root, directed=False, return_predecessors=True)
    parent = pred.astype(np.int32)
    parent[root] = -1
    if np.count_nonzero(parent < 0) != 1:
        raise ValueError("tree does not span the graph")
    return parent


def _largest_component(n: int, eu: np.ndarray, ev: np.ndarray):
    a = sp.csr_matrix((np.ones(eu.shape[0], dtype=np.int8), (eu, ev)), shape=(n, n))
    ncomp, lab = csg.connected_components(a, directed=False)
    if ncomp == 1:
        return n, eu, ev
    big = np.argmax(np.bincount(lab))
    keep = lab == big
    newid = np.full(n, -1, dtype=np.int64)
    newid[keep] = np.arange(np.count_nonzero(keep))
    sel = keep[eu]  # both endpoints share a component
    return int(np.count_nonzero(keep)), newid[eu[sel]].astype(np.int32), newid[ev[sel]].astype(np.int32)


def build_graph(n: int, eu: np.ndarray, ev: np.ndarray, ew: np.ndarray, name: str = "") -> Graph:
    row_ptr, col, w = csr_from_edges(n, eu, ev, ew)
    parent = max_spanning_tree_parent(n, eu, ev, ew)
    return Graph(n=n, row_ptr=row_ptr, col=col, w=w, parent=parent, name=name)


# ----------------------------------------------------------------------------
# weight distributions (drawn in canonical edge-id order)

def weights_uniform_1_10(rng: np.random.Generator, m: int) -> np.ndarray:
    return 1.0 + 9.0 * rng.random(m)


def weights_loguniform(rng: np.random.Generator, m: int, lo: float = 1e-3, hi: float = 1e3) -> np.ndarray:
    return np.power(10.0, rng.uniform(math.log10(lo), math.log10(hi), m))


def weights_uniform_0_1(rng: np.random.Generator, m: int) -> np.ndarray:
    return 1.0 - rng.random(m)  # (0, 1]


# ----------------------------------------------------------------------------
# graph families

def grid2d_edges(sx: int, sy: int):
    idx = np.arange(sx * sy, dtype=np.int64).reshape(sx, sy)
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return _canonical(sx * sy, a, b)


def mesh3d_edges(s: int):
    idx = np.arange(s ** 3, dtype=np.int64).reshape(s, s, s)
    a = np.concatenate([idx[:-1].ravel(), idx[:, :-1].ravel(), idx[:, :, :-1].ravel()])
    b = np.concatenate([idx[1:].ravel(), idx[:, 1:].ravel(), idx[:, :, 1:].ravel()])
    return _canonical(s ** 3, a, b)


def _rmat_chunk(args):
    """One chunk of R-MAT samples from its own seeded stream (float32 draws:
    the quadrant thresholds need far fewer than 24 bits)."""
    seed, idx, cnt, scale, a, b, c = args
    rng = np.random.default_rng([seed, idx])
    ab, abc = a + b, a + b + c
    su = np.zeros(cnt, dtype=np.int32)
    sv = np.zeros(cnt, dtype=np.int32)
    for lvl in range(scale):
        r = rng.random(cnt, dtype=np.float32)
        su |= (r >= ab).astype(np.int32) << lvl
        sv |= (((r >= a) & (r < ab)) | (r >= abc)).astype(np.int32) << lvl
    return su, sv


def rmat_edges(rng: np.random.Generator, scale: int, edge_factor: int = 16,
               a: float = 0.57, b: float = 0.19, c: float = 0.19, permute: bool = True,
               chunk: int = 1 << 22, workers: int = 0):
    """R-MAT edge samples, symmetrised and deduplicated; vertex labels are
    randomly permuted (Graph500 practice) so ids carry no degree order.
    Samples come in chunks with seeds derived from `rng`, optionally drawn in a
    spawn pool; the result does not depend on the number of workers."""
    nv = 1 << scale
    ne = edge_factor * nv
    seed = int(rng.integers(0, 1 << 62))
    jobs = [(seed, i, min(chunk, ne - s0), scale, a, b, c) for i, s0 in enumerate(range(0, ne, chunk))]
    if workers and workers > 1 and len(jobs) > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_rmat_chunk, jobs)
    else:
        parts = [_rmat_chunk(j) for j in jobs]
    src = np.concatenate([p[0] for p in parts])
    dst = np.concatenate([p[1] for p in parts])
    del parts
    if permute:
        perm = rng.permutation(nv).astype(np.int32)
        src = perm[src]
        dst = perm[dst]
    eu, ev = _canonical(nv, src, dst)
    return nv, eu, ev


def rgg_edges(rng: np.random.Generator, n: int, mean_degree: float):
    from scipy.spatial import cKDTree

    pts = rng.random((n, 2))
    r = math.sqrt(mean_degree / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    return _canonical(n, pairs[:, 0], pairs[:, 1])


def delaunay_edges(rng: np.random.Generator, n: int):
    from scipy.spatial import Delaunay

    pts = rng.random((n, 2))
    tri = Delaunay(pts).simplices.astype(np.int64)
    a = np.concatenate([tri[:, 0], tri[:, 1], tri[:, 2]])
    b = np.concatenate([tri[:, 1], tri[:, 2], tri[:, 0]])
    return _canonical(n, a, b)


def _finish(n, eu, ev, weight_fn, rng, name, lcc=True) -> Graph:
    if lcc:
        n, eu, ev = _largest_component(n, eu, ev)
        eu, ev = _canonical(n, eu, ev)
    ew = weight_fn(rng, eu.shape[0])
    return build_graph(n, eu, ev, ew, name=name)


# ----------------------------------------------------------------------------
# the five workload configurations

def grid_graph(sx: int = 100, sy: Optional[int] = None, seed: int = SEED_BASE + 0) -> Graph:
    """2D 4-connected grid, weights i.i.d. U[1, 10]."""
    sy = sx if sy is None else sy
    rng = np.random.default_rng(seed)
    eu, ev = grid2d_edges(sx, sy)
    return _finish(sx * sy, eu, ev, weights_uniform_1_10, rng, f"grid{sx}x{sy}", lcc=False)


def mesh3d_graph(s: int = 128, seed: int = SEED_BASE + 1) -> Graph:
    """3D 7-point mesh s^3, weights log-uniform over [1e-3, 1e3]."""
    rng = np.random.default_rng(seed)
    eu, ev = mesh3d_edges(s)
    return _finish(s ** 3, eu, ev, weights_loguniform, rng, f"mesh{s}^3", lcc=False)


def rmat_graph(scale: int = 22, edge_factor: int = 16, seed: int = SEED_BASE + 2, workers: int = 0) -> Graph:
    """Skewed R-MAT (a=.57, b=c=.19), symmetrised, deduplicated, largest
    connected component, weights U(0, 1]."""
    rng = np.random.default_rng(seed)
    nv, eu, ev = rmat_edges(rng, scale, edge_factor, workers=workers)
    return _finish(nv, eu, ev, weights_uniform_0_1, rng, f"rmat-s{scale}-ef{edge_factor}")


def rgg_graph(n: int, mean_degree: float, rng: np.random.Generator, name: str = "") -> Graph:
    eu, ev = rgg_edges(rng, n, mean_degree)
    return _finish(n, eu, ev, weights_uniform_1_10, rng, name or f"rgg{n}")


def delaunay_graph(n: int, rng: np.random.Generator, name: str = "") -> Graph:
    eu, ev = delaunay_edges(rng, n)
    return _finish(n, eu, ev, weights_uniform_1_10, rng, name or f"delaunay{n}", lcc=False)


def batch_member(index: int, seed: int = SEED_BASE + 3, n_lo: float = 1e3, n_hi: float = 2e5,
                 side_lo: int = 30, side_hi: int = 300) -> Graph:
    """Member `index` of the batching mix: 70% random geometric graphs in the
    unit square (n log-uniform in [n_lo, n_hi], radius for mean degree U[6,20],
    largest component kept), 30% square 2D grids with side U[side_lo, side_hi];
    weights U[1, 10]."""
    rng = np.random.default_rng([seed, index])
    if rng.random() < 0.7:
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        deg = rng.uniform(6.0, 20.0)
        return rgg_graph(n, deg, rng, name=f"rgg{n}-d{deg:.1f}")
    side = int(rng.integers(side_lo, side_hi + 1))
    eu, ev = grid2d_edges(side, side)
    return _finish(side * side, eu, ev, weights_uniform_1_10, rng, f"grid{side}x{side}", lcc=False)


def serve_member(index: int, seed: int = SEED_BASE + 4) -> Graph:
    """Member of the serving mix: half from the batching mix, half Delaunay
    triangulations of n uniform points, n log-uniform in [1e4, 1e6]."""
    rng = np.random.default_rng([seed, index])
    if rng.random() < 0.5:
        return batch_member(int(rng.integers(0, 1 << 30)), seed=seed + 1000)
    n = int(round(math.exp(rng.uniform(math.log(1e4), math.log(1e6)))))
    return delaunay_graph(n, rng)


def batch_graphs(count: int = 2000, seed: int = SEED_BASE + 3, workers: int = 0, **kw) -> List[Graph]:
    """The batching mix; `workers` > 0 generates members in a spawn pool."""
    if workers and workers > 1 and count > 8:
        import multiprocessing as mp
        import functools

        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            return pool.map(functools.partial(batch_member, seed=seed, **kw), range(count), chunksize=4)
    return [batch_member(i, seed=seed, **kw) for i in range(count)]


# ----------------------------------------------------------------------------
# packing several graphs into one disjoint union (a forest of spanning trees)

@dataclasses.dataclass
class PackedGraphs:
    """Disjoint union of graphs with global vertex ids.

    vtx_ptr[g] is graph g's first vertex; edge_ptr[g] its first canonical
    edge id (edge ids are row-major over the packed CSR, so graph g's local
    edge id is the global id minus edge_ptr[g]).  parent holds global ids and
    -1 at every graph's root.
    """

    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    parent: np.ndarray
    vtx_ptr: np.ndarray  # int64[G+1]
    edge_ptr: np.ndarray  # int64[G+1]

    @property
    def num_graphs(self) -> int:
        return self.vtx_ptr.shape[0] - 1

    @property
    def n(self) -> int:
        return int(self.vtx_ptr[-1])


def packed_sizes(graphs: Sequence[Graph]):
    """(vertices, CSR entries) of the disjoint union of `graphs`."""
    return sum(g.n for g in graphs), sum(2 * g.m for g in graphs)


def pack_graphs(graphs: Sequence[Graph], out=None) -> PackedGraphs:
    """The disjoint union of `graphs`.  `out` may hold preallocated arrays (row_ptr int64[N+1], col int32[nnz],
    w float64[nnz], parent int32[N], at least that long; e.g. views of pinned host memory) to write into."""
    G = len(graphs)
    vtx_ptr = np.zeros(G + 1, dtype=np.int64)
    edge_ptr = np.zeros(G + 1, dtype=np.int64)
    nnz_ptr = np.zeros(G + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        vtx_ptr[i + 1] = vtx_ptr[i] + g.n
        edge_ptr[i + 1] = edge_ptr[i] + g.m
        nnz_ptr[i + 1] = nnz_ptr[i] + 2 * g.m
    N = int(vtx_ptr[-1])
    nnz = int(nnz_ptr[-1])
    if N >= 2 ** 31 - 1 or nnz >= 2 ** 62:
        raise ValueError("packed batch too large for int32 vertex ids")
    if out is None:
        row_ptr = np.empty(N + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int32)
        w = np.empty(nnz, dtype=np.float64)
        parent = np.empty(N, dtype=np.int32)
    else:
        row_ptr, col, w, parent = out[0][:N + 1], out[1][:nnz], out[2][:nnz], out[3][:N]
    for i, g in enumerate(graphs):
        v0, v1 = int(vtx_ptr[i]), int(vtx_ptr[i + 1])
        e0, e1 = int(nnz_ptr[i]), int(nnz_ptr[i + 1])
        np.add(g.row_ptr[:-1], e0, out=row_ptr[v0:v1], casting="unsafe")
        np.add(g.col, v0, out=col[e0:e1], casting="unsafe")
        w[e0:e1] = g.w
        pv = parent[v0:v1]
        np.add(g.parent, v0, out=pv, casting="unsafe")
        pv[np.asarray(g.parent) < 0] = -1
    row_ptr[N] = nnz
    return PackedGraphs(row_ptr=row_ptr, col=col, w=w, parent=parent, vtx_ptr=vtx_ptr, edge_ptr=edge_ptr)


CONFIGS = {
    "grid100": dict(desc="2D 4-connected grid 100x100, w~U[1,10], alpha=2%, beta cap c=2", alphas=(0.02,)),
    "mesh128": dict(desc="3D 7-point mesh 128^3, w log-uniform [1e-3,1e3], alpha in {2,5,10}%, c=2",
                    alphas=(0.02, 0.05, 0.10)),
    "rmat22": dict(desc="R-MAT scale 22 (a=.57,b=c=.19, ef 16), symmetrised, dedup, LCC, w~U(0,1], "
                        "alpha in {2,5,10}%, c=2", alphas=(0.02, 0.05, 0.10)),
}


def config_graph(name: str, **kw) -> Graph:
    if name == "grid100":
        return grid_graph(100, **kw)
    if name == "mesh128":
        return mesh3d_graph(128, **kw)
    if name == "rmat22":
        return rmat_graph(22, **kw)
    raise KeyError(name)
