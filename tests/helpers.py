"""Small input builders shared by the tests (inputs only, no method arithmetic)."""
from __future__ import annotations

import json
import os

import numpy as np

from paper_2508_20403_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def graph_from_edges(n, edges, parent, name=""):
    edges = sorted((min(u, v), max(u, v), w) for (u, v, w) in edges)
    eu = np.array([e[0] for e in edges], dtype=np.int32)
    ev = np.array([e[1] for e in edges], dtype=np.int32)
    ew = np.array([e[2] for e in edges], dtype=np.float64)
    rp, col, w = W.csr_from_edges(n, eu, ev, ew)
    return W.Graph(n=n, row_ptr=rp, col=col, w=w, parent=np.asarray(parent, dtype=np.int32), name=name)


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def handtree():
    d = load_golden("handtree.json")
    return graph_from_edges(d["n"], [tuple(e) for e in d["edges"]], d["parent"], "handtree"), d


def random_spanning_parent(rng, n, eu, ev):
    """A random spanning tree (randomised BFS from a random root)."""
    adj = [[] for _ in range(n)]
    for a, b in zip(eu.tolist(), ev.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    root = int(rng.integers(n))
    parent = np.full(n, -2, dtype=np.int32)
    parent[root] = -1
    frontier = [root]
    while frontier:
        x = frontier.pop(int(rng.integers(len(frontier))))
        nb = adj[x][:]
        rng.shuffle(nb)
        for y in nb:
            if parent[y] == -2:
                parent[y] = x
                frontier.append(y)
    assert (parent != -2).all()
    return parent


def random_small_graph(rng, n_lo=2, n_hi=14, tree="random", weights="mixed"):
    """Random connected simple graph with a spanning tree."""
    n = int(rng.integers(n_lo, n_hi + 1))
    # random tree backbone to guarantee connectivity, plus random extra edges
    perm = rng.permutation(n)
    pairs = set()
    for i in range(1, n):
        a, b = int(perm[i]), int(perm[rng.integers(i)])
        pairs.add((min(a, b), max(a, b)))
    extra = int(rng.integers(0, n * (n - 1) // 2 + 1))
    for _ in range(extra):
        a, b = int(rng.integers(n)), int(rng.integers(n))
        if a != b:
            pairs.add((min(a, b), max(a, b)))
    pairs = sorted(pairs)
    eu = np.array([p[0] for p in pairs], dtype=np.int32)
    ev = np.array([p[1] for p in pairs], dtype=np.int32)
    m = len(pairs)
    kind = weights if weights != "mixed" else ["uniform", "ties", "wide"][int(rng.integers(3))]
    if kind == "ties":
        ew = rng.choice([1.0, 2.0, 3.0], size=m)
    elif kind == "wide":
        ew = np.power(10.0, rng.uniform(-3, 3, m))
    else:
        ew = 1.0 + 9.0 * rng.random(m)
    rp, col, w = W.csr_from_edges(n, eu, ev, ew)
    if tree == "max" or (tree == "mixed" and rng.random() < 0.5):
        parent = W.max_spanning_tree_parent(n, eu, ev, ew)
    else:
        parent = random_spanning_parent(rng, n, eu, ev)
    return W.Graph(n=n, row_ptr=rp, col=col, w=w, parent=parent, name=f"rand{n}")
