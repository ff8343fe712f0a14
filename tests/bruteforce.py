"""Brute-force restatement of the recovery step for tiny graphs.

Independent of both the C oracle and the CUDA library: tree paths and BFS
neighbourhoods come from networkx, sums are exact `fractions.Fraction`s, and
the greedy checks every candidate against *every* earlier recovered edge (no
use of Lemma "share LCA"), exactly as Def. "Similar edge (Strict)" reads.
"""
from __future__ import annotations

import math
from fractions import Fraction

import networkx as nx
import numpy as np


def canonical_edges(g):
    """[(id, u, v, w)] with u < v in row-major CSR order."""
    out = []
    nid = 0
    for u in range(g.n):
        for p in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
            v = int(g.col[p])
            if u < v:
                out.append((nid, u, v, float(g.w[p])))
                nid += 1
    return out


def tree_graph(g):
    t = nx.Graph()
    t.add_nodes_from(range(g.n))
    for v in range(g.n):
        p = int(g.parent[v])
        if p >= 0:
            t.add_edge(v, p)
    return t


def depths(g):
    root = int(np.flatnonzero(g.parent < 0)[0])
    return nx.single_source_shortest_path_length(tree_graph(g), root)


def tree_weight(g, v):
    p = int(g.parent[v])
    for q in range(int(g.row_ptr[v]), int(g.row_ptr[v + 1])):
        if int(g.col[q]) == p:
            return float(g.w[q])
    raise ValueError("tree edge missing from graph")


def offtree(g):
    par = g.parent
    return [(i, u, v, w) for (i, u, v, w) in canonical_edges(g) if not (par[v] == u or par[u] == v)]


def edge_facts(g, c, score_mode="stretch"):
    """id -> dict(u, v, w, lca, R, score, beta) computed from explicit tree paths."""
    T = tree_graph(g)
    dep = depths(g)
    facts = {}
    for (i, u, v, w) in offtree(g):
        path = nx.shortest_path(T, u, v)
        lca = min(path, key=lambda x: dep[x])
        exact = Fraction(0)
        for a, b in zip(path[:-1], path[1:]):
            child = a if dep[a] > dep[b] else b
            exact += Fraction(1.0 / tree_weight(g, child))  # W_re = fl(1/w), summed exactly
        R = float(exact)  # correctly rounded
        score = R if score_mode == "resistance" else w * R
        hu, hv = dep[u] - dep[lca], dep[v] - dep[lca]
        facts[i] = dict(u=u, v=v, w=w, lca=lca, R=R, exact=exact, score=score, beta=min(hu, hv, c), hu=hu, hv=hv)
    return facts


def order(facts):
    return sorted(facts, key=lambda i: (-facts[i]["score"], i))


def neighbourhood(T, x, b):
    return set(nx.single_source_shortest_path_length(T, x, cutoff=b))


def strictly_similar(T, e, a):
    """Is e strictly similar to the recovered edge a (using a's beta*)?"""
    Su = neighbourhood(T, a["u"], a["beta"])
    Sv = neighbourhood(T, a["v"], a["beta"])
    u, v = e["u"], e["v"]
    return (u in Su and v in Sv) or (u in Sv and v in Su)


def greedy(g, k, c, score_mode="stretch", sequence=None):
    """Sequential strict-similarity greedy over `sequence` (default: the
    score order); checks each edge against all earlier recovered edges."""
    T = tree_graph(g)
    facts = edge_facts(g, c, score_mode)
    seq = order(facts) if sequence is None else list(sequence)
    acc = []
    for i in seq:
        if len(acc) >= k:
            break
        if any(strictly_similar(T, facts[i], facts[a]) for a in acc):
            continue
        acc.append(i)
    return acc, facts


def budget(n, alpha):
    return int(math.floor(alpha * n))


def laplacian(n, edges):
    L = np.zeros((n, n))
    for (u, v, w) in edges:
        L[u, u] += w
        L[v, v] += w
        L[u, v] -= w
        L[v, u] -= w
    return L


def generalized_eigs(LG, LP):
    """Nonzero generalised eigenvalues of (LG, LP) for connected graphs:
    restrict to the complement of the all-ones vector."""
    n = LG.shape[0]
    Q, _ = np.linalg.qr(np.concatenate([np.ones((n, 1)), np.eye(n)[:, : n - 1]], axis=1))
    B = Q[:, 1:]
    A = B.T @ LG @ B
    P = B.T @ LP @ B
    ev = np.linalg.eigvals(np.linalg.solve(P, A)).real
    return np.sort(ev)
