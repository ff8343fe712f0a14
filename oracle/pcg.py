"""Sparsifier quality by preconditioned conjugate gradients -- plain numpy/scipy ORACLE.

TEST INFRASTRUCTURE ONLY: the test-suite and the benchmark's CPU legs are the only callers; the product path never
imports this module.  Sec. 5 of the paper measures a sparsifier P = T + A (spanning tree plus recovered edges) by
the number of PCG iterations that solving L_G x = b takes with L_P as the preconditioner, to a relative residual of
1e-3.  Written out:

  b' = b - mean(b)            (L_G is singular: the right-hand side is taken in the range, the complement of 1)
  M(r) = the solution z of L_P z = r grounded at the tree root (z(root) = 0, the root's equation dropped; an exact
         sparse LU of the grounded L_P), then centred (z - mean(z))
  x = 0, r = b', z = M(r), p = z
  repeat: a = (r.z) / (p.L_G p); x += a p; r -= a L_G p; stop when ||r|| <= tol ||b'||;
          z = M(r); beta = (r.z)_new / (r.z)_old; p = z + beta p
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def laplacian_from_csr(n: int, row_ptr, col, w) -> sp.csr_matrix:
    A = sp.csr_matrix((np.asarray(w, dtype=np.float64), np.asarray(col), np.asarray(row_ptr)), shape=(n, n))
    return (sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A).tocsr()


def canonical_edges(n: int, row_ptr, col, w):
    """(u, v, w) of every undirected edge, u < v, in canonical id order (row-major over the CSR)."""
    eu, ev, ew = [], [], []
    for u in range(n):
        for p in range(int(row_ptr[u]), int(row_ptr[u + 1])):
            if col[p] > u:
                eu.append(u)
                ev.append(int(col[p]))
                ew.append(float(w[p]))
    return np.array(eu, dtype=np.int64), np.array(ev, dtype=np.int64), np.array(ew)


def sparsifier_laplacian(g, edge_ids) -> sp.csr_matrix:
    """L_P of the tree (g.parent) plus the canonical edges `edge_ids`."""
    eu, ev, ew = canonical_edges(g.n, g.row_ptr, g.col, g.w)
    rows, cols, vals = [], [], []
    wmap = {}
    for u, v, x in zip(eu, ev, ew):
        wmap[(int(u), int(v))] = x
    tree = []
    for v in range(g.n):
        p = int(g.parent[v])
        if p >= 0:
            a, b = min(p, v), max(p, v)
            tree.append((a, b, wmap[(a, b)]))
    extra = [(int(eu[i]), int(ev[i]), float(ew[i])) for i in edge_ids]
    for a, b, x in tree + extra:
        rows += [a, b, a, b]
        cols += [a, b, b, a]
        vals += [x, x, -x, -x]
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.n, g.n))


def pcg_quality(g, edge_ids, b, tol: float = 1e-3, max_iter: int = 1000):
    """Returns (iterations, final relative residual)."""
    it, rel, _, _ = pcg_trace(g, edge_ids, b, tol, max_iter)
    return it, rel


def pcg_trace(g, edge_ids, b, tol: float = 1e-3, max_iter: int = 1000):
    """Returns (iterations, final relative residual, the relative residual after each iteration, M(b'))."""
    n = g.n
    LG = laplacian_from_csr(n, g.row_ptr, g.col, g.w)
    LP = sparsifier_laplacian(g, edge_ids)
    root = int(np.flatnonzero(np.asarray(g.parent) < 0)[0])
    keep = np.flatnonzero(np.arange(n) != root)
    lu = spla.splu(LP[keep][:, keep].tocsc())

    def M(r):
        z = np.zeros(n)
        z[keep] = lu.solve(r[keep])
        return z - z.mean()

    bb = np.asarray(b, dtype=np.float64)
    bb = bb - bb.mean()
    nb = np.linalg.norm(bb)
    x = np.zeros(n)
    r = bb.copy()
    z = M(r)
    z0 = z.copy()
    p = z.copy()
    rz = r @ z
    hist = []
    for it in range(1, max_iter + 1):
        Ap = LG @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= tol:
            return it, rel, np.array(hist), z0
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return max_iter, np.linalg.norm(r) / nb, np.array(hist), z0
