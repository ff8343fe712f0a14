"""The paper's multi-threaded CPU method (baseline_cpu/, OpenMP) against the oracle: the same recovered ids, in
the same order, with the same scores, for any thread count, with and without inner parallelism (the cutoff set
low so that the blocked path with judge-before-parallel runs on every subtask)."""
from __future__ import annotations

import numpy as np
import pytest

from baseline_cpu import omp as P
from oracle import oracle as O
from paper_2508_20403_gb300 import workloads as W
from tests.helpers import random_small_graph


def _same(g, alpha, c=2, mode=0, k_override=-1, **kw):
    st, ids, sc = P.recover(g, alpha, c=c, score_mode=mode, k_override=k_override, **kw)
    ost, oids, osc, _ = O.recover(g, alpha, c=c, score_mode=mode, k_override=k_override)
    assert ids.tolist() == oids.tolist(), (g.name, alpha, c, mode, kw)
    assert np.array_equal(sc, osc)
    assert (st == P.UNDER_BUDGET) == (ost == O.UNDER_BUDGET)


@pytest.mark.parametrize("threads,cutoff", [(1, -1), (4, -1), (4, 1), (3, 2)])
def test_random_small_graphs(threads, cutoff):
    rng = np.random.default_rng(77)
    for _ in range(30):
        g = random_small_graph(rng, n_lo=2, n_hi=60, tree="mixed")
        c = int(rng.integers(0, 4))
        mode = int(rng.integers(0, 2))
        k = int(rng.integers(0, g.m + 1))
        _same(g, 0.0, c=c, mode=mode, k_override=k, threads=threads, cutoff=cutoff)


@pytest.mark.parametrize("threads,cutoff", [(4, -1), (4, 50)])
def test_mesh_rmat_grid(threads, cutoff):
    _same(W.mesh3d_graph(20, seed=5), 0.10, threads=threads, cutoff=cutoff)
    _same(W.rmat_graph(12, seed=9), 0.05, threads=threads, cutoff=cutoff)
    _same(W.grid_graph(40), 0.02, c=1, threads=threads, cutoff=cutoff)


def test_under_budget_and_tiny():
    g = W.grid_graph(6)
    _same(g, 0.9, threads=2)
    _same(W.grid_graph(1, 2), 0.5, threads=2)
