"""GPU spanning-tree generation (pdg_spanning_tree) against the oracle: bit-identical parent arrays."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_20403_gb300 import workloads as W
from tests.helpers import random_small_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2508_20403_gb300 import binding, build

    build.build()
    binding.load()
    return binding


def _gpu_tree(B, g, kind):
    return np.asarray(B.spanning_tree(g.n, g.row_ptr, g.col, g.w, kind=kind))


KINDS = [O.TREE_MAX_WEIGHT, O.TREE_FEGRASS]


@pytest.mark.parametrize("kind", KINDS)
def test_tree_workloads(B, kind):
    for g in (W.grid_graph(40), W.mesh3d_graph(20), W.rmat_graph(12, seed=9),
              W.delaunay_graph(3000, np.random.default_rng(2)), W.batch_member(3, n_hi=2e4)):
        assert np.array_equal(_gpu_tree(B, g, kind), O.spanning_tree(g, kind)), (g.name, kind)


@pytest.mark.parametrize("kind", KINDS)
def test_tree_random_small_with_ties(B, kind):
    rng = np.random.default_rng(77)
    for _ in range(60):
        g = random_small_graph(rng, n_lo=1, n_hi=40)
        assert np.array_equal(_gpu_tree(B, g, kind), O.spanning_tree(g, kind)), (g.name, kind)


def test_forest_and_disconnected(B):
    pk = W.pack_graphs([W.grid_graph(5), W.grid_graph(9), W.rmat_graph(8, seed=1)])
    g = W.Graph(n=int(pk.vtx_ptr[-1]), row_ptr=pk.row_ptr, col=pk.col, w=pk.w, parent=pk.parent, name="forest")
    p = _gpu_tree(B, g, O.TREE_MAX_WEIGHT)
    assert np.array_equal(p, O.spanning_tree(g, O.TREE_MAX_WEIGHT)) and (p < 0).sum() == 3
    with pytest.raises(B.PdgError) as e:
        _gpu_tree(B, g, O.TREE_FEGRASS)
    assert e.value.status == B.PDG_E_INVALID_ARG
    one = W.Graph(n=1, row_ptr=np.zeros(2, dtype=np.int64), col=np.zeros(0, dtype=np.int32),
                  w=np.zeros(0), parent=-np.ones(1, dtype=np.int32))
    assert _gpu_tree(B, one, O.TREE_MAX_WEIGHT).tolist() == [-1]


def test_device_buffers_and_recovery_on_the_tree(B):
    """Device CSR in, device parent out; the recovery on the generated tree matches the oracle's."""
    import torch

    g0 = W.mesh3d_graph(24, seed=8)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()
    out = torch.zeros(g0.n, dtype=torch.int32, device="cuda")
    B.spanning_tree(g0.n, t(g0.row_ptr, torch.int64), t(g0.col, torch.int32), t(g0.w, torch.float64),
                    kind=O.TREE_FEGRASS, parent_out=out)
    par = out.cpu().numpy()
    assert np.array_equal(par, O.spanning_tree(g0, O.TREE_FEGRASS))
    g = W.Graph(n=g0.n, row_ptr=g0.row_ptr, col=g0.col, w=g0.w, parent=par, name="mesh24-weff")
    _, oids, osc, _ = O.recover(g, 0.1, c=2)
    with B.Sparsifier.from_graph(g) as sp:
        st, ids, sc, _ = sp.recover(0.1, 2, capacity=g.m)
    assert np.array(ids).tolist() == oids.tolist() and np.array_equal(np.array(sc), osc)


def test_mesh128_full_size(B):
    """The full-size mesh: the maximum-weight tree equals the workload generator's (scipy) tree, and the
    effective-weight tree equals the oracle's."""
    g = W.mesh3d_graph(128)
    assert np.array_equal(_gpu_tree(B, g, O.TREE_MAX_WEIGHT), g.parent)
    assert np.array_equal(_gpu_tree(B, g, O.TREE_FEGRASS), O.spanning_tree(g, O.TREE_FEGRASS))
