"""pdg_edge_endpoints_noalloc: the endpoint mapping for callers that cannot
allocate device memory (only their own pool, or no allocator stalls allowed).
It must return exactly what pdg_edge_endpoints returns, on consecutive calls
that reuse the library's fixed scratch array.  This file is collected last
so that a failure here leaves every other test already run."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2508_20403_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2508_20403_gb300 import binding, build

    build.build()
    binding.load()
    return binding


def _device(a, dt):
    import torch

    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()


def test_noalloc_endpoints_match_handle_path_twice(B):
    import torch

    for g in (W.grid_graph(60, seed=71), W.mesh3d_graph(20, seed=72)):
        with B.Sparsifier.from_graph(g) as sp:
            st, rec_ids, _, k = sp.recover(0.1, 2)
            rec_ids = np.array(rec_ids)
            rp, col = _device(g.row_ptr, torch.int64), _device(g.col, torch.int32)
            # two calls in a row with different ids: the shared scratch must not leak state
            for ids_np in (rec_ids, np.arange(g.m, dtype=np.int32)[::-7].copy()):
                ids = _device(ids_np, torch.int32)
                want_u, want_v = sp.endpoints(ids)
                u = torch.full_like(ids, -5)
                v = torch.full_like(ids, -5)
                st = B.edge_endpoints_noalloc(g.n, rp, col, ids, u, v)
                torch.cuda.synchronize()
                assert st == B.PDG_OK
                assert torch.equal(u, want_u) and torch.equal(v, want_v)
                eu, ev, _ = g.edges()
                assert u.cpu().numpy().tolist() == eu[ids_np].tolist()
                assert v.cpu().numpy().tolist() == ev[ids_np].tolist()


def test_noalloc_rejects_out_of_range(B):
    import torch

    g = W.grid_graph(10, seed=73)
    rp, col = _device(g.row_ptr, torch.int64), _device(g.col, torch.int32)
    ids = _device(np.array([0, g.m], dtype=np.int32), torch.int32)
    u = torch.zeros_like(ids)
    v = torch.zeros_like(ids)
    assert B.edge_endpoints_noalloc(g.n, rp, col, ids, u, v) == B.PDG_E_INVALID_ARG
    assert B.edge_endpoints_noalloc(B.NOALLOC_MAX_N + 1, rp, col, ids, u, v) == B.PDG_E_INVALID_ARG
    # a valid call afterwards still succeeds (the error word is cleared per call)
    ids = _device(np.array([0, g.m - 1], dtype=np.int32), torch.int32)
    assert B.edge_endpoints_noalloc(g.n, rp, col, ids, u, v) == B.PDG_OK


def test_noalloc_at_the_size_limit(B):
    """n = PDG_NOALLOC_MAX_N exactly (the 128^3 mesh has 2^21 vertices): every scan block is used and the last
    row prefix lands in the slot next to the block sums.  A strided set of ids that includes the last id m - 1,
    twice in a row, must equal the handle path."""
    import torch

    g = W.mesh3d_graph(128)
    assert g.n == B.NOALLOC_MAX_N
    rp, col = _device(g.row_ptr, torch.int64), _device(g.col, torch.int32)
    ids_np = np.unique(np.concatenate([np.arange(0, g.m, 9973), [g.m - 1, g.m - 2, 1]])).astype(np.int32)
    eu, ev, _ = g.edges()
    with B.Sparsifier.from_graph(g, device=True) as sp:
        for ids_host in (ids_np, ids_np[::-1].copy()):
            ids = _device(ids_host, torch.int32)
            want_u, want_v = sp.endpoints(ids)
            u = torch.full_like(ids, -5)
            v = torch.full_like(ids, -5)
            assert B.edge_endpoints_noalloc(g.n, rp, col, ids, u, v) == B.PDG_OK
            torch.cuda.synchronize()
            assert torch.equal(u, want_u) and torch.equal(v, want_v)
            assert u.cpu().numpy().tolist() == eu[ids_host].tolist()
            assert v.cpu().numpy().tolist() == ev[ids_host].tolist()
