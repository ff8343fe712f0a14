"""Continuous-batching server: admission logic (CPU) and results that are the
same alone and in the mix (GPU)."""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_2508_20403_gb300 import serve as S
from paper_2508_20403_gb300 import workloads as W


def _pool(count=12, seed=5):
    return [W.batch_member(i, seed=seed, n_lo=300, n_hi=4000, side_lo=8, side_hi=50) for i in range(count)]


def test_admission_respects_memory_and_order():
    pool = _pool(6)
    srv = S.Server(mem_budget_bytes=10 ** 12, slots=1)
    for i, g in enumerate(pool):
        srv.queue.append(S.Request(graph=g, alpha=0.05, rid=i))
    need = [S.device_bytes_estimate(g) for g in pool]
    srv.mem_free = need[0] + need[1] + need[2] // 2  # room for exactly two
    batch, mem = srv._take_batch()
    assert [r.rid for r in batch] == [0, 1] and mem == need[0] + need[1]
    assert srv.mem_free == need[2] // 2
    batch, mem = srv._take_batch()  # the head no longer fits: nothing is skipped ahead of it
    assert batch == [] and mem == 0


def test_admission_groups_by_beta_cap():
    pool = _pool(3)
    srv = S.Server(mem_budget_bytes=10 ** 12, slots=1)
    srv.queue.extend([S.Request(graph=pool[0], alpha=0.1, c=2, rid=0), S.Request(graph=pool[1], alpha=0.1, c=1, rid=1),
                      S.Request(graph=pool[2], alpha=0.1, c=2, rid=2)])
    batch, _ = srv._take_batch()
    assert [r.rid for r in batch] == [0]


def test_poisson_arrivals_rate():
    t = S.poisson_arrivals(200.0, 30.0, np.random.default_rng(1))
    assert abs(len(t) / 30.0 - 200.0) < 15 and np.all(np.diff(t) > 0)


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix():
    from oracle import oracle as O
    from paper_2508_20403_gb300 import binding as B, build

    build.build()
    pool = _pool(12, seed=9)
    # a small budget forces requests to wait for memory; three slots overlap batches
    budget = 3 * max(S.device_bytes_estimate(g) for g in pool)
    srv = S.Server(mem_budget_bytes=budget, slots=3).start()
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(60):
        g = pool[int(rng.integers(len(pool)))]
        reqs.append(srv.submit(g, float(rng.choice([0.02, 0.05, 0.10]))))
        if i % 7 == 0:
            time.sleep(0.002)
    for r in reqs:
        assert r.done.wait(120)
    srv.stop()
    assert not srv.errors, srv.errors
    assert max(srv.batch_sizes) > 1  # requests were batched together
    for r in reqs:
        ost, oids, osc, _ = O.recover(r.graph, r.alpha, c=2)
        assert np.array_equal(r.ids, oids)
        assert np.array_equal(r.scores, osc)
        with B.Sparsifier.from_graph(r.graph) as sp:  # alone, through the single-graph entry point
            st, ids, sc, k = sp.recover(r.alpha, 2)
        assert np.array_equal(np.asarray(ids), r.ids)
