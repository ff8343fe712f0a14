"""The autotuner: graph classes, the cache, the search (CPU); one small tuning run on the GPU."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_20403_gb300 import autotune as AT
from paper_2508_20403_gb300 import workloads as W


def test_graph_class_buckets():
    assert AT.graph_class(2 ** 21, 3 * 2 ** 21, 6) == "n2^21-deg2^3-skew2^0-g2^0"
    assert AT.graph_class(1000, 16000, 2000, graphs=2000) == "n2^10-deg2^5-skew2^6-g2^11"
    g = W.grid_graph(20)
    assert AT.class_of(g).startswith("n2^9-deg2^2-")
    pk = W.pack_graphs([W.grid_graph(10), W.grid_graph(12)])
    assert AT.class_of(pk).endswith("-g2^1")


def test_cache_round_trip_and_options(tmp_path):
    path = str(tmp_path / "cache.json")
    assert AT.load_cache(path) == {}
    g = W.grid_graph(20)
    cache = {"GPU X|sm152": {AT.class_of(g): {"options": {"warp_tier_max": 16, "sort_tile_keys": 2048},
                                               "ms": 1.0}}}
    AT.save_cache(cache, path)
    assert AT.load_cache(path) == cache
    o = AT.options_for(g, cache_path=path, dev="GPU X|sm152", use_graph=1)
    assert (o.warp_tier_max, o.sort_tile_keys, o.use_graph) == (16, 2048, 1)
    d = AT.options_for(g, cache_path=path, dev="another GPU|sm1")  # no entry: the library defaults
    assert (d.warp_tier_max, d.sort_tile_keys, d.block_tier_max) == (32, 3072, 0)


def test_coordinate_descent_finds_the_separable_minimum():
    space = {"a": [0, 1, 2], "b": [5, 6], "c": [7, 8, 9]}
    cost = lambda s: abs(s["a"] - 2) + (s["b"] == 5) * 3 + abs(s["c"] - 8)
    best, t, tried = AT.coordinate_descent(cost, space)
    assert best == {"a": 2, "b": 6, "c": 8} and t == 0
    assert len(tried) == 1 + 2 + 1 + 2  # start + the other values of each knob


@pytest.mark.gpu
def test_tune_small_graph_is_exact(tmp_path):
    import torch

    from paper_2508_20403_gb300 import binding as B, build

    build.build()
    B.load()
    torch.cuda.init()
    g = W.rmat_graph(13, seed=77)
    space = {"warp_tier_max": [32, 8], "block_tier_max": [0, 96], "sort_tile_keys": [3072, 2048, 4096]}
    entry = AT.tune(g, 0.1, c=2, repeats=1, warmup=1, space=space)
    assert len(entry["tried"]) == 5 and entry["ms"] > 0
    path = str(tmp_path / "cache.json")
    AT.save_cache({AT.device_key(): {AT.class_of(g): entry}}, path)
    opt = AT.options_for(g, cache_path=path)
    for k, v in entry["options"].items():
        assert getattr(opt, k) == v
    _, oids, osc, _ = O.recover(g, 0.1, c=2)
    with B.Sparsifier.from_graph(g, options=opt) as sp:
        st, ids, sc, _ = sp.recover(0.1, 2, capacity=g.m)
    assert np.array(ids).tolist() == oids.tolist() and np.array_equal(np.array(sc), osc)


def test_committed_cache_is_valid():
    """The cache shipped with the package parses, and every entry holds settings the library accepts."""
    cache = AT.load_cache(AT.DEFAULT_CACHE)
    assert cache, "the package ships a tuned cache"
    for dev, classes in cache.items():
        assert "|sm" in dev
        for cls, entry in classes.items():
            assert cls.startswith("n2^") and "-g2^" in cls
            o = entry["options"]
            assert set(o) == set(AT.SPACE)
            assert 1 <= o["warp_tier_max"] <= 32
            assert 0 <= o["block_tier_max"] <= 896
            assert o["sort_tile_keys"] in (2048, 3072, 4096)
            assert entry["ms"] <= entry["default_ms"] * 1.0001  # never worse than the defaults it was timed against
