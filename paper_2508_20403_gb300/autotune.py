"""Autotuner of the recovery's launch shape (step A5's tier bounds and the radix-sort tile size).

Every setting gives the same recovered edges (each tier runs the exact sequential greedy; the sort is a stable
sort whatever its tile size); only the time changes.  The tuner times recoveries on the GPU for a few settings of

  warp_tier_max   subtasks of 2..T_w candidates get one warp,
  block_tier_max  subtasks of T_w+1..T_b candidates get one block (0: none; larger ones go cooperative),
  sort_tile_keys  keys per scatter tile of the one-sweep radix sort,

by coordinate descent from the library defaults, checks that every setting returned the default's edges, and
caches the winner in a JSON file keyed by the GPU (name and SM count) and a coarse graph class (size, mean degree,
degree skew, graphs per batch).  `options_for` reads the cache; a graph class with no entry gets the defaults.

    python -m paper_2508_20403_gb300.autotune --workload mesh128 --workload batch2000 [--cache PATH]
"""
from __future__ import annotations

import argparse
import json
import math
import os
from typing import Callable, Dict, List, Optional

import numpy as np

from . import binding as B

SPACE: Dict[str, List[int]] = {
    "warp_tier_max": [32, 16],
    "block_tier_max": [0, 64, 160, 320, 640],
    "sort_tile_keys": [3072, 2048, 4096],
}
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def _bucket(x: float) -> int:
    return int(round(math.log2(max(x, 1.0))))


def graph_class(n: int, m: int, max_degree: int, graphs: int = 1) -> str:
    """Coarse class: log2 buckets of the vertex count, the mean degree, the max/mean degree skew and the number
    of graphs packed together."""
    mean_deg = 2.0 * m / max(n, 1)
    return (f"n2^{_bucket(n)}-deg2^{_bucket(mean_deg)}-skew2^{_bucket(max_degree / max(mean_deg, 1e-9))}"
            f"-g2^{_bucket(graphs)}")


def class_of(obj) -> str:
    """graph_class of a workloads.Graph or a workloads.PackedGraphs."""
    deg = np.diff(np.asarray(obj.row_ptr))
    graphs = len(obj.vtx_ptr) - 1 if hasattr(obj, "vtx_ptr") else 1
    n = int(deg.shape[0])
    return graph_class(n, int(obj.row_ptr[-1]) // 2, int(deg.max()) if n else 0, graphs)


def device_key() -> str:
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}"


def load_cache(path: Optional[str] = None) -> dict:
    path = path or os.environ.get("PDG_AUTOTUNE_CACHE", DEFAULT_CACHE)
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: Optional[str] = None) -> None:
    path = path or os.environ.get("PDG_AUTOTUNE_CACHE", DEFAULT_CACHE)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(cache: dict, dev: str, cls: str) -> Optional[dict]:
    return cache.get(dev, {}).get(cls)


def options_for(obj, cache_path: Optional[str] = None, dev: Optional[str] = None, **overrides) -> B.Options:
    """Library options for a Graph / PackedGraphs: the cached tuned settings of its class on this GPU (if any),
    then `overrides`."""
    entry = lookup(load_cache(cache_path), dev or device_key(), class_of(obj))
    settings = dict(entry["options"]) if entry else {}
    settings.update(overrides)
    return B.default_options(**settings)


def coordinate_descent(run: Callable[[dict], float], space: Dict[str, List[int]] = SPACE) -> tuple:
    """Minimise run(settings) one knob at a time, starting from each knob's first value.  Returns (best settings,
    best time, every (settings, time) tried)."""
    best = {k: v[0] for k, v in space.items()}
    best_t = run(dict(best))
    tried = [(dict(best), best_t)]
    for k, values in space.items():
        for v in values[1:]:
            cand = dict(best)
            cand[k] = v
            t = run(cand)
            tried.append((cand, t))
            if t < best_t:
                best, best_t = cand, t
    return best, best_t, tried


def tune(obj, alpha: float, c: int = 2, repeats: int = 5, warmup: int = 2, space: Dict[str, List[int]] = SPACE,
         stream=None) -> dict:
    """Time recoveries of `obj` (Graph or PackedGraphs, copied to the device) for the settings coordinate descent
    visits; every setting must return the default's edges.  Returns the cache entry."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = stream or torch.cuda.current_stream(dev)
    packed = hasattr(obj, "vtx_ptr")
    reference = {}

    def run(settings: dict) -> float:
        opt = B.default_options(use_graph=1, **settings)
        if packed:
            h = B.BatchSparsifier.from_packed(obj, device=True, options=opt, stream=stream)
            alphas = np.full(h.num_graphs, alpha)
            op = h.out_ptr_for(alphas)
            out = torch.zeros(max(int(op[-1]), 1), dtype=torch.int32, device=dev)
            call = lambda: h.recover_batch(alphas, c=c, out_ptr=op, out_ids=out, out_scores=None)
        else:
            h = B.Sparsifier.from_graph(obj, device=True, options=opt, stream=stream)
            k = max(1, min(int(math.floor(alpha * obj.n)), obj.n_offtree))
            out = torch.zeros(k, dtype=torch.int32, device=dev)
            call = lambda: h.recover(alpha, c, out_ids=out)
        try:
            for _ in range(warmup):
                call()
            times = []
            for _ in range(repeats):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ids = out.cpu().numpy()
        finally:
            h.close()
        if "ids" not in reference:
            reference["ids"] = ids
        elif not np.array_equal(ids, reference["ids"]):
            raise RuntimeError(f"autotune: settings {settings} changed the recovered edges")
        return float(np.median(times))

    best, best_t, tried = coordinate_descent(run, space)
    return {"options": best, "ms": best_t, "default_ms": tried[0][1], "alpha": alpha, "c": c,
            "tried": [{"options": s, "ms": t} for s, t in tried]}


def _workload(name: str):
    from . import workloads as W

    if name == "mesh128":
        return W.mesh3d_graph(128), 0.10
    if name == "rmat22":
        return W.rmat_graph(22, workers=8), 0.02
    if name.startswith("batch"):
        return W.pack_graphs(W.batch_graphs(int(name[5:]), workers=8)), 0.05
    raise ValueError(name)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", action="append", required=True, help="mesh128, rmat22 or batchN")
    ap.add_argument("--cache", default=None)
    ap.add_argument("--c", type=int, default=2)
    ap.add_argument("--repeats", type=int, default=5)
    args = ap.parse_args(argv)
    from . import build

    build.build()
    B.load()
    cache = load_cache(args.cache)
    dev = device_key()
    for name in args.workload:
        obj, alpha = _workload(name)
        entry = tune(obj, alpha, c=args.c, repeats=args.repeats)
        entry["workload"] = name
        cache.setdefault(dev, {})[class_of(obj)] = entry
        save_cache(cache, args.cache)
        print(json.dumps({"workload": name, "class": class_of(obj), "options": entry["options"],
                          "ms": entry["ms"], "default_ms": entry["default_ms"]}), flush=True)


if __name__ == "__main__":
    main()
