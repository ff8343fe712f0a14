"""Writes full_size_expect.json: the oracle's recovery of the full-size benchmark graphs, stored as digests.

Run with `python -m tests.golden.make_full_size_expect` from the repository root.  It calls the workload
generators and the CPU oracle only (never the CUDA library).  The oracle's greedy is quadratic in the size of
a subtask, and R-MAT scale 22 has one giant subtask at the hub, so its recoveries at alpha = .05 and .10 take
tens of minutes on one core; the GPU tests compare against these stored results instead of re-running them.
For each graph the file keeps the sha256 of its arrays (so a test can tell whether its generator produced the
same graph on another host) and, per alpha, the oracle's status, the number of ids, the sha256 of the ids
(int32, little endian) and of the scores (float64, little endian), and the first and last ids."""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "full_size_expect.json")


def graph_digest(g) -> str:
    h = hashlib.sha256()
    for a, dt in ((g.row_ptr, "<i8"), (g.col, "<i4"), (g.w, "<f8"), (g.parent, "<i4")):
        h.update(np.ascontiguousarray(a, dtype=dt).tobytes())
    return h.hexdigest()


def result_record(st, ids, scores) -> dict:
    ids = np.ascontiguousarray(ids, dtype="<i4")
    scores = np.ascontiguousarray(scores, dtype="<f8")
    return {"status": int(st), "count": int(ids.size), "ids_sha256": hashlib.sha256(ids.tobytes()).hexdigest(),
            "scores_sha256": hashlib.sha256(scores.tobytes()).hexdigest(), "head": ids[:8].tolist(),
            "tail": ids[-8:].tolist()}


def main():
    sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
    from oracle import oracle as O
    from paper_2508_20403_gb300 import workloads as W

    O.build()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    todo = [("rmat22", lambda: W.rmat_graph(22, workers=min(16, os.cpu_count() or 1)), (0.02, 0.05, 0.10)),
            ("mesh128", lambda: W.mesh3d_graph(128), (0.02, 0.05, 0.10))]
    names = sys.argv[1:] or [t[0] for t in todo]
    for name, make, alphas in todo:
        if name not in names:
            continue
        g = make()
        rec = {"graph_sha256": graph_digest(g), "n": int(g.n), "m": int(g.m), "c": 2, "alphas": {}}
        for alpha in alphas:
            t0 = time.time()
            st, ids, sc, _ = O.recover(g, alpha, c=2)
            rec["alphas"][repr(alpha)] = dict(result_record(st, ids, sc), oracle_seconds=round(time.time() - t0, 1))
            print(name, alpha, rec["alphas"][repr(alpha)]["count"], f"{time.time() - t0:.1f}s", flush=True)
            data[name] = rec
            with open(OUT, "w") as f:
                json.dump(data, f, indent=1)


if __name__ == "__main__":
    main()
