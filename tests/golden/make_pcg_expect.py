"""Writes pcg_mesh64_expect.json: the oracle's PCG sparsifier-quality run (Sec. 5 measure, tol 1e-3) on the
3D mesh 64^3 with the oracle's own recovery at alpha = .02 (c = 2) as the extra edges.

Run with `python -m tests.golden.make_pcg_expect` from the repository root.  It calls the workload generators and
the CPU oracle only (never the CUDA library).  One oracle PCG run there takes tens of seconds and the iteration
count is checked against the range of counts under rounding-level perturbations of b (nine runs), so the GPU test
and the benchmark compare against these stored results.  Kept: the graph's sha256, the sha256 of the recovered ids
(int32, little endian), the right-hand side's seed, the oracle's iteration count and final relative residual, the
relative residual after each of the first 10 iterations, the count range under eight perturbations of relative
size 1e-13, max |z0| and z0 at 4096 evenly spaced vertices (z0 = the preconditioner applied to b')."""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "pcg_mesh64_expect.json")
SIDE, ALPHA, C, TOL, B_SEED = 64, 0.02, 2, 1e-3, 0
PERTURB, N_PERTURB, PERTURB_SEED = 1e-13, 8, 20250828
N_SAMPLE = 4096


def main():
    sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
    from oracle import oracle as O
    from oracle import pcg as PC
    from paper_2508_20403_gb300 import workloads as W
    from tests.golden.make_full_size_expect import graph_digest

    O.build()
    g = W.mesh3d_graph(SIDE)
    t0 = time.time()
    ids = np.ascontiguousarray(O.recover(g, ALPHA, c=C)[1], dtype="<i4")
    b = np.random.default_rng(B_SEED).standard_normal(g.n)
    it, rel, hist, z0 = PC.pcg_trace(g, ids, b, tol=TOL)
    rng = np.random.default_rng(PERTURB_SEED)
    its = [it] + [PC.pcg_quality(g, ids, b * (1 + PERTURB * rng.standard_normal(b.shape)), tol=TOL)[0]
                  for _ in range(N_PERTURB)]
    sample = np.linspace(0, g.n - 1, N_SAMPLE).astype(np.int64)
    rec = {"graph": f"mesh{SIDE}", "graph_sha256": graph_digest(g), "n": int(g.n), "m": int(g.m), "alpha": ALPHA,
           "c": C, "tol": TOL, "b_seed": B_SEED, "edges": int(ids.size),
           "ids_sha256": hashlib.sha256(ids.tobytes()).hexdigest(), "iterations": int(it), "relres": float(rel),
           "history": [float(x) for x in hist[:10]], "count_range": [int(min(its)), int(max(its))],
           "perturbation": PERTURB, "perturbations": N_PERTURB, "z0_max_abs": float(np.abs(z0).max()),
           "z0_sample_index": sample.tolist(), "z0_sample": [float(x) for x in z0[sample]],
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(f"mesh{SIDE}: {ids.size} edges, {it} iterations (range {min(its)}..{max(its)}), "
          f"{rec['oracle_seconds']} s")


if __name__ == "__main__":
    main()
