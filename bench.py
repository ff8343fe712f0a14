"""Benchmark of GB300 off-tree edge recovery (pdGRASS recovery step).

Headline: off-tree edges/s of one recovery (steps A1-A7) on the 3D 7-point
mesh 128^3 (2,097,152 vertices, 6,242,304 edges, 4,145,153 off-tree edges),
weights log-uniform over [1e-3, 1e3], maximum-weight spanning tree,
alpha = 0.10, beta cap c = 2, graph resident in HBM after sparsify_init.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the single-graph path
is replicas only; value = edges of all ranks / max rank time, weak scaling).
`--impl reference` times the CPU oracle on the host cores instead (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
METRIC = "Off-tree edges/s in recovery"
# The oracle's bounded sample of the headline workload: the same mesh 128^3 inputs and c, with the budget cut to
# k = floor(0.02 n) -- exactly the first 41,943 edges of the alpha = 0.10 output, since the greedy decides every
# edge from earlier edges only.  The oracle still scores, orders and groups all off-tree edges; only the greedy
# stops earlier (a full alpha = 0.10 run takes 30-40 s on one core, too long for K timed steps).
ORACLE_SAMPLE_ALPHA = 0.02


def host_cpu() -> dict:
    """Model name and logical core count of the host (read-only)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    import platform

    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class _NvmlSampler:
    """SM clock and clock-event reasons read through NVML every ~1 ms on a
    background thread (read-only queries; nothing is set)."""

    # nvmlClocksEventReasons bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, torch_index: int):
        import ctypes
        import threading

        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        ok = False
        try:
            import torch

            prop = torch.cuda.get_device_properties(torch_index)
            bus = getattr(prop, "pci_bus_id", None)
            dom = getattr(prop, "pci_domain_id", 0)
            pdev = getattr(prop, "pci_device_id", 0)
            if bus is not None:
                pci = f"{dom:08x}:{bus:02x}:{pdev:02x}.0".encode()
                ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci, ctypes.byref(self.dev)) == 0
        except Exception:
            ok = False
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(torch_index), ctypes.byref(self.dev)) != 0:
            raise RuntimeError("no NVML handle")
        mx = ctypes.c_uint(0)
        self.lib.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx))
        self.max_mhz = float(mx.value)
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples = []
        self.stop = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        ct = self.ct
        clk = ct.c_uint(0)
        rs = ct.c_ulonglong(0)
        while not self.stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.dev, 1, ct.byref(clk)) == 0 and \
                    self.reasons_fn(self.dev, ct.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(0.001)

    def start(self):
        self.thread.start()

    def finish(self):
        self.stop.set()
        self.thread.join(timeout=5)
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass


class ClockSampler:
    """Clocks during the timed region: NVML every ~1 ms, else nvidia-smi
    every 100 ms (read-only queries)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.nvml = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"pdgrass_clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.nvml = _NvmlSampler(self.index)
            self.nvml.start()
            return self
        except Exception:
            self.nvml = None
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.nvml is not None:
            self.nvml.finish()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.nvml is not None:
            sm = [c for c, _ in self.nvml.samples]
            if not sm:
                return {"sm_mhz": None, "sm_max_mhz": self.nvml.max_mhz, "reasons": ["no samples"], "source": "nvml"}
            reasons = sorted({nm for _, r in self.nvml.samples for nm, bit in _NvmlSampler.BITS.items() if r & bit})
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.nvml.max_mhz, "reasons": reasons,
                    "samples": len(sm), "source": "nvml"}
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, p[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi"}


# ---------------------------------------------------------------- algorithmic bytes

def step_bytes(n, nnz, E, G, R, k):
    """Compulsory DRAM bytes of each step of the GPU pipeline (each stream
    once, gathers at element size), per recovery."""
    A = 2 * (n - G)  # Euler-tour arcs
    return {
        # stream the canonical edge list (u, v: 4 B, w: 8 B), gather parent, write r(v) and the off-tree SoA
        "classify": 16 * (nnz // 2) + 4 * n + 8 * n + 20 * E,
        # two passes over the tour (arc 4 B + r gather 8 B); write P (16 B) and the range-minimum key (8 B),
        # read parent (4 B); the range-minimum build reads the keys (8 B) and writes the masks (4 B)
        "tree": 2 * 12 * A + 28 * n + 12 * n,
        # read (u, v, w) 16 B, gather P(u), P(v), P(LCA) 48 B, write key + lca 12 B
        "score": 76 * E,
        # two histogram passes + one compaction pass over the keys, write candidates (idx, key, val)
        "select": 24 * E + 16 * R,
        # 8 score digits + 3 LCA digits, each: read key+val 12 B, write 12 B
        "sort": 11 * 24 * R,
        # records (~44 B written + read), tier lists
        "accept": 100 * R,
        "budget": 8 * R + 12 * k,
    }


# the longest single launch of a recovery: step A3 is one kernel, k_score
DOMINANT_KERNEL = "k_score"
SCORE_BYTES_PER_EDGE = 76  # read u, v (8 B), w (8 B); gather P(u), P(v), P(lca) (48 B); write key, lca (12 B)


def path_bytes(n, m, E, k):
    """Algorithmic bytes of one recovery (compulsory traffic of the method:
    read the CSR and parent, write and read depth and D, one write and one
    read of a 24-byte sort record per off-tree edge, the output)."""
    return 8 * (n + 1) + 24 * m + 4 * n + 40 * n + 48 * E + 4 * k


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, if
    the summary was taken on the kernel source as it is now (else None)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    scaled = "dram bytes per launch (scaled to mesh 128^3 by off-tree edges, x 1.21459)"
    src = os.path.join(ROOT, "paper_2508_20403_gb300", "csrc", "pdg_score.cu")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if line.startswith("- ") and ": " in line:
                    key, val = line[2:].split(": ", 1)
                    fields[key.strip()] = val.strip().strip("`")
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
        if fields.get("kernel source sha256") != digest:
            return None
        return float(fields[scaled] if scaled in fields else fields["dram bytes per launch"])
    except Exception:
        return None


def sources_digest() -> str:
    """sha256 over the CUDA sources of the library (file names and contents, sorted)."""
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2508_20403_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def ncu_recovery_traffic(workload: str):
    """DRAM bytes (read + write) of all kernels of one recovery, from the committed ncu summary, if it was
    taken on the CUDA sources as they are now (else None)."""
    path = os.path.join(ROOT, "profiles", f"recovery_traffic_{workload}.md")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if line.startswith("- ") and ": " in line:
                    key, val = line[2:].split(": ", 1)
                    fields[key.strip()] = val.strip().strip("`")
        if fields.get("sources sha256") != sources_digest():
            return None
        return float(fields["dram bytes per recovery"])
    except Exception:
        return None


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time (all ranks call this; one all-reduce)."""
    if world <= 1:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, units_per_rank: int, t_max_ms: float) -> float:
    """Replicas: every rank recovers its own copy of the workload, so the job processes world x the units in the
    slowest rank's time (weak scaling)."""
    return world * units_per_rank / (t_max_ms / 1e3)


def time_recoveries(sp, alpha, c, steps, warmup, flush, stream, out_ids, out_sc):
    """CUDA-event times (ms) of `steps` recoveries after `warmup` untimed ones; L2 is flushed before each."""
    import torch

    for _ in range(warmup):
        sp.recover(alpha, c, out_ids=out_ids, out_scores=out_sc)
    torch.cuda.synchronize()
    times, launches = [], []
    for i in range(steps):
        flush.fill_(i & 0xff)  # evict L2 between steps (outside the timed interval)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sp.recover(alpha, c, out_ids=out_ids, out_scores=out_sc)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        launches.append(sp.last_stats()["launches"])
    return times, launches


def step_list(avg, bytes_, peak):
    """Per-step rows {step, ms, model bytes, GB/s, fraction of the peak}, in pipeline order."""
    rows = []
    for nm in ("classify", "tree", "score", "select", "sort", "accept", "budget"):
        gbs = bytes_[nm] / (avg[nm] / 1e3) / 1e9 if avg[nm] > 0 else None
        rows.append({"step": nm, "ms": round(avg[nm], 4), "model_bytes": int(bytes_[nm]),
                     "gbs": None if gbs is None else round(gbs, 1),
                     "frac": None if gbs is None else round(gbs / peak, 4)})
    return rows


def config_leg(args, g, dev, B, AT, torch, flush, stream, alphas, steps, label):
    """Extra configurations: min and median ms per recovery, edges/s and the path roofline fraction."""
    peak, _ = measured_peaks()
    opt = AT.options_for(g, use_graph=1)
    rows = []
    with B.Sparsifier.from_graph(g, device=True, options=opt, stream=stream) as sp:
        info = sp.info()
        for alpha in alphas:
            k = int(math.floor(alpha * g.n))
            out_ids = torch.zeros(max(k, 1), dtype=torch.int32, device=dev)
            out_sc = torch.zeros(max(k, 1), dtype=torch.float64, device=dev)
            times, _ = time_recoveries(sp, alpha, args.c, steps, 3, flush, stream, out_ids, out_sc)
            st = sp.last_stats()
            b_alg = path_bytes(info["n"], info["m"], info["n_offtree"], k)
            t_med = float(np.median(times))
            rows.append({"workload": label, "n": info["n"], "m": info["m"], "n_offtree": info["n_offtree"],
                         "alpha": alpha, "c": args.c, "k": k, "steps": steps, "min_ms": float(np.min(times)),
                         "median_ms": t_med, "edges_per_s": info["n_offtree"] / (t_med / 1e3),
                         "path_frac": b_alg / (t_med / 1e3) / 1e9 / peak, "algorithmic_bytes": b_alg,
                         "candidates": st["candidates"], "max_subtask": st["max_subtask"],
                         "launch_shape": {kk: getattr(opt, kk) for kk in AT.SPACE}})
    return rows


def run_ours(args, rank, world, local_rank, batch_graphs=None, serve_graphs=None, extra_graphs=None):
    import torch

    from paper_2508_20403_gb300 import binding as B, build as BLD, workloads as W

    torch.cuda.set_device(local_rank)
    if rank == 0:
        BLD.build()
    if world > 1:
        torch.distributed.barrier()
    B.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    t0 = time.time()
    g = W.mesh3d_graph(MESH_SIDE)
    log(f"[rank {rank}] generated {g.name} n={g.n} m={g.m} E_off={g.n_offtree} in {time.time() - t0:.1f}s")
    k = int(math.floor(args.alpha * g.n))
    # timed handle: the recovery is captured once and replayed as a CUDA graph
    # launch shape (tier bounds, sort tiles) from the autotuner's cache for this GPU and graph class
    from paper_2508_20403_gb300 import autotune as AT

    opt = AT.options_for(g, use_graph=0 if args.no_graph else 1)
    tuned = {kk: getattr(opt, kk) for kk in AT.SPACE}
    dev_inputs = [torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
                  for a, dt in ((g.row_ptr, torch.int64), (g.col, torch.int32), (g.w, torch.float64),
                                (g.parent, torch.int32))]
    # sparsify_init from device-resident inputs (upload of the graph excluded): validation, the resident
    # canonical edge list and the tree layout
    init_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t_init = time.perf_counter()
        sp = B.Sparsifier(g.n, *dev_inputs, options=opt, stream=stream)
        torch.cuda.synchronize()
        init_ms.append((time.perf_counter() - t_init) * 1e3)
        sp.close()
    sp = B.Sparsifier(g.n, *dev_inputs, options=opt, stream=stream)
    info = sp.info()
    out_ids = torch.zeros(max(k, 1), dtype=torch.int32, device=dev)
    out_sc = torch.zeros(max(k, 1), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        times, launches = time_recoveries(sp, args.alpha, args.c, args.steps, args.warmup, flush, stream, out_ids,
                                          out_sc)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    stats = sp.last_stats()
    sp.close()
    # per-step breakdown: a second handle, launched step by step with CUDA events
    step_ms = []
    sp = B.Sparsifier(g.n, *dev_inputs, options=AT.options_for(g, profile=1), stream=stream)
    last = None
    for i in range(args.warmup + args.steps):
        flush.fill_(i & 0xff)
        last = sp.recover(args.alpha, args.c, out_ids=out_ids, out_scores=out_sc)
        if i >= args.warmup:
            step_ms.append(sp.last_timings())
    sp.close()
    gpu_ids = last[1].cpu().numpy() if hasattr(last[1], "cpu") else np.asarray(last[1])
    mean_ms = float(np.mean(times))
    t_max = max_over_ranks(mean_ms, world, dev)
    value = whole_job_value(world, info["n_offtree"], t_max)
    names = ["classify", "tree", "score", "select", "sort", "accept", "budget"]
    avg = {nm: float(np.mean([s_[nm] for s_ in step_ms])) for nm in names}
    nnz = 2 * info["m"]
    bytes_ = step_bytes(info["n"], nnz, info["n_offtree"], info["num_graphs"], stats["candidates"], k)
    peak, peak_kind = measured_peaks()
    b_alg = path_bytes(info["n"], info["m"], info["n_offtree"], k)
    achieved = b_alg / (t_max / 1e3) / 1e9
    steps_rows = step_list(avg, bytes_, peak)
    top = max(steps_rows, key=lambda r: r["ms"])
    dom_bytes = SCORE_BYTES_PER_EDGE * info["n_offtree"]
    dom_ms = avg["score"]  # the events around step A3 bracket exactly one launch of k_score
    result = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(args, world),
        "min_ms": float(np.min(times)), "median_ms": float(np.median(times)),
        "init_ms": {"median": float(np.median(init_ms)), "runs": [round(x, 3) for x in init_ms],
                    "includes": "sparsify_init from device-resident CSR and parent: validation, canonical edge "
                                "list, tree layout (Euler tour, preorder labels)"},
        "tree_max_depth": info["max_depth"],
        "step_ms": {nm: round(avg[nm], 4) for nm in names},
        "recovery_stats": stats,
        "launch_shape": dict(tuned, source="autotune cache" if AT.lookup(AT.load_cache(), AT.device_key(),
                                                                          AT.class_of(g)) else "defaults"),
        # The roofline of the whole recovery (steps A1-A7 in one CUDA-graph replay) against the method's
        # compulsory traffic; the per-step rows and the longest single kernel explain it.
        "roofline": {"bound": "hbm", "kernel": "recovery A1-A7 (one CUDA-graph replay)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_recovery_traffic("mesh128_a010"), "peak_source": peak_kind,
                     "algorithmic_bytes": b_alg, "duration_ms": t_max,
                     "steps": steps_rows, "top_step": top["step"],
                     "longest_kernel": {"kernel": DOMINANT_KERNEL, "algorithmic_bytes": dom_bytes,
                                        "duration_ms": dom_ms,
                                        "achieved": dom_bytes / (dom_ms / 1e3) / 1e9,
                                        "frac": dom_bytes / (dom_ms / 1e3) / 1e9 / peak,
                                        "traffic": ncu_traffic(DOMINANT_KERNEL, "mesh120_a010")}},
        "gpu_launches": int(np.sum(launches)),
        "gpu_launches_per_step": int(np.mean(launches)),
    }
    if rank == 0 and not args.no_configs:
        t0 = time.time()
        rows = config_leg(args, g, dev, B, AT, torch, flush, stream, (0.02, 0.05), min(args.steps, 10),
                          WORKLOAD)
        rows += config_leg(args, W.grid_graph(100), dev, B, AT, torch, flush, stream, (0.02,), min(args.steps, 10),
                           "grid100 (2D grid 100x100, w U[1,10], max-weight spanning tree)")
        if extra_graphs is not None and "rmat22" in extra_graphs:
            rows += config_leg(args, extra_graphs["rmat22"], dev, B, AT, torch, flush, stream, (0.02, 0.05, 0.10),
                               min(args.steps, 10),
                               "rmat22 (R-MAT scale 22, a=.57 b=c=.19, ef 16, LCC, w U(0,1], max-weight tree)")
        result["configs"] = rows
        log(f"[rank {rank}] config leg {time.time() - t0:.1f}s")
    del flush
    if rank == 0 and not args.no_e2e:
        result["e2e"] = e2e_leg(args, g, dev, B, torch)
    if rank == 0 and not args.no_tree:
        result["tree_build"] = tree_leg(args, g, dev, B, torch)
    if rank == 0 and not args.no_pcg:
        result["pcg_quality"] = pcg_leg(args, B)
    if batch_graphs is not None:
        t0 = time.time()
        result["batch"] = batch_leg(args, batch_graphs, dev, B, torch)
        log(f"[rank {rank}] batch leg {time.time() - t0:.1f}s")
    if serve_graphs is not None:
        t0 = time.time()
        result["serve"] = serve_leg(args, serve_graphs, dev, torch)
        log(f"[rank {rank}] serve leg {time.time() - t0:.1f}s")
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_leg(args, g)
        result["cpu_parallel"] = cpu_parallel_leg(args, g, gpu_ids)
    result["clocks"] = clk.summary()
    return result


def batch_leg(args, graphs, dev, B, torch):
    """Config 4: 2,000 graphs of the batching mix.  Batched = ONE
    recover_offtree_batch over the packed CSR (CUDA-graph replay); per-graph =
    the same graphs each resident in its own handle, one recover_offtree each
    (plain launches).  Outputs must be identical."""
    from paper_2508_20403_gb300 import workloads as W

    stream = torch.cuda.current_stream(dev)
    pk = W.pack_graphs(graphs)
    G = len(graphs)
    alphas = np.full(G, args.batch_alpha)
    e_off = int(sum(g.n_offtree for g in graphs))
    from paper_2508_20403_gb300 import autotune as AT

    opt = AT.options_for(pk, use_graph=1)  # the autotuner's launch shape for this class, if cached
    bs = B.BatchSparsifier.from_packed(pk, device=True, options=opt, stream=stream)
    op = bs.out_ptr_for(alphas)
    out = torch.zeros(max(int(op[-1]), 1), dtype=torch.int32, device=dev)
    outs = torch.zeros(max(int(op[-1]), 1), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        bs.recover_batch(alphas, c=args.c, out_ptr=op, out_ids=out, out_scores=outs)
    torch.cuda.synchronize()
    tb = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, _, _, _, counts, gst = bs.recover_batch(alphas, c=args.c, out_ptr=op, out_ids=out, out_scores=outs)
        e1.record(stream)
        e1.synchronize()
        tb.append(e0.elapsed_time(e1))
    bstats = bs.last_stats()
    batch_ids = out.cpu().numpy()
    bs.close()
    # per-graph plain launches on resident handles
    handles = [B.Sparsifier.from_graph(g, device=True, stream=stream) for g in graphs]
    kk = [int(math.floor(args.batch_alpha * g.n)) for g in graphs]
    outs_pg = [torch.zeros(max(min(k, g.n_offtree), 1), dtype=torch.int32, device=dev) for k, g in zip(kk, graphs)]
    for sp, o in zip(handles, outs_pg):
        sp.recover(args.batch_alpha, args.c, out_ids=o)
    torch.cuda.synchronize()
    tp = []
    for _ in range(max(1, min(args.steps, 3))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [sp.recover(args.batch_alpha, args.c, out_ids=o) for sp, o in zip(handles, outs_pg)]
        e1.record(stream)
        e1.synchronize()
        tp.append(e0.elapsed_time(e1))
    identical = all(
        np.array_equal(batch_ids[op[i]:op[i] + counts[i]], outs_pg[i][:res[i][3]].cpu().numpy()) and
        counts[i] == res[i][3] for i in range(G))
    for sp in handles:
        sp.close()
    mb, mp = float(np.mean(tb)), float(np.mean(tp))
    return {"graphs": G, "n": int(pk.n), "m": int(sum(g.m for g in graphs)), "n_offtree": e_off,
            "alpha": args.batch_alpha, "c": args.c, "identical_output": bool(identical),
            "launch_shape": {k: getattr(opt, k) for k in AT.SPACE}, "graph_class": AT.class_of(pk),
            "batched": {"ms": mb, "graphs_per_s": G / (mb / 1e3), "edges_per_s": e_off / (mb / 1e3),
                        "launch": "one recover_offtree_batch (CUDA graph replay)", "stats": bstats},
            "per_graph": {"ms": mp, "graphs_per_s": G / (mp / 1e3), "edges_per_s": e_off / (mp / 1e3),
                          "launch": f"{G} x recover_offtree, graphs resident, plain launches"},
            "batched_over_per_graph": mp / mb}


def serve_pool(args, workers):
    """Config 5's graph pool: half from the batching mix, half Delaunay
    triangulations with n log-uniform in [1e4, 1e6] (requests draw from it)."""
    import functools
    import multiprocessing as mp

    from paper_2508_20403_gb300 import workloads as W

    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        return pool.map(functools.partial(W.serve_member, seed=W.SEED_BASE + 4), range(args.serve_pool),
                        chunksize=1)


def serve_point(args, pool, dev, rate, seconds, seed):
    """One Poisson stream at `rate` requests/s for `seconds` into a fresh continuous-batching server; latency =
    completion - arrival."""
    from paper_2508_20403_gb300 import serve as S

    from paper_2508_20403_gb300 import workloads as W

    biggest = sorted(pool, key=lambda g: -g.m)[:16]  # staging for a batch of the 16 largest graphs of the pool
    srv = S.Server(mem_budget_bytes=args.serve_mem_gb << 30, slots=args.serve_slots, device=dev.index,
                   staging_hint=W.packed_sizes(biggest)).start()
    # warm the library (first-call set-up) outside the measured stream
    S.run_stream(srv, pool[:4], rate=50.0, duration=0.2, seed=1)
    srv.completed.clear()
    srv.batch_sizes.clear()
    srv.max_inflight = 0
    t0 = time.perf_counter()
    reqs = S.run_stream(srv, pool, rate=rate, duration=seconds, seed=seed)
    wall = time.perf_counter() - t0
    srv.stop()
    out = S.summarize(reqs, wall)
    out.update({"rate_req_s": rate, "seconds": seconds, "pool_graphs": len(pool), "slots": args.serve_slots,
                "mem_budget_gb": args.serve_mem_gb, "batches": len(srv.batch_sizes),
                "mean_batch": float(np.mean(srv.batch_sizes)) if srv.batch_sizes else 0.0,
                "max_batch": int(max(srv.batch_sizes)) if srv.batch_sizes else 0,
                "max_batches_in_flight": srv.max_inflight, "errors": len(srv.errors),
                "alphas": [0.02, 0.05, 0.10], "c": args.c})
    return out


def serve_leg(args, pool, dev, torch):
    """Config 5: Poisson arrivals into the continuous-batching server, at the configured rate (200 requests/s for
    60 s by default) and at a rate above what one request at a time can serve (--serve-high-rate), where the
    queue builds up and requests are admitted into shared batches while others run."""
    out = serve_point(args, pool, dev, args.serve_rate, args.serve_seconds, seed=20250833)
    if args.serve_high_rate > 0:
        out["high_rate"] = serve_point(args, pool, dev, args.serve_high_rate, args.serve_high_seconds, seed=20250834)
    return out


def e2e_leg(args, g, dev, B, torch):
    """Same metric through the public API from pinned HOST buffers: upload +
    validation (sparsify_init), recovery, D2H of the result, free."""
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (g.row_ptr, g.col, g.w, g.parent)]
    k = int(math.floor(args.alpha * g.n))
    out_ids = torch.zeros(max(k, 1), dtype=torch.int32).pin_memory()
    out_sc = torch.zeros(max(k, 1), dtype=torch.float64).pin_memory()
    ts = []
    steps = max(1, min(args.steps, 3))
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sp = B.Sparsifier(g.n, *host, stream=torch.cuda.current_stream(dev))
        st, ids, sc, cnt = sp.recover(args.alpha, args.c, out_ids=out_ids, out_scores=out_sc)
        sp.close()
        torch.cuda.synchronize()
        if i > 0:  # first call warms the allocator
            ts.append(time.perf_counter() - t0)
    h2d = sum(int(h.numel() * h.element_size()) for h in host)
    t = float(np.mean(ts))
    return {"value": g.n_offtree / t, "unit": "edges/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": int(cnt) * 12, "ms_per_step": t * 1e3, "steps": steps,
            "includes": "sparsify_init (upload + validation) + recover_offtree + D2H + sparsifier_free"}


def tree_leg(args, g, dev, B, torch):
    """Spanning-tree generation (pdg_spanning_tree) on the headline mesh, device CSR in and device parent out,
    both trees; the maximum-weight tree must equal the workload's own (scipy) tree.  The oracle's Kruskal is
    timed on the same mesh."""
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rp, col, w = t(g.row_ptr, torch.int64), t(g.col, torch.int32), t(g.w, torch.float64)
    out = torch.zeros(g.n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"workload": f"mesh {MESH_SIDE}^3 (n={g.n}, m={g.m})", "unit": "edges/s"}
    for name, kind in (("max_weight", B.TREE_MAX_WEIGHT), ("fegrass_weff", B.TREE_FEGRASS)):
        B.spanning_tree(g.n, rp, col, w, kind=kind, parent_out=out, stream=stream)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.spanning_tree(g.n, rp, col, w, kind=kind, parent_out=out, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        res[name] = {"ms": ms, "value": g.m / (ms / 1e3)}
        if kind == B.TREE_MAX_WEIGHT:
            res[name]["equals_workload_tree"] = bool(np.array_equal(out.cpu().numpy(), g.parent))
    if not args.no_cpu:
        from oracle import oracle as O

        for name, kind in (("max_weight", O.TREE_MAX_WEIGHT), ("fegrass_weff", O.TREE_FEGRASS)):
            t0 = time.perf_counter()
            O.spanning_tree(g, kind)
            dt = time.perf_counter() - t0
            res[name]["cpu_oracle"] = {"value": g.m / dt, "unit": "edges/s", "cores": 1,
                                       "sample": f"the same mesh {MESH_SIDE}^3 (m={g.m}), single-threaded C "
                                                 f"Kruskal, {dt:.2f} s"}
    return res


def pcg_leg(args, B):
    """Sparsifier quality as Sec. 5 measures it: PCG iterations on L_G x = b (tol 1e-3) preconditioned by the
    tree plus the recovered edges, on the 100x100 grid (weights U[1,10], max-weight tree) for alpha = 2/5/10 %
    and the tree alone; the oracle's PCG (scipy LU) beside it unless --no-cpu."""
    from paper_2508_20403_gb300 import workloads as W

    g = W.grid_graph(100)
    b = np.random.default_rng(0).standard_normal(g.n)
    k_max = int(np.floor(0.10 * g.n))
    rows = []
    with B.Sparsifier.from_graph(g) as sp:
        for alpha in (0.0, 0.02, 0.05, 0.10):
            ids = np.zeros(0, dtype=np.int32)
            if alpha > 0:
                st, ids, _, _ = sp.recover(alpha, args.c, capacity=k_max)
                ids = np.asarray(ids, dtype=np.int32)
            t0 = time.perf_counter()
            it, rel = B.pcg_quality(g, ids, b, tol=1e-3)
            row = {"alpha": alpha, "edges": int(ids.size), "iterations": it, "relres": rel,
                   "ms": (time.perf_counter() - t0) * 1e3}
            if not args.no_cpu:
                from oracle import pcg as PC

                row["iterations_oracle"] = PC.pcg_quality(g, ids, b, tol=1e-3)[0]
            rows.append(row)
    return {"workload": f"grid 100x100 (n={g.n}, m={g.m}), weights U[1,10], max-weight tree, c={args.c}",
            "tol": 1e-3, "rows": rows, "mesh64": pcg_mesh64(args, B)}


def pcg_mesh64(args, B):
    """The same measure on the 3D mesh 64^3 (the headline family at 1/8 of its size) at alpha = .02: 5,242 extra
    edges, inside the dense capacitance bound (8,192 edges; mesh 128^3 at .02 has 41,943).  The oracle's count
    (and its range under rounding-level perturbations of b) is the stored one, written by an oracle-only script
    (tests/golden/make_pcg_expect.py), valid when this run recovers the same edges."""
    import hashlib

    from paper_2508_20403_gb300 import workloads as W

    with open(os.path.join(ROOT, "tests", "golden", "pcg_mesh64_expect.json")) as f:
        e = json.load(f)
    g = W.mesh3d_graph(64)
    k = int(math.floor(e["alpha"] * g.n))
    with B.Sparsifier.from_graph(g) as sp:
        st, ids, _, _ = sp.recover(e["alpha"], e["c"], capacity=max(k, 1))
    ids = np.ascontiguousarray(ids, dtype="<i4")
    b = np.random.default_rng(e["b_seed"]).standard_normal(g.n)
    t0 = time.perf_counter()
    it, rel = B.pcg_quality(g, ids, b, tol=e["tol"])
    row = {"workload": f"mesh 64^3 (n={g.n}, m={g.m}), w log-uniform [1e-3,1e3], max-weight tree, c={e['c']}",
           "alpha": e["alpha"], "edges": int(ids.size), "iterations": it, "relres": rel,
           "ms": (time.perf_counter() - t0) * 1e3, "tol": e["tol"]}
    if hashlib.sha256(ids.tobytes()).hexdigest() == e["ids_sha256"]:
        row.update(iterations_oracle=e["iterations"], oracle_count_range=e["count_range"],
                   oracle_source="stored by tests/golden/make_pcg_expect.py (oracle only; same recovered edges)")
    return row


def oracle_sample_recovery(g, args):
    """One step of the oracle's bounded sample (see ORACLE_SAMPLE_ALPHA); returns seconds."""
    from oracle import oracle as O

    t0 = time.perf_counter()
    O.recover(g, ORACLE_SAMPLE_ALPHA, c=args.c)
    return time.perf_counter() - t0


def oracle_sample_text(g, args) -> str:
    ks = int(math.floor(ORACLE_SAMPLE_ALPHA * g.n))
    return (f"one oracle recovery per step on the same mesh {MESH_SIDE}^3 inputs (E_off={g.n_offtree}) and c={args.c} "
            f"with the budget cut to k={ks} (alpha={ORACLE_SAMPLE_ALPHA}): the first {ks} edges of the "
            f"alpha={args.alpha} output (the greedy decides each edge from earlier edges only); all off-tree edges "
            f"are still scored, ordered and grouped; value = E_off / seconds; single-threaded C oracle")


def cpu_parallel_leg(args, g, gpu_ids):
    """The paper's own multi-threaded CPU method (Sec. 4.1 mixed strategy; baseline_cpu/, OpenMP) on the
    headline inputs with every host core: context for the GPU number, with the check that it recovers the same
    edges as the GPU path."""
    from baseline_cpu import omp as P

    P.build()
    cores = os.cpu_count() or 1
    P.recover(g, args.alpha, c=args.c, threads=cores)  # first call: library load, page-in
    ts, ids = [], None
    for _ in range(2):
        t0 = time.perf_counter()
        st, ids, _ = P.recover(g, args.alpha, c=args.c, threads=cores)
        ts.append(time.perf_counter() - t0)
    t = min(ts)
    return {"value": g.n_offtree / t, "unit": "edges/s", "cores": cores, "seconds": t,
            "kind": "the paper's multi-threaded CPU method (mixed outer/inner strategy, cutoff min(1e5, 10 %), "
                    "blocks of p, judge-before-parallel), OpenMP, all steps of the recovery; best of 2",
            "same_edges_as_gpu": bool(np.array_equal(np.asarray(ids), np.asarray(gpu_ids)[:len(ids)]) and
                                      len(ids) == len(gpu_ids)),
            "host": host_cpu()}


def cpu_leg(args, g):
    """The oracle as it stands, single thread, on the bounded sample of the headline workload."""
    from oracle import oracle as O

    O.build()
    t = oracle_sample_recovery(g, args)
    return {"value": g.n_offtree / t, "unit": "edges/s", "cores": 1, "kind": "oracle", "seconds": t,
            "sample": oracle_sample_text(g, args), "host": host_cpu()}


MESH_SIDE = 128
WORKLOAD = "mesh128 (3D 7-point mesh 128^3, w log-uniform [1e-3,1e3], max-weight spanning tree)"


def headline_config(args, world):
    s_ = MESH_SIDE
    n = s_ ** 3
    m = 3 * s_ * s_ * (s_ - 1)
    return {"workload": WORKLOAD, "n": n, "m": m, "n_offtree": m - n + 1, "alpha": args.alpha, "c": args.c,
            "k": int(math.floor(args.alpha * n)), "parallelism": "replicas" if world > 1 else "1 GPU",
            "l2": "256 MB buffer written between timed steps; inputs (175 MB) exceed L2"}


def run_reference(args, rank, world):
    """The oracle on the headline inputs (mesh 128^3), each step the bounded sample described by
    oracle_sample_text; rank 0 only."""
    if rank != 0:
        return None
    from oracle import oracle as O
    from paper_2508_20403_gb300 import workloads as W

    g = W.mesh3d_graph(MESH_SIDE)
    O.build()
    for _ in range(args.warmup):
        oracle_sample_recovery(g, args)
    ts = [oracle_sample_recovery(g, args) for _ in range(args.steps)]
    t = float(np.mean(ts))
    v = g.n_offtree / t
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(args, world),
            "cpu_baseline": {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": oracle_sample_text(g, args), "host": host_cpu()},
            "e2e": {"value": v, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--alpha", type=float, default=0.10)
    ap.add_argument("--c", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tree", action="store_true", help="skip the spanning-tree generation leg")
    ap.add_argument("--no-pcg", action="store_true", help="skip the PCG sparsifier-quality leg")
    ap.add_argument("--no-graph", action="store_true", help="launch kernel by kernel instead of a CUDA graph")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the extra configurations (mesh alpha .02/.05, grid 100^2, R-MAT scale 22)")
    ap.add_argument("--no-rmat", action="store_true", help="skip R-MAT scale 22 in the extra configurations")
    ap.add_argument("--mesh-side", type=int, default=128,
                    help="side of the headline mesh (smaller sides only for profiling captures; the line then "
                         "describes that mesh)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-graphs", type=int, default=2000)
    ap.add_argument("--batch-alpha", type=float, default=0.05)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-pool", type=int, default=128)
    ap.add_argument("--serve-high-rate", type=float, default=1500.0)
    ap.add_argument("--serve-high-seconds", type=float, default=20.0)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-mem-gb", type=int, default=32)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global MESH_SIDE, WORKLOAD
    if args.mesh_side != MESH_SIDE:
        MESH_SIDE = args.mesh_side
        WORKLOAD = WORKLOAD.replace("128^3", f"{MESH_SIDE}^3").replace("mesh128", f"mesh{MESH_SIDE}")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    # the batch and serving legs are reported by rank 0 only (the headline is the replicated recovery)
    batch_graphs = None
    if not args.no_batch and rank == 0:
        # generated in a spawn pool before any CUDA call in this process
        from paper_2508_20403_gb300 import workloads as W

        t0 = time.time()
        batch_graphs = W.batch_graphs(args.batch_graphs, seed=W.SEED_BASE + 3 + 1000 * rank,
                                      workers=min(16, os.cpu_count() or 1))
        log(f"[rank {rank}] generated {len(batch_graphs)} batch graphs in {time.time() - t0:.1f}s")
    serve_graphs = None
    if not args.no_serve and rank == 0:
        t0 = time.time()
        serve_graphs = serve_pool(args, workers=min(16, os.cpu_count() or 1))
        log(f"[rank {rank}] generated {len(serve_graphs)} serving-pool graphs in {time.time() - t0:.1f}s")
    extra_graphs = None
    if not args.no_configs and not args.no_rmat and rank == 0:
        from paper_2508_20403_gb300 import workloads as W

        t0 = time.time()
        extra_graphs = {"rmat22": W.rmat_graph(22, workers=min(16, os.cpu_count() or 1))}
        log(f"[rank {rank}] generated R-MAT scale 22 in {time.time() - t0:.1f}s")
    if world > 1:
        import torch

        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank, batch_graphs, serve_graphs, extra_graphs)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
