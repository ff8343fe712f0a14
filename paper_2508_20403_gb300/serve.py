"""Continuous-batching server for off-tree edge recovery.

Requests (a graph with its spanning tree, a ratio alpha, a cap c) arrive at
any time.  Each of `slots` workers owns a CUDA stream; whenever a worker is
free it takes every queued request that fits the device-memory budget (in
arrival order), packs them into one CSR in the worker's pinned staging
buffers, uploads the batch (sparsify_batch_init: the graphs stay resident in
device memory while the batch runs), runs ONE recover_offtree_batch and
completes the requests.
Requests that arrive while batches are on the GPU are admitted into the next
batch as soon as a slot and memory free up, so the work of several batches
overlaps on the device.  Each request's result is exactly what
recover_offtree returns for its graph alone (the batch path decides every
graph independently).

All recovery work runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import binding as B
from . import workloads as W


def device_bytes_estimate(g) -> int:
    """Upper estimate of the device memory one graph needs inside a batch
    handle (resident CSR and tree, per-edge work arrays, candidate buffers).
    Calibrated from pdg_handle_info on meshes and random geometric graphs."""
    n, m = g.n, g.m
    e_off = max(m - n + 1, 0)
    return int(8 * n + 24 * m + 4 * n  # CSR + parent
               + 8 * n + 16 * n + 12 * n + 2 * 28 * n  # r, P, Euler tour + labels, range-minimum levels (x2 margin)
               + 36 * e_off  # off-tree SoA, keys, LCAs
               + 400 * max(int(0.2 * n), 1024)  # candidate buffers and tables
               + (1 << 20))


@dataclass
class Request:
    graph: object
    alpha: float
    c: int = 2
    rid: int = 0
    t_arrive: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    ids: Optional[np.ndarray] = None
    scores: Optional[np.ndarray] = None
    status: int = 0
    batch: int = -1
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


class Server:
    def __init__(self, mem_budget_bytes: int = 16 << 30, slots: int = 4, max_batch_graphs: int = 512,
                 device: int = 0, use_graph: bool = False, staging_hint=(0, 0)):
        import torch

        self.torch = torch
        self.device = device
        self.mem_budget = int(mem_budget_bytes)
        self.mem_free = int(mem_budget_bytes)
        self.max_batch = max_batch_graphs
        self.slots = slots
        self.use_graph = use_graph
        self.queue: collections.deque = collections.deque()
        self.cv = threading.Condition()
        self.stop_flag = False
        self.workers: List[threading.Thread] = []
        self.batches = 0
        self.batch_sizes: List[int] = []
        self.inflight = 0
        self.max_inflight = 0
        self.completed: List[Request] = []
        self.errors: List[str] = []
        self._rid = 0
        # (vertices, CSR entries) every worker's pinned staging holds from the start (pinned allocations are
        # slow: growing them under load stalls the worker)
        self.staging_hint = staging_hint

    # ------------------------------------------------------------------ API
    def start(self):
        B.load()
        self._ready = threading.Semaphore(0)
        for i in range(self.slots):
            t = threading.Thread(target=self._worker, args=(i,), daemon=True)
            t.start()
            self.workers.append(t)
        for _ in range(self.slots):  # every worker has its stream and staging before requests are taken
            self._ready.acquire()
        return self

    def submit(self, graph, alpha: float, c: int = 2) -> Request:
        need = device_bytes_estimate(graph)
        if need > self.mem_budget:
            raise ValueError("request larger than the whole device-memory budget")
        with self.cv:
            r = Request(graph=graph, alpha=float(alpha), c=int(c), rid=self._rid, t_arrive=time.perf_counter())
            self._rid += 1
            self.queue.append(r)
            self.cv.notify()
        return r

    def stop(self):
        with self.cv:
            self.stop_flag = True
            self.cv.notify_all()
        for t in self.workers:
            t.join()

    # ------------------------------------------------------------ internals
    def _take_batch(self):
        """Under the lock: take queued requests in arrival order while they
        fit the free memory; all share one c."""
        taken, mem = [], 0
        while self.queue and len(taken) < self.max_batch:
            r = self.queue[0]
            need = device_bytes_estimate(r.graph)
            if mem + need > self.mem_free or (taken and r.c != taken[0].c):
                break
            taken.append(self.queue.popleft())
            mem += need
        self.mem_free -= mem
        return taken, mem

    def _worker(self, slot: int):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        staging = _Staging(torch)
        try:
            if self.staging_hint[0] > 0:
                staging.get(*self.staging_hint)
        finally:
            self._ready.release()
        while True:
            with self.cv:
                while not self.stop_flag and not self.queue:
                    self.cv.wait()
                if self.stop_flag and not self.queue:
                    return
                batch, mem = self._take_batch()
                if not batch:  # the head request waits for memory to free up
                    self.cv.wait(timeout=0.001)
                    continue
                self.batches += 1
                bid = self.batches
                self.inflight += 1
                self.max_inflight = max(self.max_inflight, self.inflight)
            try:
                self._run_batch(batch, bid, stream, staging)
            except Exception as e:  # report, complete the requests with an error status
                self.errors.append(repr(e))
                for r in batch:
                    r.status = B.PDG_E_CUDA
                    r.t_done = time.perf_counter()
                    r.done.set()
            finally:
                with self.cv:
                    self.mem_free += mem
                    self.inflight -= 1
                    self.batch_sizes.append(len(batch))
                    self.cv.notify_all()

    def _run_batch(self, batch, bid, stream, staging):
        t0 = time.perf_counter()
        for r in batch:
            r.t_start = t0
            r.batch = bid
        graphs = [r.graph for r in batch]
        N, nnz = W.packed_sizes(graphs)
        bufs = staging.get(N, nnz)  # the batch is packed straight into pinned memory (one copy, DMA upload)
        pk = W.pack_graphs(graphs, out=tuple(b.numpy() for b in bufs))
        alphas = np.array([r.alpha for r in batch], dtype=np.float64)
        opt = B.default_options(use_graph=1 if self.use_graph else 0)
        with B.BatchSparsifier(pk.vtx_ptr, bufs[0][:N + 1], bufs[1][:nnz], bufs[2][:nnz], bufs[3][:N], options=opt,
                               stream=stream.cuda_stream) as bs:
            st, op, ids, sc, counts, gst = bs.recover_batch(alphas, c=batch[0].c)
        t1 = time.perf_counter()
        with self.cv:
            for i, r in enumerate(batch):
                r.ids = ids[op[i]:op[i] + counts[i]].copy()
                r.scores = sc[op[i]:op[i] + counts[i]].copy()
                r.status = int(gst[i])
                r.t_done = t1
                self.completed.append(r)
                r.done.set()


class _Staging:
    """Pinned host buffers of one worker (row_ptr, col, w, parent of a packed batch), grown on demand."""

    def __init__(self, torch):
        self.torch = torch
        self.cap = (0, 0)
        self.bufs = None

    def get(self, N: int, nnz: int):
        if self.bufs is None or N + 1 > self.cap[0] or nnz > self.cap[1]:
            torch = self.torch
            cn, ce = max(N + 1, 2 * self.cap[0]), max(nnz, 2 * self.cap[1], 1)
            self.bufs = (torch.empty(cn, dtype=torch.int64, pin_memory=True),
                         torch.empty(ce, dtype=torch.int32, pin_memory=True),
                         torch.empty(ce, dtype=torch.float64, pin_memory=True),
                         torch.empty(cn, dtype=torch.int32, pin_memory=True))
            self.cap = (cn, ce)
        return self.bufs


def poisson_arrivals(rate: float, duration: float, rng: np.random.Generator) -> np.ndarray:
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.array(out)
        out.append(t)


def run_stream(server: Server, pool, rate: float, duration: float, seed: int = 20250833,
               alphas=(0.02, 0.05, 0.10), c: int = 2):
    """Feed a Poisson stream drawn from `pool`; returns the requests."""
    rng = np.random.default_rng(seed)
    times = poisson_arrivals(rate, duration, rng)
    picks = rng.integers(0, len(pool), size=times.shape[0])
    avals = rng.choice(np.asarray(alphas), size=times.shape[0])
    reqs = []
    t0 = time.perf_counter()
    for t, p, a in zip(times, picks, avals):
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        reqs.append(server.submit(pool[int(p)], float(a), c))
    for r in reqs:
        r.done.wait()
    return reqs


def summarize(reqs, wall: float) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    ok = sum(1 for r in reqs if r.status >= 0)
    edges = sum(r.graph.n_offtree for r in reqs)
    return {"requests": len(reqs), "ok": ok, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "graphs_per_s": len(reqs) / wall, "offtree_edges_per_s": edges / wall}
