"""Python binding of the C ABI in include/pdgrass.h (argument marshalling only).

Every step of the recovery runs in the CUDA library; this module converts
numpy arrays / torch tensors into pointers and sizes.  It never falls back
to anything: if the compiled library is missing it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdgrass.so")

PDG_OK = 0
PDG_UNDER_BUDGET = 1
PDG_E_INVALID_ARG = -1
PDG_E_NOT_SYMMETRIC = -2
PDG_E_NOT_A_TREE = -3
PDG_E_BAD_WEIGHT = -4
PDG_E_RANGE = -5
PDG_E_CAPACITY = -6
PDG_E_OOM = -7
PDG_E_CUDA = -8
PDG_E_TIMEOUT = -9
PDG_E_NOT_CSR = -10
MEM_HOST = 0
MEM_DEVICE = 1
SCORE_STRETCH = 0
SCORE_RESISTANCE = 1
MAX_C = 3
TREE_MAX_WEIGHT = 0
TREE_FEGRASS = 1

EXPORTS = ("pdg_default_options", "pdg_status_string", "sparsify_init", "recover_offtree", "sparsifier_free",
           "pdg_edge_endpoints", "sparsify_batch_init", "recover_offtree_batch", "pdg_handle_info",
           "pdg_last_stats", "pdg_last_timings", "pdg_spanning_tree", "pdg_pcg_quality", "pdg_pcg_trace",
           "pdg_edge_endpoints_noalloc")
STEP_NAMES = ("classify", "tree", "score", "select", "sort", "accept", "budget", "total")


class PdgError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: status {status} ({status_string(status)})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("score_mode", ctypes.c_int32), ("warp_tier_max", ctypes.c_int32), ("k_override", ctypes.c_int64),
                ("candidate_factor", ctypes.c_double), ("max_rounds", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("profile", ctypes.c_int32), ("block_tier_max", ctypes.c_int32),
                ("sort_tile_keys", ctypes.c_int32), ("sort_one_launch", ctypes.c_int32)]


_lib = None


def load(path: Optional[str] = None):
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CUDA library not built: {p} (run paper_2508_20403_gb300.build.build())")
    L = ctypes.CDLL(p)
    P, i64, i32, f64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
    L.pdg_default_options.argtypes = [ctypes.POINTER(Options)]
    L.pdg_default_options.restype = None
    L.pdg_status_string.argtypes = [c_int]
    L.pdg_status_string.restype = ctypes.c_char_p
    L.sparsify_init.argtypes = [ctypes.POINTER(P), i64, P, P, P, P, c_int, ctypes.POINTER(Options), P]
    L.sparsify_init.restype = c_int
    L.recover_offtree.argtypes = [P, f64, i32, P, i64, ctypes.POINTER(i64), P, c_int]
    L.recover_offtree.restype = c_int
    L.sparsifier_free.argtypes = [P]
    L.sparsifier_free.restype = None
    L.pdg_edge_endpoints.argtypes = [P, P, i64, P, P, c_int]
    L.pdg_edge_endpoints.restype = c_int
    L.sparsify_batch_init.argtypes = [ctypes.POINTER(P), i32, P, P, P, P, P, c_int, ctypes.POINTER(Options), P]
    L.sparsify_batch_init.restype = c_int
    L.recover_offtree_batch.argtypes = [P, P, i32, P, P, P, P, P, c_int]
    L.recover_offtree_batch.restype = c_int
    L.pdg_handle_info.argtypes = [P, P, P, P, P, P, P]
    L.pdg_handle_info.restype = c_int
    L.pdg_last_stats.argtypes = [P, P]
    L.pdg_last_stats.restype = c_int
    L.pdg_last_timings.argtypes = [P, P]
    L.pdg_last_timings.restype = c_int
    L.pdg_edge_endpoints_noalloc.argtypes = [i64, P, P, P, i64, P, P, P]
    L.pdg_edge_endpoints_noalloc.restype = c_int
    L.pdg_spanning_tree.argtypes = [i64, P, P, P, c_int, c_int, P, c_int, P]
    L.pdg_spanning_tree.restype = c_int
    L.pdg_pcg_quality.argtypes = [i64, P, P, P, P, P, i64, P, f64, i32, c_int, P, P, P]
    L.pdg_pcg_quality.restype = c_int
    L.pdg_pcg_trace.argtypes = [i64, P, P, P, P, P, i64, P, f64, i32, c_int, P, P, P, P, P]
    L.pdg_pcg_trace.restype = c_int
    if path is None:
        _lib = L
    return L


def spanning_tree(n: int, row_ptr, col, w, kind: int = TREE_MAX_WEIGHT, parent_out=None, stream=None):
    """pdg_spanning_tree: the parent array of the generated spanning tree (numpy int32, or written into the
    given device tensor `parent_out`).  Inputs are numpy arrays or CUDA tensors (all in one memory)."""
    L = load()
    kind_in = _mem_kind([row_ptr, col, w])
    if kind_in == MEM_HOST:
        row_ptr = _host_arr(row_ptr, np.int64)
        col = _host_arr(col, np.int32)
        w = _host_arr(w, np.float64)
    out = parent_out if parent_out is not None else np.zeros(int(n), dtype=np.int32)
    st = L.pdg_spanning_tree(int(n), _ptr(row_ptr), _ptr(col), _ptr(w), kind_in, int(kind), _ptr(out),
                             _mem_kind([out]), _stream_ptr(stream))
    if st != PDG_OK:
        raise PdgError(st, "pdg_spanning_tree")
    return out


def pcg_quality(g, edge_ids, b, tol: float = 1e-3, max_iter: int = 1000, stream=None):
    """pdg_pcg_quality on a workloads.Graph (host arrays): (iterations, final relative residual)."""
    L = load()
    rp = _host_arr(g.row_ptr, np.int64)
    col = _host_arr(g.col, np.int32)
    w = _host_arr(g.w, np.float64)
    par = _host_arr(g.parent, np.int32)
    ids = _host_arr(edge_ids, np.int32)
    bb = _host_arr(b, np.float64)
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = L.pdg_pcg_quality(int(g.n), _ptr(rp), _ptr(col), _ptr(w), _ptr(par), _ptr(ids) if ids.size else None,
                           int(ids.size), _ptr(bb), float(tol), int(max_iter), MEM_HOST, ctypes.byref(it),
                           ctypes.byref(rel), _stream_ptr(stream))
    if st != PDG_OK:
        raise PdgError(st, "pdg_pcg_quality")
    return int(it.value), float(rel.value)


def pcg_trace(g, edge_ids, b, tol: float = 1e-3, max_iter: int = 1000, stream=None):
    """pdg_pcg_trace on a workloads.Graph (host arrays): (iterations, final relative residual, the relative
    residual after each iteration, the preconditioner applied to the centred right-hand side)."""
    L = load()
    rp = _host_arr(g.row_ptr, np.int64)
    col = _host_arr(g.col, np.int32)
    w = _host_arr(g.w, np.float64)
    par = _host_arr(g.parent, np.int32)
    ids = _host_arr(edge_ids, np.int32)
    bb = _host_arr(b, np.float64)
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    hist = np.zeros(int(max_iter), dtype=np.float64)
    z0 = np.zeros(int(g.n), dtype=np.float64)
    st = L.pdg_pcg_trace(int(g.n), _ptr(rp), _ptr(col), _ptr(w), _ptr(par), _ptr(ids) if ids.size else None,
                         int(ids.size), _ptr(bb), float(tol), int(max_iter), MEM_HOST, ctypes.byref(it),
                         ctypes.byref(rel), _ptr(hist), _ptr(z0), _stream_ptr(stream))
    if st != PDG_OK:
        raise PdgError(st, "pdg_pcg_trace")
    return int(it.value), float(rel.value), hist[:int(it.value)].copy(), z0


def status_string(status: int) -> str:
    return load().pdg_status_string(int(status)).decode()


def default_options(**overrides) -> Options:
    o = Options()
    load().pdg_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(a) -> int:
    if _is_torch(a):
        assert a.is_contiguous()
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _mem_kind(arrays) -> int:
    kinds = {MEM_DEVICE if (_is_torch(a) and a.is_cuda) else MEM_HOST for a in arrays}
    if len(kinds) != 1:
        raise ValueError("all arrays of one call must live in the same memory (host or device)")
    return kinds.pop()


def _host_arr(a, dtype):
    if _is_torch(a):
        import torch

        tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        return (a if a.dtype == tdt else a.to(tdt)).contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_ptr(stream) -> int:
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    return stream if isinstance(stream, int) else stream.cuda_stream


class Sparsifier:
    """One graph + spanning tree resident on the device (sparsify_init)."""

    def __init__(self, n: int, row_ptr, col, w, parent, options: Optional[Options] = None, stream=None):
        L = load()
        self._L = L
        self._h = ctypes.c_void_p()
        kind = _mem_kind([row_ptr, col, w, parent])
        if kind == MEM_HOST:
            row_ptr = _host_arr(row_ptr, np.int64)
            col = _host_arr(col, np.int32)
            w = _host_arr(w, np.float64)
            parent = _host_arr(parent, np.int32)
        self._keep = (row_ptr, col, w, parent)
        opt = options or default_options()
        st = L.sparsify_init(ctypes.byref(self._h), int(n), _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(parent), kind,
                             ctypes.byref(opt), _stream_ptr(stream))
        self._keep = None
        if st != PDG_OK:
            raise PdgError(st, "sparsify_init")
        self.n = int(n)

    @classmethod
    def from_graph(cls, g, device: bool = False, **kw):
        if device:
            import torch

            t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()
            return cls(g.n, t(g.row_ptr, torch.int64), t(g.col, torch.int32), t(g.w, torch.float64),
                       t(g.parent, torch.int32), **kw)
        return cls(g.n, g.row_ptr, g.col, g.w, g.parent, **kw)

    def info(self) -> dict:
        v = [ctypes.c_int64() for _ in range(3)]
        G = ctypes.c_int32()
        md = ctypes.c_int64()
        db = ctypes.c_int64()
        st = self._L.pdg_handle_info(self._h, ctypes.byref(v[0]), ctypes.byref(v[1]), ctypes.byref(v[2]),
                                     ctypes.byref(G), ctypes.byref(md), ctypes.byref(db))
        if st:
            raise PdgError(st, "pdg_handle_info")
        return dict(n=v[0].value, m=v[1].value, n_offtree=v[2].value, num_graphs=G.value, max_depth=md.value,
                    device_bytes=db.value)

    def last_stats(self) -> dict:
        a = np.zeros(12, dtype=np.int64)
        self._L.pdg_last_stats(self._h, a.ctypes.data)
        keys = ("candidates", "subtasks", "max_subtask", "warp_or_single", "coop_candidates", "coop_rounds",
                "retries", "attempts", "launches", "coop_constrained", "coop_pairs", "bounds_site")
        return dict(zip(keys, (int(x) for x in a)))

    def last_timings(self) -> dict:
        a = np.zeros(8, dtype=np.float32)
        self._L.pdg_last_timings(self._h, a.ctypes.data)
        return dict(zip(STEP_NAMES, (float(x) for x in a)))

    def recover(self, alpha: float, c: int = 2, out_ids=None, out_scores=None, capacity: Optional[int] = None,
                want_scores: bool = True):
        """Returns (status, ids, scores, count).  With out_ids given (numpy or
        torch, host or device) the results are written there."""
        if out_ids is None:
            info = self.info()
            cap = capacity if capacity is not None else max(1, min(int(np.floor(alpha * self.n)), info["n_offtree"]))
            out_ids = np.zeros(cap, dtype=np.int32)
            out_scores = np.zeros(cap, dtype=np.float64) if want_scores else None
        cap = out_ids.shape[0] if capacity is None else capacity
        kind = _mem_kind([out_ids] + ([out_scores] if out_scores is not None else []))
        cnt = ctypes.c_int64()
        st = self._L.recover_offtree(self._h, float(alpha), int(c), _ptr(out_ids), int(cap), ctypes.byref(cnt),
                                     _ptr(out_scores) if out_scores is not None else None, kind)
        if st < 0:
            raise PdgError(st, "recover_offtree")
        k = cnt.value
        return st, out_ids[:k], (out_scores[:k] if out_scores is not None else None), k

    def endpoints(self, ids) -> tuple:
        ids = _host_arr(ids, np.int32) if not (_is_torch(ids) and ids.is_cuda) else ids
        kind = _mem_kind([ids])
        if kind == MEM_HOST:
            u = np.zeros(ids.shape[0], dtype=np.int32)
            v = np.zeros(ids.shape[0], dtype=np.int32)
        else:
            import torch

            u = torch.empty_like(ids)
            v = torch.empty_like(ids)
        st = self._L.pdg_edge_endpoints(self._h, _ptr(ids), int(ids.shape[0]), _ptr(u), _ptr(v), kind)
        if st:
            raise PdgError(st, "pdg_edge_endpoints")
        return u, v

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.sparsifier_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


NOALLOC_MAX_N = 1 << 21


def edge_endpoints_noalloc(n: int, row_ptr, col, ids, u, v, stream=None) -> int:
    """pdg_edge_endpoints_noalloc on caller-owned DEVICE tensors: maps
    canonical edge ids to endpoints without allocating device memory (for
    callers restricted to their own memory pool or that must not stall on
    the allocator).  Calls on one device share the library's fixed scratch
    array and must not overlap.  Returns the status code."""
    return load().pdg_edge_endpoints_noalloc(int(n), _ptr(row_ptr), _ptr(col), _ptr(ids), int(ids.shape[0]),
                                             _ptr(u), _ptr(v), _stream_ptr(stream))


class BatchSparsifier(Sparsifier):
    """Many graphs packed into one CSR (sparsify_batch_init)."""

    def __init__(self, vtx_ptr, row_ptr, col, w, parent, options: Optional[Options] = None, stream=None):
        L = load()
        self._L = L
        self._h = ctypes.c_void_p()
        vp = np.ascontiguousarray(vtx_ptr, dtype=np.int64)
        kind = _mem_kind([row_ptr, col, w, parent])
        if kind == MEM_HOST:
            row_ptr = _host_arr(row_ptr, np.int64)
            col = _host_arr(col, np.int32)
            w = _host_arr(w, np.float64)
            parent = _host_arr(parent, np.int32)
        opt = options or default_options()
        st = L.sparsify_batch_init(ctypes.byref(self._h), int(vp.shape[0] - 1), vp.ctypes.data, _ptr(row_ptr),
                                   _ptr(col), _ptr(w), _ptr(parent), kind, ctypes.byref(opt), _stream_ptr(stream))
        if st != PDG_OK:
            raise PdgError(st, "sparsify_batch_init")
        self.vtx_ptr = vp
        self.num_graphs = int(vp.shape[0] - 1)
        self.n = int(vp[-1])

    @classmethod
    def from_packed(cls, pk, device: bool = False, **kw):
        if device:
            import torch

            t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()
            return cls(pk.vtx_ptr, t(pk.row_ptr, torch.int64), t(pk.col, torch.int32), t(pk.w, torch.float64),
                       t(pk.parent, torch.int32), **kw)
        return cls(pk.vtx_ptr, pk.row_ptr, pk.col, pk.w, pk.parent, **kw)

    def out_ptr_for(self, alphas: Sequence[float]) -> np.ndarray:
        nv = np.diff(self.vtx_ptr)
        k = np.floor(np.asarray(alphas, dtype=np.float64) * nv.astype(np.float64)).astype(np.int64)
        op = np.zeros(self.num_graphs + 1, dtype=np.int64)
        np.cumsum(np.maximum(k, 0), out=op[1:])
        return op

    def recover_batch(self, alphas, c: int = 2, out_ptr=None, out_ids=None, out_scores=None,
                      want_scores: bool = True):
        """Returns (status, out_ptr, ids, scores, counts, per_graph_status)."""
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(alphas, dtype=np.float64), (self.num_graphs,)))
        op = self.out_ptr_for(a) if out_ptr is None else np.ascontiguousarray(out_ptr, dtype=np.int64)
        if out_ids is None:
            out_ids = np.zeros(max(int(op[-1]), 1), dtype=np.int32)
            out_scores = np.zeros(max(int(op[-1]), 1), dtype=np.float64) if want_scores else None
        kind = _mem_kind([out_ids] + ([out_scores] if out_scores is not None else []))
        counts = np.zeros(self.num_graphs, dtype=np.int64)
        gst = np.zeros(self.num_graphs, dtype=np.int32)
        st = self._L.recover_offtree_batch(self._h, a.ctypes.data, int(c), op.ctypes.data, _ptr(out_ids),
                                           counts.ctypes.data,
                                           _ptr(out_scores) if out_scores is not None else None, gst.ctypes.data,
                                           kind)
        if st < 0:
            raise PdgError(st, "recover_offtree_batch")
        return st, op, out_ids, out_scores, counts, gst
