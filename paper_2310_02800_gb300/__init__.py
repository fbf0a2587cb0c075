"""GB300-native temporal motif mining (Everest problem, paper arXiv 2310.02800).

Thin Python binding over the C ABI in include/tm.h (libtmgb300.so): argument
marshalling only -- every step of the search runs in the library's CUDA
kernels.  PyTorch supplies device memory (tensors) and streams.  There is no
CPU fallback: importing the binding without the compiled library raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libtmgb300.so")

MAX_EDGES = 8
MAX_NODES = 8
MAX_ANTI = 4
INT64_MAX = np.iinfo(np.int64).max

OK, E_INVALID, E_OOM, E_TRUNCATED, E_TIMEOUT, E_CUDA, E_BUSY, E_ADMISSION = range(8)


class TMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tm status {status}: {msg}")
        self.status = status


class _Edges(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("t", ctypes.c_void_p),
                ("elabel", ctypes.c_void_p), ("nlabel", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class _Motif(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("esrc", ctypes.c_uint8 * MAX_EDGES), ("edst", ctypes.c_uint8 * MAX_EDGES),
                ("delta", ctypes.c_int64), ("gap", ctypes.c_int64 * (MAX_EDGES - 1)),
                ("elabel", ctypes.c_int16 * MAX_EDGES), ("nlabel", ctypes.c_int16 * MAX_NODES),
                ("n_anti", ctypes.c_int32), ("anti_src", ctypes.c_uint8 * MAX_ANTI),
                ("anti_dst", ctypes.c_uint8 * MAX_ANTI), ("anti_edge", ctypes.c_uint8 * MAX_ANTI),
                ("anti_delta", ctypes.c_int64 * MAX_ANTI)]


class Tuning(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("chunk_roots", ctypes.c_int32),
                ("split_depth", ctypes.c_int32), ("split_min", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class _Work(ctypes.Structure):
    _fields_ = [("roots", ctypes.c_uint64), ("nodes", ctypes.c_uint64 * MAX_EDGES),
                ("entries", ctypes.c_uint64 * MAX_EDGES), ("probe_sectors", ctypes.c_uint64),
                ("matches", ctypes.c_uint64)]


class _ServeCfg(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("grid_pct", ctypes.c_int32), ("policy", ctypes.c_int32), ("long_ms", ctypes.c_double),
                ("batch_ms", ctypes.c_double)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("total", ctypes.c_uint64), ("n_written", ctypes.c_uint64),
                ("matches_dev", ctypes.c_void_p), ("k", ctypes.c_int32), ("submit_to_done_ms", ctypes.c_double)]


_lib = None

# (name, restype, argtypes) of every entry point in include/tm.h
_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_SIGS = [
    ("tm_graph_load", ctypes.c_int, [ctypes.POINTER(_Edges), ctypes.c_int, _P, _PP]),
    ("tm_graph_free", ctypes.c_int, [_P]),
    ("tm_graph_info", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _U64P]),
    ("tm_graph_edge_perm", ctypes.c_int, [_P, _P]),
    ("tm_query_compile", ctypes.c_int, [_P, ctypes.POINTER(_Motif), _PP]),
    ("tm_query_free", ctypes.c_int, [_P]),
    ("tm_query_set_tuning", ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    ("tm_query_get_tuning", ctypes.c_int, [_P, ctypes.POINTER(Tuning)]),
    ("tm_count", ctypes.c_int, [_P, _P, _P, _U64P, _P]),
    ("tm_count_roots", ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P, _U64P, _P]),
    ("tm_enumerate", ctypes.c_int, [_P, _P, _P, _P, ctypes.c_uint64, _U64P, _U64P]),
    ("tm_count_batch", ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    ("tm_enumerate_batch", ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P, _P, _P, _P, _P]),
    ("tm_count_batch_noalloc", ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
    ("tm_autotune", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Tuning)]),
    ("tm_count_baseline", ctypes.c_int, [_P, _P, _P, _U64P, ctypes.POINTER(ctypes.c_double)]),
    ("tm_query_work", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_Work)]),
    ("tm_serve_start", ctypes.c_int, [_P, ctypes.POINTER(_ServeCfg), _PP]),
    ("tm_serve_submit", ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_uint64, _U64P]),
    ("tm_serve_poll", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_Result)]),
    ("tm_serve_wait", ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(_Result)]),
    ("tm_result_release", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("tm_serve_stop", ctypes.c_int, [_P]),
    ("tm_query_profile", ctypes.c_int, [_P, ctypes.c_int]),
    ("tm_query_last_ms", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("tm_kernel_launches", ctypes.c_uint64, []),
    ("tm_query_inject_fault", ctypes.c_int, [_P, ctypes.c_int]),
    ("tm_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("tm_last_error", ctypes.c_char_p, []),
    ("tm_last_search_stats", ctypes.c_int, [_U64P, _U64P]),
    ("tm_inject_alloc_failure", ctypes.c_int, [ctypes.c_int64]),
]


def kernel_launches() -> int:
    return int(lib().tm_kernel_launches())


def last_search_stats() -> dict:
    """Donation counters of the calling thread's last count-mode launch."""
    d, r = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().tm_last_search_stats(ctypes.byref(d), ctypes.byref(r)))
    return {"donated": int(d.value), "reserved": int(r.value)}


def inject_alloc_failure(after: int = 0):
    """Test hook: the library's allocation after `after` further successful ones fails (TM_E_OOM)."""
    _check(lib().tm_inject_alloc_failure(int(after)))


def library_path() -> str:
    return _SO


def lib():
    """The loaded C library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise ImportError(f"{_SO} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(_SO)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, allow=(OK,)):
    if status not in allow:
        L = lib()
        raise TMError(status, f"{L.tm_status_str(status).decode()}: {L.tm_last_error().decode()}")
    return status


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def make_motif(edges, delta, gaps=None, elabel=None, nlabel=None, n_nodes=None, anti=None) -> _Motif:
    """anti: list of (src node, dst node, attached edge index, delta) temporal anti-edges."""
    m = _Motif()
    m.k = len(edges)
    m.n_nodes = n_nodes if n_nodes is not None else 1 + max(max(e) for e in edges)
    for i, (x, y) in enumerate(edges):
        m.esrc[i] = x; m.edst[i] = y
    m.delta = int(delta)
    for i in range(MAX_EDGES - 1):
        g = None if gaps is None or i >= len(gaps) else gaps[i]
        m.gap[i] = INT64_MAX if g is None else int(g)
    for i in range(MAX_EDGES):
        m.elabel[i] = -1 if elabel is None or i >= len(elabel) else int(elabel[i])
    for j in range(MAX_NODES):
        m.nlabel[j] = -1 if nlabel is None or j >= len(nlabel) else int(nlabel[j])
    anti = anti or []
    m.n_anti = len(anti)
    for a, (x, y, e, d) in enumerate(anti):
        m.anti_src[a] = x; m.anti_dst[a] = y; m.anti_edge[a] = e; m.anti_delta[a] = int(d)
    return m


def motif_of(obj) -> _Motif:
    """Motif struct from an object with edges / delta / gaps / elabel / nlabel."""
    if isinstance(obj, _Motif):
        return obj
    return make_motif(obj.edges, obj.delta, getattr(obj, "gaps", None), getattr(obj, "elabel", None),
                      getattr(obj, "nlabel", None), anti=getattr(obj, "anti", None))


def _ptr(x):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


class Graph:
    """Device-resident temporal graph (tm_graph)."""

    def __init__(self, handle, device, keep=None):
        self._h = handle
        self.device = device
        info_n, info_m, info_b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint64()
        _check(lib().tm_graph_info(self._h, ctypes.byref(info_n), ctypes.byref(info_m), ctypes.byref(info_b)))
        self.n_nodes, self.n_edges, self.device_bytes = info_n.value, info_m.value, info_b.value

    @classmethod
    def load(cls, n_nodes, src, dst, t, elabel=None, nlabel=None, device=0, stream=None):
        """src/dst int32, t int64, labels uint8: numpy arrays (host) or CUDA tensors (device)."""
        on_dev = not isinstance(src, np.ndarray)
        if not on_dev:
            src = np.ascontiguousarray(src, np.int32); dst = np.ascontiguousarray(dst, np.int32)
            t = np.ascontiguousarray(t, np.int64)
            elabel = None if elabel is None else np.ascontiguousarray(elabel, np.uint8)
            nlabel = None if nlabel is None else np.ascontiguousarray(nlabel, np.uint8)
        e = _Edges(int(n_nodes), int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(t), _ptr(elabel), _ptr(nlabel),
                   1 if on_dev else 0)
        h = ctypes.c_void_p()
        _check(lib().tm_graph_load(ctypes.byref(e), int(device), _stream_ptr(stream), ctypes.byref(h)))
        return cls(h, device)

    @classmethod
    def from_synth(cls, g, device=0, stream=None):
        return cls.load(g.n_nodes, g.src, g.dst, g.t, g.elabel, g.nlabel, device, stream)

    def free(self):
        if getattr(self, "_h", None):
            lib().tm_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def edge_perm(self) -> np.ndarray:
        out = np.empty(self.n_edges, np.int64)
        _check(lib().tm_graph_edge_perm(self._h, out.ctypes.data))
        return out

    def compile(self, motif) -> "Query":
        h = ctypes.c_void_p()
        m = motif_of(motif)
        _check(lib().tm_query_compile(self._h, ctypes.byref(m), ctypes.byref(h)))
        return Query(self, h, m)

    def count_batch(self, queries, stream=None) -> list:
        arr = (ctypes.c_void_p * len(queries))(*[q._h.value for q in queries])
        out = np.zeros(len(queries), np.uint64)
        _check(lib().tm_count_batch(self._h, arr, len(queries), _stream_ptr(stream), out.ctypes.data))
        return [int(x) for x in out]

    def enumerate_batch(self, queries, outs, stream=None, timed=False):
        """Enumerate several queries together (tm_enumerate_batch).  outs[j]: int32 CUDA tensor
        [cap_j, k_j] (or None for a count only).  Returns (n_written, totals, truncated) lists /
        flag, plus (count ms, fill ms) when timed."""
        n = len(queries)
        arr = (ctypes.c_void_p * n)(*[q._h.value for q in queries])
        bufs = (ctypes.c_void_p * n)(*[None if o is None else _ptr(o) for o in outs])
        caps = np.array([0 if o is None else int(o.shape[0]) for o in outs], np.uint64)
        nw = np.zeros(n, np.uint64)
        tot = np.zeros(n, np.uint64)
        ms = (ctypes.c_double * 2)()
        st = _check(lib().tm_enumerate_batch(self._h, arr, n, _stream_ptr(stream), bufs, caps.ctypes.data,
                                             nw.ctypes.data, tot.ctypes.data, ms if timed else None),
                    allow=(OK, E_TRUNCATED))
        res = ([int(x) for x in nw], [int(x) for x in tot], st == E_TRUNCATED)
        return res + ((ms[0], ms[1]),) if timed else res

    def count_batch_noalloc(self, queries, totals, stream=None):
        """Batched count that allocates nothing: totals is a caller-owned uint64/int64 CUDA tensor
        with len(queries) entries (at most 64 queries per call)."""
        arr = (ctypes.c_void_p * len(queries))(*[q._h.value for q in queries])
        _check(lib().tm_count_batch_noalloc(self._h, arr, len(queries), _stream_ptr(stream), _ptr(totals)))
        return totals

    def serve(self, mem_budget_bytes=0, streams=0, max_batch=0, grid_pct=0, policy=0, long_ms=0.0,
              batch_ms=0.0) -> "Server":
        """Start a serving loop (tm_serve_start); zeros select the library defaults."""
        cfg = _ServeCfg(int(mem_budget_bytes), int(streams), int(max_batch), int(grid_pct), int(policy),
                        float(long_ms), float(batch_ms))
        h = ctypes.c_void_p()
        _check(lib().tm_serve_start(self._h, ctypes.byref(cfg), ctypes.byref(h)))
        return Server(self, h)


class Query:
    """Compiled motif query (tm_query)."""

    def __init__(self, graph: Graph, handle, motif: _Motif):
        self.graph = graph
        self._h = handle
        self.k = int(motif.k)

    def free(self):
        if getattr(self, "_h", None):
            lib().tm_query_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def tuning(self) -> Tuning:
        t = Tuning()
        _check(lib().tm_query_get_tuning(self._h, ctypes.byref(t)))
        return t

    def set_tuning(self, warps_per_block=4, chunk_roots=256, split_depth=1, split_min=256):
        t = Tuning(warps_per_block, chunk_roots, split_depth, split_min)
        _check(lib().tm_query_set_tuning(self._h, ctypes.byref(t)))

    def count(self, per_root=None, stream=None) -> int:
        """Exact count; per_root: optional uint64/int64 CUDA tensor of n_edges entries (filled)."""
        tot = ctypes.c_uint64()
        _check(lib().tm_count(self.graph._h, self._h, _stream_ptr(stream), ctypes.byref(tot), _ptr(per_root)))
        return tot.value

    def count_roots(self, root_begin, root_end, per_root=None, stream=None) -> int:
        tot = ctypes.c_uint64()
        _check(lib().tm_count_roots(self.graph._h, self._h, int(root_begin), int(root_end), _stream_ptr(stream),
                                    ctypes.byref(tot), _ptr(per_root)))
        return tot.value

    def enumerate(self, out, stream=None):
        """Fill out (int32 CUDA tensor [cap, k]); returns (n_written, total, truncated)."""
        cap = int(out.shape[0])
        nw, tot = ctypes.c_uint64(), ctypes.c_uint64()
        st = _check(lib().tm_enumerate(self.graph._h, self._h, _stream_ptr(stream), _ptr(out), cap,
                                       ctypes.byref(nw), ctypes.byref(tot)), allow=(OK, E_TRUNCATED))
        return nw.value, tot.value, st == E_TRUNCATED

    def count_baseline(self, stream=None):
        """(count, kernel ms) with the paper's thread-per-tree GPU baseline design (ablation)."""
        tot, ms = ctypes.c_uint64(), ctypes.c_double()
        _check(lib().tm_count_baseline(self.graph._h, self._h, _stream_ptr(stream), ctypes.byref(tot), ctypes.byref(ms)))
        return tot.value, ms.value

    def profile(self, enable=True):
        _check(lib().tm_query_profile(self._h, 1 if enable else 0))

    def last_ms(self):
        """(search kernel ms, fill kernel ms) of the last count / enumerate call."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().tm_query_last_ms(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def inject_fault(self, kind=1):
        """Test hook: make the next count call exercise the bounded-wait timeout path."""
        _check(lib().tm_query_inject_fault(self._h, int(kind)))

    def autotune(self, stream=None) -> dict:
        t = Tuning()
        _check(lib().tm_autotune(self.graph._h, self._h, _stream_ptr(stream), ctypes.byref(t)))
        return t.as_dict()

    def work(self, stream=None) -> dict:
        w = _Work()
        _check(lib().tm_query_work(self.graph._h, self._h, _stream_ptr(stream), ctypes.byref(w)))
        return {"roots": int(w.roots), "nodes": [int(x) for x in w.nodes], "entries": [int(x) for x in w.entries],
                "probe_sectors": int(w.probe_sectors), "matches": int(w.matches)}


@dataclass
class Result:
    status: int
    total: int
    n_written: int
    matches_ptr: int
    k: int
    latency_ms: float


class Server:
    """Continuous-batching request loop over one resident graph (tm_server)."""

    def __init__(self, graph: Graph, handle):
        self.graph = graph
        self._h = handle

    def submit(self, query: Query, enumerate=False, cap=0) -> int:
        t = ctypes.c_uint64()
        _check(lib().tm_serve_submit(self._h, query._h, 1 if enumerate else 0, int(cap), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        r = _Result()
        st = lib().tm_serve_poll(self._h, int(ticket), ctypes.byref(r))
        if st == E_BUSY:
            return None
        _check(st)
        return Result(r.status, r.total, r.n_written, r.matches_dev or 0, r.k, r.submit_to_done_ms)

    def wait(self, ticket, timeout_ms=600_000) -> Result:
        r = _Result()
        _check(lib().tm_serve_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(r)))
        return Result(r.status, r.total, r.n_written, r.matches_dev or 0, r.k, r.submit_to_done_ms)

    def matches(self, res: Result):
        """Copy a finished request's rows (library-owned until release) to a new int32 CUDA
        tensor [n_written, k]."""
        import torch
        dev = f"cuda:{self.graph.device}"
        if not res.n_written:
            return torch.empty((0, res.k), dtype=torch.int32, device=dev)

        class _View:
            __cuda_array_interface__ = {"shape": (res.n_written, res.k), "typestr": "<i4",
                                        "data": (res.matches_ptr, False), "version": 2, "strides": None}
        return torch.as_tensor(_View(), device=dev).clone()

    def release(self, ticket):
        _check(lib().tm_result_release(self._h, int(ticket)))

    def stop(self):
        if getattr(self, "_h", None):
            _check(lib().tm_serve_stop(self._h))
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
