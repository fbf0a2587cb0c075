"""CPU oracle for temporal motif mining -- TEST INFRASTRUCTURE ONLY.

Plain single-threaded C (oracle.c) following the paper's problem definition
(Section 2.1) and the chronological DFS of Algorithm 1.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may use
it.  It shares no code with the CUDA library; both take their inputs from the
seeded generators in synth/.

Every function is pinned by tests/test_oracle_pins.py against brute force,
closed forms, invariants and the paper's worked-example fragments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None
MAX_EDGES = 8
MAX_NODES = 8
MAX_ANTI = 4
INT64_MAX = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


class Motif(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("esrc", ctypes.c_uint8 * MAX_EDGES), ("edst", ctypes.c_uint8 * MAX_EDGES),
                ("delta", ctypes.c_int64), ("gap", ctypes.c_int64 * (MAX_EDGES - 1)),
                ("elabel", ctypes.c_int16 * MAX_EDGES), ("nlabel", ctypes.c_int16 * MAX_NODES),
                ("n_anti", ctypes.c_int32), ("anti_src", ctypes.c_uint8 * MAX_ANTI),
                ("anti_dst", ctypes.c_uint8 * MAX_ANTI), ("anti_edge", ctypes.c_uint8 * MAX_ANTI),
                ("anti_delta", ctypes.c_int64 * MAX_ANTI)]


class Work(ctypes.Structure):
    _fields_ = [("roots", ctypes.c_uint64), ("nodes", ctypes.c_uint64 * MAX_EDGES),
                ("entries", ctypes.c_uint64 * MAX_EDGES), ("probes", ctypes.c_uint64),
                ("matches", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {"roots": int(self.roots), "nodes": [int(x) for x in self.nodes],
                "entries": [int(x) for x in self.entries], "probes": int(self.probes),
                "matches": int(self.matches)}


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        p = ctypes.c_void_p
        lib.or_graph_build.restype = p
        lib.or_graph_build.argtypes = [ctypes.c_int64, ctypes.c_int64, p, p, p, p, p]
        lib.or_graph_free.argtypes = [p]
        lib.or_graph_free.restype = None
        lib.or_graph_edges.argtypes = [p]
        lib.or_graph_edges.restype = ctypes.c_int64
        lib.or_graph_sorted.argtypes = [p, p, p, p, p]
        lib.or_graph_sorted.restype = None
        lib.or_count.argtypes = [p, ctypes.POINTER(Motif), ctypes.c_int64, ctypes.c_int64, p, p,
                                 ctypes.POINTER(Work)]
        lib.or_enumerate.argtypes = [p, ctypes.POINTER(Motif), p, ctypes.c_uint64, p, p]
        lib.or_enumerate_roots.argtypes = [p, ctypes.POINTER(Motif), ctypes.c_int64, ctypes.c_int64, p,
                                           ctypes.c_uint64, p, p]
        _lib = lib
    return _lib


def make_motif(edges, delta, gaps=None, elabel=None, nlabel=None, n_nodes=None, anti=None) -> Motif:
    """Oracle motif struct from plain lists (gaps: k-1 values, None/INT64_MAX = none;
    anti: list of (src node, dst node, attached edge index, delta))."""
    k = len(edges)
    q = Motif()
    q.k = k
    q.n_nodes = n_nodes if n_nodes is not None else (1 + max(max(e) for e in edges))
    for i, (x, y) in enumerate(edges):
        q.esrc[i] = x; q.edst[i] = y
    q.delta = int(delta)
    for i in range(MAX_EDGES - 1):
        g = None if gaps is None or i >= len(gaps) else gaps[i]
        q.gap[i] = INT64_MAX if g is None else int(g)
    for i in range(MAX_EDGES):
        q.elabel[i] = -1 if elabel is None or i >= len(elabel) else int(elabel[i])
    for i in range(MAX_NODES):
        q.nlabel[i] = -1 if nlabel is None or i >= len(nlabel) else int(nlabel[i])
    anti = anti or []
    q.n_anti = len(anti)
    for a, (x, y, e, d) in enumerate(anti):
        q.anti_src[a] = x; q.anti_dst[a] = y; q.anti_edge[a] = e; q.anti_delta[a] = int(d)
    return q


def motif_from(m) -> Motif:
    """Oracle motif struct from a synth.Motif-like object."""
    return make_motif(m.edges, m.delta, m.gaps, m.elabel, m.nlabel, anti=getattr(m, "anti", None))


class Graph:
    """Oracle-side graph: stable (t, input index) ordering plus per-node edge-id lists."""

    def __init__(self, n_nodes, src, dst, t, elabel=None, nlabel=None):
        lib = _load()
        self._keep = [np.ascontiguousarray(src, np.int32), np.ascontiguousarray(dst, np.int32),
                      np.ascontiguousarray(t, np.int64)]
        el = None if elabel is None else np.ascontiguousarray(elabel, np.uint8)
        nl = None if nlabel is None else np.ascontiguousarray(nlabel, np.uint8)
        self._keep += [el, nl]
        m = self._keep[0].shape[0]
        self.n_nodes, self.m = int(n_nodes), int(m)
        self._h = lib.or_graph_build(self.n_nodes, self.m, self._keep[0].ctypes.data,
                                     self._keep[1].ctypes.data, self._keep[2].ctypes.data,
                                     None if el is None else el.ctypes.data,
                                     None if nl is None else nl.ctypes.data)
        if not self._h:
            raise ValueError("oracle: invalid graph (endpoint out of range or negative time)")

    @classmethod
    def from_synth(cls, g):
        return cls(g.n_nodes, g.src, g.dst, g.t, g.elabel, g.nlabel)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_graph_free(self._h)
            self._h = None

    def sorted_edges(self):
        """(src, dst, t, perm) in edge-id order; perm maps edge id -> input index."""
        s = np.empty(self.m, np.int32); d = np.empty(self.m, np.int32)
        t = np.empty(self.m, np.int64); p = np.empty(self.m, np.int64)
        _load().or_graph_sorted(self._h, s.ctypes.data, d.ctypes.data, t.ctypes.data, p.ctypes.data)
        return s, d, t, p

    def count(self, motif, root_begin=0, root_end=None, per_root=False, work=False):
        q = motif if isinstance(motif, Motif) else motif_from(motif)
        r1 = self.m if root_end is None else int(root_end)
        tot = ctypes.c_uint64(0)
        pr = np.zeros(max(0, r1 - root_begin), np.uint64) if per_root else None
        w = Work()
        rc = _load().or_count(self._h, ctypes.byref(q), int(root_begin), r1, ctypes.addressof(tot),
                              None if pr is None else pr.ctypes.data, ctypes.byref(w))
        if rc != 0:
            raise ValueError("oracle: invalid motif")
        out = [int(tot.value)]
        if per_root:
            out.append(pr)
        if work:
            out.append(w.as_dict())
        return out[0] if len(out) == 1 else tuple(out)

    def enumerate(self, motif, cap=None, root_begin=None, root_end=None):
        """(matches int32[n_written, k], total) -- lexicographically first cap matches, of the
        whole graph or of the roots in [root_begin, root_end)."""
        q = motif if isinstance(motif, Motif) else motif_from(motif)
        ranged = root_begin is not None or root_end is not None
        r0 = 0 if root_begin is None else int(root_begin)
        r1 = self.m if root_end is None else int(root_end)
        if cap is None:
            cap = self.count(q, r0, r1)
        out = np.zeros((max(int(cap), 1), q.k), np.int32)
        nw = ctypes.c_uint64(0); tot = ctypes.c_uint64(0)
        if ranged:
            rc = _load().or_enumerate_roots(self._h, ctypes.byref(q), r0, r1, out.ctypes.data, int(cap),
                                            ctypes.addressof(nw), ctypes.addressof(tot))
        else:
            rc = _load().or_enumerate(self._h, ctypes.byref(q), out.ctypes.data, int(cap),
                                      ctypes.addressof(nw), ctypes.addressof(tot))
        if rc != 0:
            raise ValueError("oracle: invalid motif")
        return out[: int(nw.value)], int(tot.value)
