"""Seeded synthetic workloads: temporal graphs, motif queries, arrival traces.

This module only draws random inputs; it holds none of the motif-mining
arithmetic.  The CPU oracle and the CUDA library both consume what it returns
(numpy arrays in input order, not sorted unless a recipe says so).

Graph shapes stand in for the paper's evaluation graphs (Section 6, Table 1:
power-law social and transaction graphs with second-resolution timestamps);
the datasets themselves are not used.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

SEED_BASE = 0x7E4D0000


def build(force: bool = False) -> str:
    """Compile the C generator in place (gcc, -O2, pthreads)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, u64, dbl, ptr, cint = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_void_p, ctypes.c_int)
        lib.synth_uniform.argtypes = [u64, i64, i64, i64, ptr, ptr, ptr, cint]
        lib.synth_powerlaw.argtypes = [u64, i64, i64, dbl, dbl, dbl, dbl, dbl, dbl, dbl, i64,
                                       cint, cint, ptr, ptr, ptr, ptr, cint]
        lib.synth_labels.argtypes = [u64, u64, i64, cint, ptr, cint]
        lib.synth_draws.argtypes = [u64, u64, i64, ptr]
        lib.synth_draws.restype = None
        _lib = lib
    return _lib


def _nthreads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


@dataclass
class TemporalGraph:
    """Edges in input order: src, dst (int32), t (int64), optional uint8 labels."""
    n_nodes: int
    src: np.ndarray
    dst: np.ndarray
    t: np.ndarray
    elabel: np.ndarray | None = None
    nlabel: np.ndarray | None = None
    name: str = ""

    @property
    def n_edges(self) -> int:
        return int(self.src.shape[0])

    def sorted_copy(self) -> "TemporalGraph":
        """Stable sort by timestamp (ties keep input order)."""
        o = np.argsort(self.t, kind="stable")
        return TemporalGraph(self.n_nodes, self.src[o].copy(), self.dst[o].copy(), self.t[o].copy(),
                             None if self.elabel is None else self.elabel[o].copy(),
                             self.nlabel, self.name)


def draws(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    if n:
        _load().synth_draws(seed, stream, n, out.ctypes.data)
    return out


def uniform_graph(n: int, m: int, tmax: int, seed: int, sort: bool = True) -> TemporalGraph:
    """src/dst uniform (no self-loops), t uniform in [0, tmax)."""
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); t = np.empty(m, np.int64)
    rc = _load().synth_uniform(seed, n, m, tmax, src.ctypes.data, dst.ctypes.data, t.ctypes.data, _nthreads())
    assert rc == 0
    g = TemporalGraph(n, src, dst, t, name=f"uniform_n{n}_m{m}")
    return g.sorted_copy() if sort else g


def powerlaw_graph(n: int, m: int, seed: int, alpha: float = 2.1, span: float = 94_608_000.0,
                   amp: float = 0.8, recip_frac: float = 0.10, burst_frac: float = 0.3,
                   burst_mean: float = 300.0, hub_share: float = 0.0, n_hubs: int = 0,
                   n_labels: int = 0, pa: bool = True) -> TemporalGraph:
    """Bursty power-law temporal graph (input order, unsorted).  pa: destinations by
    preferential attachment (copy model); else drawn from the same popularity as sources."""
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); t = np.empty(m, np.int64)
    el = np.empty(m, np.uint8) if n_labels > 0 else None
    rc = _load().synth_powerlaw(seed, n, m, alpha, span, amp, recip_frac, burst_frac, burst_mean,
                                hub_share, n_hubs, n_labels, 1 if pa else 0, src.ctypes.data, dst.ctypes.data,
                                t.ctypes.data, None if el is None else el.ctypes.data, _nthreads())
    assert rc == 0
    return TemporalGraph(n, src, dst, t, el, None, f"powerlaw_n{n}_m{m}_a{alpha}")


def node_labels(n: int, n_labels: int, seed: int, stream: int = 7) -> np.ndarray:
    out = np.empty(n, np.uint8)
    rc = _load().synth_labels(seed, stream, n, n_labels, out.ctypes.data, _nthreads())
    assert rc == 0
    return out


# ------------------------------------------------------------ named workloads

def tiny_uniform(seed: int = SEED_BASE + 1) -> TemporalGraph:
    """1,000 nodes, 20,000 edges, uniform endpoints, t uniform in [0, 1e6), sorted."""
    g = uniform_graph(1000, 20_000, 1_000_000, seed, sort=True)
    g.name = "tiny_uniform_1k_20k"
    return g


def powerlaw_10m(seed: int = SEED_BASE + 2, scale: float = 1.0) -> TemporalGraph:
    """1M nodes, 10M edges, Zipf 2.1, 3-year bursty daily-modulated times, 10% reciprocated."""
    n = max(16, int(1_000_000 * scale)); m = max(16, int(10_000_000 * scale))
    g = powerlaw_graph(n, m, seed, alpha=2.1, span=94_608_000.0)
    g.name = f"powerlaw_{n}n_{m}e"
    return g


def hub_skewed_100m(seed: int = SEED_BASE + 3, scale: float = 1.0) -> TemporalGraph:
    """10M nodes, 100M edges, Zipf 1.8, top 0.01% nodes own 20% of endpoints, 16 edge labels, 30 days.
    Both endpoints follow the same popularity, so hubs send as much as they receive."""
    n = max(16, int(10_000_000 * scale)); m = max(16, int(100_000_000 * scale))
    g = powerlaw_graph(n, m, seed, alpha=1.8, span=30 * 86_400.0, recip_frac=0.0, burst_frac=0.0,
                       hub_share=0.2, n_hubs=max(1, n // 10_000), n_labels=16, pa=False)
    g.name = f"hubskew_{n}n_{m}e"
    return g


def powerlaw_1b(seed: int = SEED_BASE + 5, scale: float = 1.0) -> TemporalGraph:
    """100M nodes, 1B edges, Zipf 2.1 popularity on both endpoints, same time process as
    powerlaw_10m.  No copy model for destinations: at 1e9 edges preferential attachment puts
    about 15% of all edges on one node."""
    n = max(16, int(100_000_000 * scale)); m = max(16, int(1_000_000_000 * scale))
    g = powerlaw_graph(n, m, seed, alpha=2.1, span=94_608_000.0, pa=False)
    g.name = f"powerlaw_{n}n_{m}e"
    return g


def time_windows(t: np.ndarray, n_windows: int, frac: float, seed: int, stream: int = 801) -> list:
    """Seeded root samples of a graph given in input order: n_windows disjoint time windows
    [T0, T1) that together hold about frac of all edges.  Because edge ids rank edges by
    (t, input index), the edges of one window are one contiguous id range [a, b) with
    a = #{t < T0} and b = #{t < T1}; returns (T0, T1, a, b) per window."""
    m = int(t.shape[0])
    tmin, tmax = int(t.min()), int(t.max()) + 1
    per = max(1, int(m * frac / n_windows))
    width = max(1, int((tmax - tmin) * per / m))
    slots = max(1, (tmax - tmin) // width)
    picks = sorted(set(int(x % slots) for x in draws(seed, stream, 4 * n_windows)))[:n_windows]
    # edges per width-wide time slot, in one pass over the times (chunked to bound memory)
    per_slot = np.zeros(slots + 1, np.int64)
    for c in range(0, m, 1 << 26):
        b = np.minimum((t[c:c + (1 << 26)] - tmin) // width, slots)
        per_slot += np.bincount(b, minlength=slots + 1)
    before = np.concatenate([[0], np.cumsum(per_slot)])
    return [(tmin + p * width, tmin + (p + 1) * width, int(before[p]), int(before[p + 1])) for p in picks]



# ------------------------------------------------------------------ motifs

NONE = np.iinfo(np.int64).max  # "no limit" for a per-gap bound


@dataclass
class Motif:
    """k motif edges (x_i -> y_i) in temporal order over nodes 0..n_nodes-1."""
    edges: list
    delta: int
    gaps: list = field(default_factory=list)      # k-1 entries, NONE = unconstrained
    elabel: list = field(default_factory=list)    # k entries, -1 = any
    nlabel: list = field(default_factory=list)    # n_nodes entries, -1 = any
    name: str = ""
    anti: list = field(default_factory=list)      # (src node, dst node, attached edge, delta) per anti-edge

    def __post_init__(self):
        k = len(self.edges)
        if not self.gaps:
            self.gaps = [NONE] * max(0, k - 1)
        if not self.elabel:
            self.elabel = [-1] * k
        if not self.nlabel:
            self.nlabel = [-1] * self.n_nodes

    @property
    def k(self) -> int:
        return len(self.edges)

    @property
    def n_nodes(self) -> int:
        return 1 + max(max(e) for e in self.edges) if self.edges else 0


def cycle(k: int, delta: int) -> Motif:
    return Motif([(i, (i + 1) % k) for i in range(k)], delta, name=f"cycle{k}")


def out_star(k: int, delta: int) -> Motif:
    return Motif([(0, i) for i in range(1, k + 1)], delta, name=f"outstar{k}")


def in_star(k: int, delta: int) -> Motif:
    return Motif([(i, 0) for i in range(1, k + 1)], delta, name=f"instar{k}")


def path(k: int, delta: int) -> Motif:
    return Motif([(i, i + 1) for i in range(k)], delta, name=f"path{k}")


def ping_pong(k: int, delta: int) -> Motif:
    return Motif([(0, 1) if i % 2 == 0 else (1, 0) for i in range(k)], delta, name=f"pingpong{k}")


def chorded_four_cycle(delta: int) -> Motif:
    """6 edges over 4 nodes: temporal 4-cycle a->b->c->d->a, then chords a->c, b->d."""
    return Motif([(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (1, 3)], delta, name="cycle4_chords")


FAMILIES = {"cycle": cycle, "outstar": out_star, "instar": in_star, "path": path, "pingpong": ping_pong}

# Families of the batched / served query mixes.  "Stars" are out-stars, the star
# form of the power-law query set; in-stars on the copy-model in-hub (about 17%
# of all edges) reach more than 1e15 matches at k >= 4 and day-long delta.
MIX_FAMILIES = ("cycle", "outstar", "path", "pingpong")


def powerlaw_queries(delta: int = 3600) -> list:
    """The four queries on the 10M-edge power-law graph."""
    return [cycle(3, delta), cycle(4, delta), out_star(3, delta), ping_pong(4, delta)]


def constraint_sweep_queries(seed: int = SEED_BASE + 6, delta: int = 3600, n_labels: int = 2) -> list:
    """Temporal 4-cycle under added constraints (a synthetic analogue of the paper's Table 4):
    N none; V node labels on all four nodes (constants drawn from the seed); V+T also every
    consecutive gap <= delta / 2; V+T+A also an anti-edge: no b -> a reply within delta / 4 of
    the first edge a -> b."""
    lab = [int(x % n_labels) for x in draws(seed, 401, 4)]
    n = cycle(4, delta); n.name = "cycle4_N"
    v = cycle(4, delta); v.nlabel = lab; v.name = "cycle4_V"
    vt = cycle(4, delta); vt.nlabel = lab; vt.gaps = [delta // 2] * 3; vt.name = "cycle4_V+T"
    vta = cycle(4, delta); vta.nlabel = lab; vta.gaps = [delta // 2] * 3
    vta.anti = [(1, 0, 0, delta // 4)]; vta.name = "cycle4_V+T+A"
    return [n, v, vt, vta]


def hub_skewed_queries(seed: int = SEED_BASE + 3, delta: int = 7200) -> list:
    """5-edge temporal path with per-edge label constants and gaps <= 600 s; chorded 4-cycle."""
    d = draws(seed, 301, 5)
    p = path(5, delta)
    p.gaps = [600] * 4
    p.elabel = [int(x % 16) for x in d]
    p.name = "path5_labels_gap600"
    return [p, chorded_four_cycle(delta)]


def query_mix(n: int = 64, seed: int = SEED_BASE + 4, kmin: int = 2, kmax: int = 6,
              dmin: float = 60.0, dmax: float = 86_400.0) -> list:
    """Family uniform over MIX_FAMILIES, k uniform in [kmin, kmax], delta log-uniform."""
    fam = list(MIX_FAMILIES)
    a = draws(seed, 401, n); b = draws(seed, 402, n); c = draws(seed, 403, n)
    out = []
    for i in range(n):
        f = fam[int(a[i] % len(fam))]
        k = kmin + int(b[i] % (kmax - kmin + 1))
        u = float(c[i] >> np.uint64(11)) / 9007199254740992.0
        delta = int(round(math.exp(math.log(dmin) + u * (math.log(dmax) - math.log(dmin)))))
        q = FAMILIES[f](k, delta)
        q.name = f"{f}{k}_d{delta}"
        out.append(q)
    return out


def arrival_trace(rate_qps: float, n: int, seed: int, stream: int = 501) -> np.ndarray:
    """Poisson arrivals: cumulative exponential gaps (seconds) at rate_qps."""
    d = draws(seed, stream, n)
    u = (d >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
    return np.cumsum(-np.log1p(-u) / rate_qps)
