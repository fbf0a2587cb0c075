"""Time-range partitions of the root space (paper Section 5.3.1, major and
minor edge-list partitions), used to mine a graph piece by piece.

Edges are in time order (edge id = rank by (t, input index)).  A major
partition is a contiguous range of root edges [root_begin, root_end).  Every
match rooted there uses only edges with times in [t(root_begin),
t(root_end - 1) + reach], where reach = delta plus the longest anti-edge
window, so the partition's minor (halo) range [edge_begin, edge_end) holds all
it needs: it reaches forward to the last edge inside that time, and backward
to the first edge whose time equals t(root_begin).  The backward part matters
for anti-edges only: an anti-edge attached to motif edge 0 has the closed
window [t(e_0), t(e_0) + delta'], which contains edges that tie with the root
in time but precede it in id order, and those can sit before root_begin.  Each piece can be
loaded, searched for its own roots and freed on its own: on one GPU this mines
graphs larger than device memory piece by piece; across GPUs each piece is one
GPU's work, with no exchange but the final sum.

Host logic only; the search runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Piece:
    root_begin: int   # first root edge id (global)
    root_end: int     # one past the last root
    edge_end: int     # one past the last edge the piece's matches can use
    edge_begin: int   # first edge the piece's matches can use: the first edge tied in time with root_begin


def reach_of(motif) -> int:
    """Time reach of a match beyond its root: delta plus the longest anti-edge window."""
    anti = getattr(motif, "anti", None) or []
    return int(motif.delta) + max([int(a[3]) for a in anti], default=0)


def plan_pieces(t_sorted: np.ndarray, n_pieces: int, reach: int) -> list:
    """Split roots [0, m) into n_pieces contiguous major partitions with their halos."""
    m = int(t_sorted.shape[0])
    if n_pieces < 1:
        raise ValueError("n_pieces >= 1")
    cuts = [m * p // n_pieces for p in range(n_pieces + 1)]
    out = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b <= a:
            continue
        last_t = int(t_sorted[b - 1])
        lim = last_t + reach if last_t <= np.iinfo(np.int64).max - reach else np.iinfo(np.int64).max
        e = int(np.searchsorted(t_sorted, lim, side="right"))
        lo = int(np.searchsorted(t_sorted, int(t_sorted[a]), side="left"))
        out.append(Piece(a, b, max(e, b), lo))
    return out


def sort_edges(src, dst, t, elabel=None):
    """Stable time order of an input edge list (edge ids of the library)."""
    o = np.argsort(np.asarray(t), kind="stable")
    el = None if elabel is None else np.asarray(elabel)[o]
    return np.asarray(src)[o], np.asarray(dst)[o], np.asarray(t)[o], el


def count_by_pieces(n_nodes, src, dst, t, motif, n_pieces, elabel=None, nlabel=None, device=0):
    """Exact count, loading one piece at a time onto the GPU (peak memory ~ one piece)."""
    from . import Graph
    s, d, tt, el = sort_edges(src, dst, t, elabel)
    total = 0
    for pc in plan_pieces(tt, n_pieces, reach_of(motif)):
        sl = slice(pc.edge_begin, pc.edge_end)
        g = Graph.load(n_nodes, s[sl], d[sl], tt[sl], None if el is None else el[sl], nlabel, device=device)
        q = g.compile(motif)
        # the slice keeps the global (t, id) order, so local id = global id - edge_begin
        total += q.count_roots(pc.root_begin - pc.edge_begin, pc.root_end - pc.edge_begin)
        q.free()
        g.free()
    return total
