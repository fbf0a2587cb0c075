"""User-defined queries (paper Section 4.3): a JSON document with four sections.

    {
      "pattern":  {"edges": [[0, 1], [1, 2], [2, 3], [3, 0]]},      # motif edges in temporal order
      "in_graph": "path/to/edges.txt",                                # "src dst t [label]" per line
      "constraints": {
        "cg_delta": 3600,                     # coarse-grained window: t_last - t_first <= cg_delta
        "fg_delta": [600, null, 600],         # per consecutive pair: t_{i+1} - t_i <= fg_delta[i]
        "node_labels": {"0": 1, "2": 1},      # motif node -> required label
        "edge_labels": {"1": 7},              # motif edge index -> required label
        "anti_edges": [{"edge": [2, 0], "t": 3, "delta": 60}]
      },
      "runtime_params": {"enumeration": false, "matches": 1000, "gpus": 1}
    }

An anti-edge (Section 2.1) lists its two motif nodes ("edge": [src, dst]),
the motif edge it is attached to and its window.  "t" gives the anti-edge's
1-based temporal order, as in the paper's example ("t:3" follows motif edge 2);
the anti-edge is attached to the motif edge just before that position
(attached edge index = t - 2, 0-based), unless "attach" names the 0-based
motif edge directly.  "delta" is the window length; without it the
anti-edge uses the fine-grained limit that follows its attached edge, else
cg_delta.  Node/edge labels are small integers (uint8).

Host-side parsing only; the search runs in the CUDA library.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

INT64_MAX = np.iinfo(np.int64).max


@dataclass
class ParsedQuery:
    edges: list
    delta: int
    gaps: list
    elabel: list
    nlabel: list
    anti: list = field(default_factory=list)
    in_graph: str | None = None
    enumeration: bool = False
    matches: int = 0
    gpus: int = 1
    name: str = "query"

    @property
    def k(self) -> int:
        return len(self.edges)


class QueryError(ValueError):
    pass


def parse_query(doc) -> ParsedQuery:
    """Parse a query document (JSON text, a path to a .json file, or a dict)."""
    if isinstance(doc, str):
        if os.path.exists(doc):
            base = os.path.dirname(os.path.abspath(doc))
            with open(doc) as f:
                d = json.load(f)
        else:
            base = os.getcwd()
            d = json.loads(doc)
    else:
        base = os.getcwd()
        d = dict(doc)
    pat = d.get("pattern")
    if not isinstance(pat, dict) or "edges" not in pat:
        raise QueryError("'pattern' must hold the motif's 'edges' in temporal order")
    edges = [tuple(int(x) for x in e) for e in pat["edges"]]
    if not edges or any(len(e) != 2 for e in edges):
        raise QueryError("each motif edge is a [source, destination] pair")
    k = len(edges)
    n_nodes = 1 + max(max(e) for e in edges)
    c = d.get("constraints", {}) or {}
    if "cg_delta" not in c:
        raise QueryError("'constraints.cg_delta' (the motif's time window) is required")
    delta = int(c["cg_delta"])
    fg = c.get("fg_delta")
    gaps = [None] * (k - 1)
    if fg is not None:
        if isinstance(fg, (int, float)):
            gaps = [int(fg)] * (k - 1)
        else:
            if len(fg) != k - 1:
                raise QueryError(f"'fg_delta' needs {k - 1} entries (one per consecutive edge pair)")
            gaps = [None if g is None else int(g) for g in fg]
    nlabel = [-1] * n_nodes
    for node, lab in (c.get("node_labels") or {}).items():
        j = int(node)
        if not 0 <= j < n_nodes:
            raise QueryError(f"node label for unknown motif node {node}")
        nlabel[j] = int(lab)
    elabel = [-1] * k
    for edge, lab in (c.get("edge_labels") or {}).items():
        i = int(edge)
        if not 0 <= i < k:
            raise QueryError(f"edge label for unknown motif edge {edge}")
        elabel[i] = int(lab)
    anti = []
    for a in c.get("anti_edges") or []:
        x, y = (int(v) for v in a["edge"])
        if "attach" in a:
            i = int(a["attach"])
        elif "t" in a:
            i = int(a["t"]) - 2
        else:
            raise QueryError("an anti-edge needs 't' (its temporal order) or 'attach'")
        if not 0 <= i < k:
            raise QueryError(f"anti-edge attached to unknown motif edge {i}")
        if "delta" in a:
            w = int(a["delta"])
        elif i < k - 1 and gaps[i] is not None:
            w = gaps[i]
        else:
            w = delta
        anti.append((x, y, i, w))
    rp = d.get("runtime_params", {}) or {}
    in_graph = d.get("in_graph")
    if in_graph is not None and not os.path.isabs(in_graph):
        in_graph = os.path.join(base, in_graph)
    return ParsedQuery(edges, delta, gaps, elabel, nlabel, anti, in_graph,
                       bool(rp.get("enumeration", False)), int(rp.get("matches", 0)), int(rp.get("gpus", 1)),
                       str(d.get("name", "query")))


def load_edge_list(path: str):
    """Text edge list: one edge per line, 'src dst t' or 'src dst t label' ('#' comments)."""
    rows = np.loadtxt(path, dtype=np.int64, comments="#", ndmin=2)
    if rows.shape[1] < 3:
        raise QueryError("edge list lines need 'src dst t'")
    src = rows[:, 0].astype(np.int32)
    dst = rows[:, 1].astype(np.int32)
    t = rows[:, 2].astype(np.int64)
    el = rows[:, 3].astype(np.uint8) if rows.shape[1] > 3 else None
    n = int(max(src.max(initial=-1), dst.max(initial=-1))) + 1
    return n, src, dst, t, el


def run_query(doc, device: int = 0) -> dict:
    """Load the query's graph, run it on the GPU and return the result as a dict."""
    import torch

    from . import Graph
    q = parse_query(doc)
    if q.in_graph is None:
        raise QueryError("'in_graph' (edge list file) is required to run a query")
    n, src, dst, t, el = load_edge_list(q.in_graph)
    g = Graph.load(n, src, dst, t, elabel=el, device=device)
    cq = g.compile(q)
    out = {"name": q.name, "k": q.k, "n_edges": g.n_edges}
    if q.enumeration:
        cap = max(1, q.matches)
        buf = torch.empty((cap, q.k), dtype=torch.int32, device=f"cuda:{device}")
        nw, tot, trunc = cq.enumerate(buf)
        perm = g.edge_perm()
        rows = buf[:nw].cpu().numpy()
        out.update({"count": tot, "truncated": bool(trunc),
                    "matches": [[int(perm[e]) for e in r] for r in rows]})   # input line numbers
    else:
        out["count"] = cq.count()
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="Run a temporal motif query (JSON) on the GPU")
    ap.add_argument("query")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    print(json.dumps(run_query(a.query, a.device)))


if __name__ == "__main__":
    main()
