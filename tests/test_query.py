"""JSON query front end (paper Section 4.3): parsing on the CPU, one end-to-end run on the GPU."""
import json

import numpy as np
import pytest

import oracle
from paper_2310_02800_gb300.query import QueryError, load_edge_list, parse_query

DOC = {
    "pattern": {"edges": [[0, 1], [1, 2], [2, 3], [3, 0]]},
    "in_graph": "edges.txt",
    "constraints": {"cg_delta": 3600, "fg_delta": [600, None, 900],
                    "node_labels": {"0": 1, "2": 1}, "edge_labels": {"1": 7},
                    "anti_edges": [{"edge": [2, 0], "t": 3}]},
    "runtime_params": {"enumeration": True, "matches": 50, "gpus": 1},
}


def test_parse_full_document():
    q = parse_query(DOC)
    assert q.edges == [(0, 1), (1, 2), (2, 3), (3, 0)]
    assert q.delta == 3600 and q.gaps == [600, None, 900]
    assert q.nlabel == [1, -1, 1, -1] and q.elabel == [-1, 7, -1, -1]
    # "t:3" follows motif edge 2 (1-based) -> attached to edge index 1; window = fg limit after it
    assert q.anti == [(2, 0, 1, 3600)]
    assert q.enumeration and q.matches == 50 and q.gpus == 1


def test_parse_defaults_and_json_text():
    q = parse_query(json.dumps({"pattern": {"edges": [[0, 1], [1, 0]]}, "constraints": {"cg_delta": 10,
                                "fg_delta": 4, "anti_edges": [{"edge": [1, 0], "attach": 0, "delta": 2}]}}))
    assert q.gaps == [4] and q.anti == [(1, 0, 0, 2)] and not q.enumeration


@pytest.mark.parametrize("bad", [
    {"constraints": {"cg_delta": 1}},
    {"pattern": {"edges": [[0, 1]]}},
    {"pattern": {"edges": [[0, 1], [1, 2]]}, "constraints": {"cg_delta": 5, "fg_delta": [1, 2]}},
    {"pattern": {"edges": [[0, 1]]}, "constraints": {"cg_delta": 5, "node_labels": {"7": 1}}},
    {"pattern": {"edges": [[0, 1]]}, "constraints": {"cg_delta": 5, "anti_edges": [{"edge": [1, 0]}]}},
])
def test_parse_errors(bad):
    with pytest.raises(QueryError):
        parse_query(bad)


def test_edge_list_loader(tmp_path):
    p = tmp_path / "e.txt"
    p.write_text("# src dst t\n0 1 10\n3 0 120\n0 2 130\n")
    n, s, d, t, el = load_edge_list(str(p))
    assert n == 4 and list(s) == [0, 3, 0] and list(t) == [10, 120, 130] and el is None


@pytest.mark.gpu
def test_run_query_end_to_end(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_02800_gb300.query import run_query
    rng = np.random.default_rng(3)
    m, n = 3000, 30
    src = rng.integers(0, n, m); dst = rng.integers(0, n, m); t = rng.integers(0, 20_000, m)
    np.savetxt(tmp_path / "edges.txt", np.stack([src, dst, t], 1), fmt="%d")
    doc = {"pattern": {"edges": [[0, 1], [1, 2], [2, 0]]}, "in_graph": "edges.txt",
           "constraints": {"cg_delta": 400, "anti_edges": [{"edge": [0, 2], "attach": 0, "delta": 100}]},
           "runtime_params": {"enumeration": True, "matches": 100000}}
    path = tmp_path / "q.json"
    path.write_text(json.dumps(doc))
    res = run_query(str(path))
    og = oracle.Graph(n, src.astype(np.int32), dst.astype(np.int32), t.astype(np.int64))
    q = oracle.make_motif([(0, 1), (1, 2), (2, 0)], 400, anti=[(0, 2, 0, 100)])
    rows, tot = og.enumerate(q)
    perm = og.sorted_edges()[3]
    assert res["count"] == tot
    assert res["matches"] == [[int(perm[e]) for e in r] for r in rows.tolist()]
