"""Major / minor time partitions (Section 5.3.1): pieces searched on their own sum to the whole."""
import numpy as np
import pytest

import oracle
import synth
from paper_2310_02800_gb300.partition import plan_pieces, reach_of, sort_edges


def _graph():
    return synth.powerlaw_graph(3000, 30_000, 23, span=3_000_000.0)


def test_pieces_cover_roots_once():
    g = _graph()
    _, _, t, _ = sort_edges(g.src, g.dst, g.t)
    for n in (1, 2, 5, 17):
        ps = plan_pieces(t, n, 3600)
        assert ps[0].root_begin == 0 and ps[-1].root_end == g.n_edges
        assert all(a.root_end == b.root_begin for a, b in zip(ps[:-1], ps[1:]))
        for p in ps:
            assert p.edge_end >= p.root_end
            assert p.edge_end == g.n_edges or t[p.edge_end] > t[p.root_end - 1] + 3600


@pytest.mark.parametrize("motif", [synth.cycle(3, 3600), synth.ping_pong(4, 3600),
                                   synth.Motif([(0, 1), (1, 2), (2, 0)], 3600, anti=[(0, 2, 0, 7200)])])
def test_oracle_on_pieces_sums_to_whole(motif):
    g = _graph()
    s, d, t, _ = sort_edges(g.src, g.dst, g.t)
    whole = oracle.Graph(g.n_nodes, s, d, t).count(motif)
    total = 0
    for p in plan_pieces(t, 6, reach_of(motif)):
        sl = slice(p.root_begin, p.edge_end)
        total += oracle.Graph(g.n_nodes, s[sl], d[sl], t[sl]).count(motif, 0, p.root_end - p.root_begin)
    assert total == whole and whole > 0


@pytest.mark.gpu
def test_gpu_pieces_equal_whole():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_02800_gb300.partition import count_by_pieces
    g = _graph()
    og = oracle.Graph.from_synth(g)
    for motif in (synth.cycle(4, 3600), synth.out_star(3, 3600)):
        assert count_by_pieces(g.n_nodes, g.src, g.dst, g.t, motif, 7) == og.count(motif)
