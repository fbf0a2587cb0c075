"""Major / minor time partitions (Section 5.3.1): pieces searched on their own sum to the whole."""
import numpy as np
import pytest

import oracle
import synth
from paper_2310_02800_gb300.partition import plan_pieces, reach_of, sort_edges


def _graph():
    return synth.powerlaw_graph(3000, 30_000, 23, span=3_000_000.0)


def _tied_graph():
    """Few distinct timestamps: most piece boundaries fall inside a run of tied edges."""
    rng = np.random.default_rng(77)
    n, m = 40, 3000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = ((src + 1 + rng.integers(0, n - 1, m)) % n).astype(np.int32)
    t = (rng.integers(0, 60, m) * 10).astype(np.int64)
    return n, src, dst, t


# The smallest case where a piece needs edges before its first root: edges
# 0->2 and 0->1 tie at t = 10, then 1->2 at t = 20.  The path a->b->c with the
# anti-edge "no a->c within 5 of the first edge" has no match in the whole
# graph (0->2 at t = 10 lies in the closed window [10, 15] of the root 0->1),
# but a piece whose roots start at 0->1 and whose edges start there too would
# count (0->1, 1->2).
TIE_EDGES = (np.array([0, 0, 1], np.int32), np.array([2, 1, 2], np.int32), np.array([10, 10, 20], np.int64))
TIE_MOTIF = synth.Motif([(0, 1), (1, 2)], 100, anti=[(0, 2, 0, 5)])


def _pieces_oracle(n, s, d, t, motif, n_pieces):
    total = 0
    for p in plan_pieces(t, n_pieces, reach_of(motif)):
        sl = slice(p.edge_begin, p.edge_end)
        total += oracle.Graph(n, s[sl], d[sl], t[sl]).count(motif, p.root_begin - p.edge_begin,
                                                            p.root_end - p.edge_begin)
    return total


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


def test_halo_reaches_back_to_time_ties():
    n, src, dst, t = _tied_graph()
    s, d, tt, _ = sort_edges(src, dst, t)
    for n_pieces in (2, 7, 31):
        for p in plan_pieces(tt, n_pieces, 50):
            assert p.edge_begin <= p.root_begin
            assert tt[p.edge_begin] == tt[p.root_begin]
            assert p.edge_begin == 0 or tt[p.edge_begin - 1] < tt[p.root_begin]


def test_anti_edge_tie_at_a_piece_boundary():
    s, d, t = TIE_EDGES
    whole = oracle.Graph(3, s, d, t).count(TIE_MOTIF)
    assert whole == 0
    for n_pieces in (1, 2, 3):
        assert _pieces_oracle(3, s, d, t, TIE_MOTIF, n_pieces) == whole


@pytest.mark.parametrize("motif", [synth.cycle(3, 3600), synth.ping_pong(4, 3600),
                                   synth.Motif([(0, 1), (1, 2), (2, 0)], 3600, anti=[(0, 2, 0, 7200)])])
def test_oracle_on_pieces_sums_to_whole(motif):
    g = _graph()
    s, d, t, _ = sort_edges(g.src, g.dst, g.t)
    whole = oracle.Graph(g.n_nodes, s, d, t).count(motif)
    assert _pieces_oracle(g.n_nodes, s, d, t, motif, 6) == whole and whole > 0


@pytest.mark.parametrize("motif", [synth.Motif([(0, 1), (1, 2)], 100, anti=[(0, 2, 0, 20)]),
                                   synth.Motif([(0, 1), (1, 2), (2, 0)], 200, anti=[(1, 0, 0, 0)])])
def test_oracle_on_tied_pieces_sums_to_whole(motif):
    n, src, dst, t = _tied_graph()
    s, d, tt, _ = sort_edges(src, dst, t)
    whole = oracle.Graph(n, s, d, tt).count(motif)
    assert whole > 0
    for n_pieces in (3, 11, 40):
        assert _pieces_oracle(n, s, d, tt, motif, n_pieces) == whole


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
    s, d, t = TIE_EDGES
    for n_pieces in (1, 2, 3):
        assert count_by_pieces(3, s, d, t, TIE_MOTIF, n_pieces) == 0
    n, src, dst, tt = _tied_graph()
    motif = synth.Motif([(0, 1), (1, 2)], 100, anti=[(0, 2, 0, 20)])
    want = oracle.Graph(n, src, dst, tt).count(motif)
    assert count_by_pieces(n, src, dst, tt, motif, 11) == want
