"""Pins for the CPU oracle (no GPU): brute force, closed forms, invariants, worked example.

Each test checks the oracle against something other than itself, chosen so a
plausible mistake (a dropped bound, a wrong inequality, a missed injectivity
case, a transposed endpoint) fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import pins

HERE = os.path.dirname(os.path.abspath(__file__))
BIG = np.iinfo(np.int64).max


def rand_graph(rng, n_nodes, m, tmax, self_loops=True, labels=0):
    src = rng.integers(0, n_nodes, m).astype(np.int32)
    dst = rng.integers(0, n_nodes, m).astype(np.int32)
    if not self_loops:
        dst = np.where(dst == src, (dst + 1) % n_nodes, dst).astype(np.int32)
    t = rng.integers(0, tmax, m).astype(np.int64)
    el = rng.integers(0, labels, m).astype(np.uint8) if labels else None
    nl = rng.integers(0, labels, n_nodes).astype(np.uint8) if labels else None
    return src, dst, t, el, nl


MOTIFS = [
    [(0, 1)],
    [(0, 1), (1, 0)],
    [(0, 1), (0, 1)],
    [(0, 1), (1, 2)],
    [(0, 1), (0, 2)],
    [(1, 0), (2, 0)],
    [(0, 1), (1, 2), (2, 0)],
    [(0, 1), (1, 0), (0, 1)],
    [(0, 1), (2, 3)],                    # disconnected prefix: all-edges candidate list
    [(0, 1), (2, 0), (1, 2)],
    [(0, 1), (1, 2), (2, 3), (3, 0)],
    [(0, 1), (0, 2), (0, 3)],
    [(0, 1), (1, 0), (0, 1), (1, 0)],
    [(0, 1), (2, 3), (1, 2)],
    [(0, 1), (1, 2), (0, 2)],
]


def oracle_matches(og, edges, delta, gaps=None, elabel=None, nlabel=None):
    q = oracle.make_motif(edges, delta, gaps, elabel, nlabel)
    ms, tot = og.enumerate(q)
    return [tuple(int(x) for x in r) for r in ms], tot


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_small(seed):
    """Matches, counts and per-root counts equal exhaustive search on tiny multigraphs
    with heavy timestamp ties, self-loops, gaps and labels."""
    rng = np.random.default_rng(1000 + seed)
    n_nodes = int(rng.integers(3, 6))
    m = int(rng.integers(10, 19))
    src, dst, t, el, nl = rand_graph(rng, n_nodes, m, tmax=int(rng.integers(4, 30)), labels=2)
    og = oracle.Graph(n_nodes, src, dst, t, el, nl)
    for edges in MOTIFS:
        k = len(edges)
        for delta in (0, 3, 10, 100):
            gaps = [None if rng.random() < 0.5 else int(rng.integers(0, 8)) for _ in range(k - 1)]
            want = pins.brute_force(src, dst, t, edges, delta, gaps)
            got, tot = oracle_matches(og, edges, delta, gaps)
            assert got == want, (edges, delta, gaps)
            assert tot == len(want)
            c, pr = og.count(oracle.make_motif(edges, delta, gaps), per_root=True)
            assert c == len(want) and int(pr.sum()) == c
            roots = np.bincount([w[0] for w in want], minlength=m) if want else np.zeros(m)
            assert np.array_equal(pr.astype(np.int64), roots.astype(np.int64))
        # label constraints: one edge label, one node label
        elab = [-1] * k
        elab[int(rng.integers(0, k))] = int(rng.integers(0, 2))
        n_m = 1 + max(max(e) for e in edges)
        nlab = [-1] * n_m
        nlab[int(rng.integers(0, n_m))] = int(rng.integers(0, 2))
        want = pins.brute_force(src, dst, t, edges, 50, None, elab, nlab, el, nl)
        got, _ = oracle_matches(og, edges, 50, None, elab, nlab)
        assert got == want, ("labels", edges, elab, nlab)


def test_brute_force_four_and_five_edges():
    rng = np.random.default_rng(77)
    src, dst, t, _, _ = rand_graph(rng, 4, 22, tmax=40)
    og = oracle.Graph(4, src, dst, t)
    for edges in ([(0, 1), (1, 2), (2, 3), (3, 0)], [(0, 1), (1, 0), (0, 1), (1, 0)],
                  [(0, 1), (1, 2), (2, 0), (0, 1)], [(0, 1), (1, 2), (2, 3), (3, 1), (1, 0)]):
        for delta in (15, 40):
            want = pins.brute_force(src, dst, t, edges, delta)
            got, _ = oracle_matches(og, edges, delta)
            assert got == want


@pytest.mark.parametrize("seed", range(6))
def test_two_edge_closed_forms(seed):
    """Two-pointer counts over per-pair / per-node time lists, with and without a gap."""
    rng = np.random.default_rng(seed)
    n_nodes = [3, 5, 20, 50, 8, 4][seed]
    m = [200, 400, 2000, 3000, 1000, 600][seed]
    src, dst, t, _, _ = rand_graph(rng, n_nodes, m, tmax=[50, 500, 5000, 20000, 100, 40][seed])
    og = oracle.Graph(n_nodes, src, dst, t)
    for delta, gap in ((0, BIG), (5, BIG), (50, BIG), (50, 7), (1000, 30)):
        want = pins.two_edge_counts(src, dst, t, delta, gap)
        for name, edges in pins.TWO_EDGE_MOTIFS.items():
            got = og.count(oracle.make_motif(edges, delta, [None if gap == BIG else gap]))
            assert got == want[name], (name, delta, gap)


def test_triangle_train():
    for n in (1, 2, 5, 17, 40):
        src, dst, t = pins.triangle_train(n)
        og = oracle.Graph(3, src, dst, t)
        assert og.count(synth.cycle(3, 10 ** 9)) == pins.triangle_train_count(n)


def test_star_burst_large_values():
    for d in (3, 10, 200, 1500):
        src, dst, t = pins.star_burst(d)
        og = oracle.Graph(d + 1, src, dst, t)
        assert og.count(synth.out_star(3, d)) == pins.star_burst_count(d, 3)
        assert og.count(synth.out_star(2, d)) == pins.star_burst_count(d, 2)
    # the window cuts the star: delta = w admits exactly the triples inside w+1 consecutive slots
    d, w = 300, 20
    src, dst, t = pins.star_burst(d)
    og = oracle.Graph(d + 1, src, dst, t)
    want = sum(pins.star_burst_count(min(w, d - i - 1), 2) for i in range(d))
    assert og.count(synth.out_star(3, w)) == want


def test_ping_pong_train():
    """Alternating a->b, b->a at t = 1..n: the 4-edge ping-pong is an ordered pattern subsequence."""
    n = 30
    src = np.array([0 if i % 2 == 0 else 1 for i in range(n)], np.int32)
    dst = 1 - src
    t = np.arange(1, n + 1, dtype=np.int64)
    og = oracle.Graph(2, src, dst, t)
    seq = [int(s) for s in src]
    want = pins.pattern_subsequences(seq, [0, 1, 0, 1]) + pins.pattern_subsequences(seq, [1, 0, 1, 0])
    assert og.count(synth.ping_pong(4, 10 ** 6)) == want


def test_walkthrough_golden():
    spec = json.load(open(os.path.join(HERE, "golden", "walkthrough.json")))
    for case in spec["cases"]:
        e = np.array(case["edges"], np.int64)
        og = oracle.Graph(int(e[:, :2].max()) + 1, e[:, 0].astype(np.int32), e[:, 1].astype(np.int32), e[:, 2])
        anti = [tuple(a) for a in case.get("anti", [])]
        q = oracle.make_motif([tuple(x) for x in case["motif"]], case["delta"], case["gaps"], anti=anti)
        assert og.count(q) == case["expected_count"], case["reason"]
        want = pins.brute_force(e[:, 0], e[:, 1], e[:, 2], [tuple(x) for x in case["motif"]], case["delta"],
                                case["gaps"], anti=anti)
        assert len(want) == case["expected_count"], case["reason"]


def _pl_small(seed=5, m=30000):
    return synth.powerlaw_graph(2000, m, seed, alpha=2.1, span=3_000_000.0, recip_frac=0.1,
                                burst_frac=0.3, burst_mean=200.0)


def test_metamorphic_relations():
    g = _pl_small()
    og = oracle.Graph.from_synth(g)
    qs = [synth.cycle(3, 3600), synth.cycle(4, 3600), synth.out_star(3, 1800), synth.ping_pong(4, 3600),
          synth.path(3, 900)]
    base = {q.name: og.count(q) for q in qs}
    assert any(v > 0 for v in base.values())
    # node relabelling: counts and (edge-id) match lists unchanged
    perm = np.random.default_rng(3).permutation(g.n_nodes).astype(np.int32)
    og_p = oracle.Graph(g.n_nodes, perm[g.src], perm[g.dst], g.t)
    for q in qs:
        assert og_p.count(q) == base[q.name]
    ms1, _ = og.enumerate(qs[0]); ms2, _ = og_p.enumerate(qs[0])
    assert np.array_equal(ms1, ms2)
    # time shift
    og_s = oracle.Graph(g.n_nodes, g.src, g.dst, g.t + 123_457)
    for q in qs:
        assert og_s.count(q) == base[q.name]
    # time reversal with reversed edge directions and reversed motif edge order
    T = int(g.t.max()) + 1
    og_r = oracle.Graph(g.n_nodes, g.dst, g.src, T - g.t)
    for q in qs:
        rev = synth.Motif([(y, x) for (x, y) in reversed(q.edges)], q.delta, list(reversed(q.gaps)))
        assert og_r.count(rev) == base[q.name], q.name
    # delta monotone, gaps equal to delta change nothing
    for q in qs:
        c_small = og.count(synth.Motif(q.edges, q.delta // 2))
        c_big = og.count(synth.Motif(q.edges, q.delta * 2))
        assert c_small <= base[q.name] <= c_big
        assert og.count(synth.Motif(q.edges, q.delta, [q.delta] * (q.k - 1))) == base[q.name]
        tight = og.count(synth.Motif(q.edges, q.delta, [q.delta // 3] * (q.k - 1)))
        assert tight <= base[q.name]


def test_label_partition():
    """Summing a single-edge label constraint over every label value gives the unconstrained count."""
    g = synth.powerlaw_graph(2000, 20000, 9, span=2_000_000.0, n_labels=4)
    og = oracle.Graph.from_synth(g)
    for q in (synth.cycle(3, 5000), synth.path(3, 2000)):
        total = og.count(q)
        for j in range(q.k):
            parts = []
            for L in range(4):
                el = [-1] * q.k; el[j] = L
                parts.append(og.count(synth.Motif(q.edges, q.delta, elabel=el)))
            assert sum(parts) == total
        assert og.count(synth.Motif(q.edges, q.delta, elabel=[-1] * q.k)) == total


def test_per_root_sum_and_ranges():
    g = _pl_small(seed=11, m=20000)
    og = oracle.Graph.from_synth(g)
    for q in (synth.cycle(3, 3600), synth.ping_pong(4, 3600), synth.out_star(3, 3600)):
        tot, pr = og.count(q, per_root=True)
        assert int(pr.sum()) == tot
        # root-range sharding: shards sum to the whole
        cuts = [0, 5000, 5001, 12345, g.n_edges]
        assert sum(og.count(q, a, b) for a, b in zip(cuts[:-1], cuts[1:])) == tot
        assert np.array_equal(og.count(q, 5000, 12345, per_root=True)[1], pr[5000:12345])
        # root-range enumeration: the shards' lists concatenate to the whole list
        rows, _ = og.enumerate(q)
        parts = [og.enumerate(q, root_begin=a, root_end=b)[0] for a, b in zip(cuts[:-1], cuts[1:])]
        assert np.array_equal(np.concatenate(parts), rows)
        assert all(np.all((p[:, 0] >= a) & (p[:, 0] < b)) for p, a, b in zip(parts, cuts[:-1], cuts[1:]))


def test_enumeration_cap_and_order():
    g = _pl_small(seed=13, m=20000)
    og = oracle.Graph.from_synth(g)
    q = synth.ping_pong(3, 7200)
    full, tot = og.enumerate(q)
    assert len(full) == tot > 10
    rows = [tuple(r) for r in full.tolist()]
    assert rows == sorted(rows)                               # lexicographic
    assert all(r[i] < r[i + 1] for r in rows for i in range(len(r) - 1))
    part, tot2 = og.enumerate(q, cap=7)
    assert tot2 == tot and np.array_equal(part, full[:7])


def test_degenerate_inputs():
    og = oracle.Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    assert og.count(synth.cycle(3, 10)) == 0
    # a self-loop never matches a motif edge; k = 1 counts the non-loop edges
    og = oracle.Graph(3, np.array([0, 1, 2], np.int32), np.array([0, 2, 2], np.int32), np.array([1, 2, 3], np.int64))
    assert og.count(synth.Motif([(0, 1)], 0)) == 1
    # equal timestamps never appear in one match
    og = oracle.Graph(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), np.array([5, 5], np.int64))
    assert og.count(synth.path(2, 100)) == 0
    # invalid motifs are rejected
    with pytest.raises(ValueError):
        og.count(oracle.make_motif([(0, 0)], 10))
    with pytest.raises(ValueError):
        og.count(oracle.make_motif([(0, 1)], -1))
    # saturating limits: delta near INT64_MAX with large times
    big = np.array([2 ** 62, 2 ** 62 + 1], np.int64)
    og = oracle.Graph(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32), big)
    assert og.count(synth.path(2, BIG)) == 1
    # eight-edge motif over eight nodes
    k = 7
    src = np.arange(k, dtype=np.int32); dst = np.arange(1, k + 1, dtype=np.int32)
    og = oracle.Graph(k + 1, src, dst, np.arange(k, dtype=np.int64))
    assert og.count(synth.path(7, 100)) == 1
    e8 = [(i, (i + 1) % 8) for i in range(8)]
    src = np.array([a for a, _ in e8], np.int32); dst = np.array([b for _, b in e8], np.int32)
    og = oracle.Graph(8, src, dst, np.arange(8, dtype=np.int64) * 10)
    assert og.count(synth.Motif(e8, 70)) == 1 and og.count(synth.Motif(e8, 69)) == 0


ANTI_CASES = [
    ([(0, 1), (1, 2), (2, 0)], [(0, 2, 0, 5)]),               # no a->c shortly after the first edge
    ([(0, 1), (1, 2), (2, 0)], [(1, 0, 1, 8), (2, 1, 2, 3)]),  # two anti-edges on later edges
    ([(0, 1), (1, 0)], [(0, 1, 0, 6)]),                         # anti-edge on the attached edge's own pair
    ([(0, 1), (0, 2), (0, 3)], [(1, 2, 2, 10)]),                # between two leaves, on the last edge
    ([(0, 1), (1, 2)], [(2, 0, 0, 0)]),                         # zero-length window (ties only)
]


@pytest.mark.parametrize("seed", range(8))
def test_anti_edges_brute_force(seed):
    """Temporal anti-edges (Section 2.1): the oracle equals exhaustive search on tiny multigraphs."""
    rng = np.random.default_rng(500 + seed)
    n_nodes = int(rng.integers(3, 6))
    m = int(rng.integers(10, 17))
    src, dst, t, _, _ = rand_graph(rng, n_nodes, m, tmax=int(rng.integers(5, 25)))
    og = oracle.Graph(n_nodes, src, dst, t)
    for edges, anti in ANTI_CASES:
        for delta in (4, 30):
            want = pins.brute_force(src, dst, t, edges, delta, anti=anti)
            q = oracle.make_motif(edges, delta, anti=anti)
            rows, tot = og.enumerate(q)
            assert [tuple(int(x) for x in r) for r in rows] == want, (edges, anti, delta)
            assert og.count(q) == len(want)
            assert og.count(q) <= og.count(oracle.make_motif(edges, delta))


def test_anti_edge_monotone_and_vacuous():
    g = _pl_small(seed=17, m=20000)
    og = oracle.Graph.from_synth(g)
    edges = [(0, 1), (1, 2), (2, 0)]
    base = og.count(oracle.make_motif(edges, 3600))
    counts = [og.count(oracle.make_motif(edges, 3600, anti=[(0, 2, 0, d)])) for d in (0, 60, 600, 3600)]
    assert counts == sorted(counts, reverse=True) and counts[0] <= base
    # an anti-edge between the endpoints of its own edge never counts that edge itself
    q = oracle.make_motif([(0, 1), (1, 2)], 3600, anti=[(0, 1, 0, 0)])
    p = oracle.make_motif([(0, 1), (1, 2)], 3600)
    assert og.count(q) <= og.count(p)



@pytest.mark.parametrize("seed", range(8))
def test_work_counters_brute_force(seed):
    """The oracle's work counters (the roofline numerator) against the search tree computed
    from its definition: per level, the valid prefixes and the entries of their candidate
    windows; the binary-search probes within the bounds of a search over each located list."""
    rng = np.random.default_rng(7000 + seed)
    n_nodes = int(rng.integers(3, 7))
    m = int(rng.integers(12, 22))
    labels = 2 if seed % 2 else 0
    src, dst, t, el, nl = rand_graph(rng, n_nodes, m, tmax=int(rng.integers(5, 40)), labels=labels)
    og = oracle.Graph(n_nodes, src, dst, t, el, nl)
    for edges in MOTIFS:
        k = len(edges)
        for delta in (2, 9, 1000):
            gaps = [None if rng.random() < 0.6 else int(rng.integers(0, 12)) for _ in range(k - 1)]
            elab = nlab = None
            if labels:
                elab = [-1] * k
                elab[int(rng.integers(0, k))] = int(rng.integers(0, 2))
                nlab = [-1] * 8
                nlab[int(rng.integers(0, 1 + max(max(e) for e in edges)))] = int(rng.integers(0, 2))
            q = oracle.make_motif(edges, delta, gaps, elab, nlab)
            r0, r1 = (0, m) if delta != 9 else (m // 3, m - 2)
            total, w = og.count(q, r0, r1, work=True)
            nodes, entries, lengths = pins.search_work(src, dst, t, edges, delta, gaps, elab, nlab, el, nl,
                                                       roots=(r0, r1))
            assert w["roots"] == r1 - r0
            assert w["nodes"] == nodes, (edges, delta, gaps)
            assert w["entries"] == entries, (edges, delta, gaps)
            lo = sum(int(np.floor(np.log2(L))) for L in lengths if L > 0)
            hi = sum(int(np.ceil(np.log2(L + 1))) for L in lengths)
            assert lo <= w["probes"] <= hi, (edges, delta, w["probes"], lo, hi)
            assert w["matches"] == total
