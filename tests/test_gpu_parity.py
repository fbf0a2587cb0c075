"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Counts are uint64 and match lists int32 edge ids: the bar is bit-exact
equality everywhere (no floating point on this path).  Inputs are seeded
synthetic graphs from synth/ with the shapes of the benchmark workloads, at
sizes the oracle finishes in seconds, plus the full-size tiny-uniform
workload and sampled root ranges of the 10M-edge power-law workload.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_02800_gb300 as m
    m.lib()
    return m


def pr_tensor(m):
    return torch.zeros(max(m, 1), dtype=torch.int64, device="cuda")


def check_query(tmg, gg, og, motif, per_root=True, enum_cap=None, ranges=None):
    """Count, per-root counts and enumeration of one motif vs the oracle."""
    q = gg.compile(motif)
    want_total, want_pr = og.count(motif, per_root=True)
    pr = pr_tensor(gg.n_edges) if per_root else None
    got = q.count(per_root=pr)
    assert got == want_total, (motif.name, got, want_total)
    if per_root:
        assert np.array_equal(pr[: gg.n_edges].cpu().numpy().astype(np.uint64), want_pr), motif.name
    if enum_cap is not None:
        cap = want_total if enum_cap == "all" else int(enum_cap)
        want_rows, _ = og.enumerate(motif, cap=cap)
        out = torch.full((max(cap, 1), motif.k), -7, dtype=torch.int32, device="cuda")
        nw, tot, trunc = q.enumerate(out)
        assert tot == want_total and nw == min(cap, want_total) and trunc == (want_total > cap)
        assert np.array_equal(out[:nw].cpu().numpy(), want_rows), motif.name
    return got


def test_tiny_uniform_workload_full(tmg):
    """1,000 nodes / 20,000 edges, 3-cycle delta = 10,000: count, per-root, full enumeration."""
    g = synth.tiny_uniform()
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    for delta in (10_000, 100_000, 1_000_000):
        check_query(tmg, gg, og, synth.cycle(3, delta), enum_cap="all")
    check_query(tmg, gg, og, synth.cycle(4, 200_000), enum_cap="all")


MOTIFS = [
    [(0, 1)], [(0, 1), (1, 0)], [(0, 1), (0, 1)], [(0, 1), (1, 2)], [(0, 1), (0, 2)], [(1, 0), (2, 0)],
    [(0, 1), (1, 2), (2, 0)], [(0, 1), (1, 0), (0, 1)], [(0, 1), (2, 3)], [(0, 1), (2, 0), (1, 2)],
    [(0, 1), (1, 2), (2, 3), (3, 0)], [(0, 1), (0, 2), (0, 3)], [(0, 1), (1, 0), (0, 1), (1, 0)],
    [(0, 1), (2, 3), (1, 2)], [(0, 1), (1, 2), (0, 2)], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)],
    [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (1, 3)],
]


@pytest.mark.parametrize("seed", [0, 1])
def test_dense_uniform_many_motifs(tmg, seed):
    """Dense small multigraph with timestamp ties: every motif shape, with and without gaps."""
    rng = np.random.default_rng(seed)
    n, m = 40, 6000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    t = rng.integers(0, 30_000, m).astype(np.int64)
    og = oracle.Graph(n, src, dst, t)
    gg = tmg.Graph.load(n, src, dst, t)
    assert np.array_equal(gg.edge_perm(), og.sorted_edges()[3])
    for edges in MOTIFS:
        k = len(edges)
        delta = 400 if k <= 3 else 150
        mo = synth.Motif(edges, delta, name=str(edges))
        check_query(tmg, gg, og, mo, enum_cap="all" if k <= 4 else None)
        if k >= 2:
            gaps = [int(x) for x in rng.integers(20, 200, k - 1)]
            check_query(tmg, gg, og, synth.Motif(edges, delta, gaps, name=f"{edges} gaps"), enum_cap=1000)


LOOKAHEAD_MOTIFS = [
    [(0, 1), (1, 2), (0, 1), (1, 2)],
    [(0, 1), (1, 2), (2, 0), (0, 1), (1, 2), (2, 0)],
    [(0, 1), (1, 2), (2, 3), (0, 1), (3, 0)],
    [(0, 1), (1, 2), (2, 0), (1, 0), (2, 1), (0, 2), (0, 1)],   # 4 later pairs bound at one level
    [(0, 1), (1, 0), (0, 1), (1, 0), (0, 1), (1, 0), (0, 1)],
    [(0, 1), (2, 3), (1, 2), (0, 3), (3, 0), (2, 1)],
    [(0, 1), (2, 3), (1, 2), (0, 3), (3, 0), (2, 1), (1, 3), (3, 1)],   # more new pairs than are checked
]


@pytest.mark.parametrize("delta", [200, 600])
def test_lookahead_motifs(tmg, delta):
    """Motifs whose later edges join nodes bound early (the search prunes partial matches
    whose later pairs have no edge left in the window): counts, per-root counts and rows,
    with and without gaps, on an 8-node multigraph dense enough that most pairs recur."""
    rng = np.random.default_rng(11)
    n, m = 8, 4000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    t = rng.integers(0, 20_000, m).astype(np.int64)
    og = oracle.Graph(n, src, dst, t)
    gg = tmg.Graph.load(n, src, dst, t)
    for edges in LOOKAHEAD_MOTIFS:
        k = len(edges)
        check_query(tmg, gg, og, synth.Motif(edges, delta, name=str(edges)), enum_cap=5000)
        gaps = [int(x) for x in rng.integers(30, delta, k - 1)]
        check_query(tmg, gg, og, synth.Motif(edges, delta, gaps, name=f"{edges} gaps"), enum_cap=5000)


def test_constraint_sweep_queries(tmg):
    """The 4-cycle of the constraint sweep with no constraints, node labels, gaps and an
    anti-edge, on a scaled power-law graph: counts and per-root counts equal the oracle's,
    and each added constraint can only remove matches."""
    g = _powerlaw_small(seed=77, n=4000, m=120_000)
    g.nlabel = synth.node_labels(g.n_nodes, 2, 78)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    counts = [check_query(tmg, gg, og, mo, enum_cap=3000) for mo in synth.constraint_sweep_queries(delta=20_000)]
    assert counts[0] >= counts[1] >= counts[2] >= counts[3] and counts[3] > 0, counts


def test_labels(tmg):
    rng = np.random.default_rng(5)
    n, m = 60, 8000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    t = rng.integers(0, 40_000, m).astype(np.int64)
    el = rng.integers(0, 3, m).astype(np.uint8)
    nl = rng.integers(0, 2, n).astype(np.uint8)
    og = oracle.Graph(n, src, dst, t, el, nl)
    gg = tmg.Graph.load(n, src, dst, t, el, nl)
    for edges in ([(0, 1), (1, 2), (2, 0)], [(0, 1), (1, 2), (2, 3)], [(0, 1), (2, 3), (1, 2)], [(0, 1), (0, 2)]):
        k = len(edges)
        nn = 1 + max(max(e) for e in edges)
        for trial in range(3):
            el_c = [int(x) if rng.random() < 0.5 else -1 for x in rng.integers(0, 3, k)]
            nl_c = [int(x) if rng.random() < 0.4 else -1 for x in rng.integers(0, 2, nn)]
            mo = synth.Motif(edges, 500, elabel=el_c, nlabel=nl_c, name=f"{edges} {el_c} {nl_c}")
            check_query(tmg, gg, og, mo, enum_cap="all")


def _powerlaw_small(seed=21, n=20_000, m=200_000):
    return synth.powerlaw_graph(n, m, seed, alpha=2.1, span=94_608_000.0 / 50)


def test_powerlaw_queries_scaled(tmg):
    """The four power-law queries (3-cycle, 4-cycle, out-star, 4-edge ping-pong, delta = 3600)
    on a scaled-down power-law graph (input unsorted), with capped enumeration."""
    g = _powerlaw_small()
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    for q in synth.powerlaw_queries(3600):
        tot = check_query(tmg, gg, og, q, enum_cap="all")
        check_query(tmg, gg, og, q, per_root=False, enum_cap=max(1, tot // 3))
    check_query(tmg, gg, og, synth.in_star(3, 3600), enum_cap=50)


def test_hub_skewed_queries_scaled(tmg):
    """Labelled 5-edge path with gaps and the 6-edge chorded 4-cycle on a scaled hub-skewed graph."""
    g = synth.hub_skewed_100m(scale=0.002)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    for q in synth.hub_skewed_queries():
        check_query(tmg, gg, og, q)
    p = synth.path(5, 7200)
    p.gaps = [600] * 4
    check_query(tmg, gg, og, p)


def test_root_ranges_and_tunings(tmg):
    """Sharded root ranges sum to the whole; every tuning gives identical per-root counts."""
    g = _powerlaw_small(seed=33, n=5000, m=100_000)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    q4 = synth.cycle(4, 3600)
    want_total, want_pr = og.count(q4, per_root=True)
    q = gg.compile(q4)
    cuts = [0, 1, 777, 40_000, 40_001, g.n_edges]
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        pr = pr_tensor(b - a)
        parts.append(q.count_roots(a, b, per_root=pr))
        assert np.array_equal(pr[: b - a].cpu().numpy().astype(np.uint64), want_pr[a:b])
    assert sum(parts) == want_total
    for w, c, d, s in [(1, 32, -1, 0), (2, 64, 0, 0), (8, 1024, 1, 1), (16, 256, 2, 8), (4, 32, 2, 0)]:
        q.set_tuning(w, c, d, s)
        pr = pr_tensor(g.n_edges)
        assert q.count(per_root=pr) == want_total, (w, c, d, s)
        assert np.array_equal(pr[: g.n_edges].cpu().numpy().astype(np.uint64), want_pr)


def test_enumerate_batch(tmg):
    """tm_enumerate_batch: each query's exact total and its lexicographically first rows,
    equal to the oracle's, for caps above the total, below it (TM_E_TRUNCATED) and zero, in
    one call; a query given twice is rejected."""
    g = _powerlaw_small(seed=88, n=5000, m=80_000)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    mix = synth.powerlaw_queries(3600) + synth.query_mix(10, seed=synth.SEED_BASE + 31, dmax=20_000)
    qs = [gg.compile(mo) for mo in mix]
    want = [og.count(mo) for mo in mix]
    caps = [w + 3 if j % 3 == 0 else (max(1, w // 2) if j % 3 == 1 else 0) for j, w in enumerate(want)]
    outs = [None if c == 0 else torch.full((c, mo.k), -5, dtype=torch.int32, device="cuda")
            for c, mo in zip(caps, mix)]
    for rep in range(2):
        nw, tot, trunc, ms = gg.enumerate_batch(qs, outs, timed=True)
        assert tot == want
        assert nw == [min(w, c) for w, c in zip(want, caps)]
        assert trunc == any(w > c for w, c in zip(want, caps))
        assert ms[0] > 0
        for mo, o, c, n in zip(mix, outs, caps, nw):
            if c:
                rows, _ = og.enumerate(mo, cap=c)
                assert np.array_equal(o[:n].cpu().numpy(), rows), (mo.name, rep)
    with pytest.raises(tmg.TMError):
        gg.enumerate_batch([qs[0], qs[0]], [None, None])


def test_donation_on_a_hub(tmg):
    """A few hubs with thousands of edges inside one window: donation to idle warps must not
    lose or duplicate work (split at every level, threshold 0)."""
    rng = np.random.default_rng(9)
    n, m = 3000, 60_000
    hubs = rng.integers(0, n, 4)
    src = np.where(rng.random(m) < 0.5, rng.choice(hubs, m), rng.integers(0, n, m)).astype(np.int32)
    dst = np.where(rng.random(m) < 0.5, rng.choice(hubs, m), rng.integers(0, n, m)).astype(np.int32)
    t = rng.integers(0, 2_000_000, m).astype(np.int64)
    og = oracle.Graph(n, src, dst, t)
    gg = tmg.Graph.load(n, src, dst, t)
    for mo in (synth.cycle(3, 20_000), synth.out_star(3, 3000), synth.ping_pong(4, 30_000), synth.cycle(4, 8000)):
        want = og.count(mo)
        q = gg.compile(mo)
        for d in (0, 1, 2):
            q.set_tuning(4, 64, d, 0)
            assert q.count() == want, (mo.name, d)


def test_star_continuations_ties_and_donation(tmg):
    """Stars search the same hub list at every level (out- and in-stars from one node): hub
    lists with many equal timestamps (each level's window starts after every tie of the
    previous edge), donation at every split depth, a gap bound on the last edge only;
    counts, per-root counts and rows vs the oracle."""
    rng = np.random.default_rng(17)
    n, m = 2000, 40_000
    hubs = rng.integers(0, n, 3)
    src = np.where(rng.random(m) < 0.6, rng.choice(hubs, m), rng.integers(0, n, m)).astype(np.int32)
    dst = np.where(rng.random(m) < 0.6, rng.choice(hubs, m), rng.integers(0, n, m)).astype(np.int32)
    t = (rng.integers(0, 400_000, m) // 50 * 50).astype(np.int64)      # ~8,000 distinct times
    og = oracle.Graph(n, src, dst, t)
    gg = tmg.Graph.load(n, src, dst, t)
    gapped = synth.out_star(4, 2000)
    gapped.gaps = [2000, 2000, 600]
    gapped.name = "outstar4_gap600"
    for mo in (synth.out_star(3, 1000), synth.out_star(4, 1000), synth.in_star(4, 1000), gapped):
        want = og.count(mo)
        q = gg.compile(mo)
        for d in (0, 1, 2, 3):
            q.set_tuning(4, 64, d, 0)
            assert q.count() == want, (mo.name, d)
        check_query(tmg, gg, og, mo, per_root=True, enum_cap=min(want, 200_000))


def test_edge_cases(tmg):
    # empty graph
    gg = tmg.Graph.load(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    q = gg.compile(synth.cycle(3, 10))
    assert q.count() == 0
    out = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    assert q.enumerate(out) == (0, 0, False)
    # one edge, a self-loop, equal times, k = 1
    src = np.array([0, 1, 2, 2], np.int32); dst = np.array([1, 1, 0, 1], np.int32)
    t = np.array([5, 5, 5, 6], np.int64)
    og = oracle.Graph(3, src, dst, t)
    gg = tmg.Graph.load(3, src, dst, t)
    for mo in (synth.Motif([(0, 1)], 0), synth.path(2, 10), synth.Motif([(0, 1), (0, 1)], 10)):
        check_query(tmg, gg, og, mo, enum_cap="all")
    # eight edges over eight nodes, saturating delta near INT64_MAX
    e8 = [(i, (i + 1) % 8) for i in range(8)]
    src = np.array([a for a, _ in e8] * 3, np.int32); dst = np.array([b for _, b in e8] * 3, np.int32)
    t = np.arange(24, dtype=np.int64) * 10 + (2 ** 62)
    og = oracle.Graph(8, src, dst, t)
    gg = tmg.Graph.load(8, src, dst, t)
    for delta in (70, 150, np.iinfo(np.int64).max):
        check_query(tmg, gg, og, synth.Motif(e8, int(delta)), enum_cap="all")
    # time gaps beyond 32 bits (successor words saturate): windows decided by the full times
    rng = np.random.default_rng(9)
    src = rng.integers(0, 6, 300).astype(np.int32); dst = rng.integers(0, 6, 300).astype(np.int32)
    t = np.sort(rng.integers(0, 40, 300)).astype(np.int64) * (2 ** 33) + rng.integers(0, 3, 300)
    og = oracle.Graph(6, src, dst, t)
    gg = tmg.Graph.load(6, src, dst, t)
    for delta in (2 ** 32 - 3, 2 ** 32 + 5, 3 * 2 ** 33, 2 ** 40, np.iinfo(np.int64).max):
        for mo in (synth.cycle(3, int(delta)), synth.ping_pong(4, int(delta)), synth.path(3, int(delta))):
            check_query(tmg, gg, og, mo, enum_cap=2000)
    # invalid motifs are rejected with TM_E_INVALID
    with pytest.raises(tmg.TMError):
        gg.compile(synth.Motif([(0, 0)], 10))
    with pytest.raises(tmg.TMError):
        gg.compile(synth.Motif([(0, 1)], 10, elabel=[1]))   # graph has no edge labels
    with pytest.raises(tmg.TMError):
        tmg.Graph.load(3, np.array([0], np.int32), np.array([3], np.int32), np.array([1], np.int64))


def test_device_input_and_unsorted_input(tmg):
    g = _powerlaw_small(seed=44, n=3000, m=50_000)
    og = oracle.Graph.from_synth(g)
    gd = tmg.Graph.load(g.n_nodes, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                        torch.from_numpy(g.t).cuda())
    assert np.array_equal(gd.edge_perm(), og.sorted_edges()[3])
    check_query(tmg, gd, og, synth.cycle(3, 3600), enum_cap="all")


def test_batch_matches_single_queries(tmg):
    """64-query mix in one persistent CUDA-graph launch: per-query totals equal the oracle's."""
    g = _powerlaw_small(seed=55, n=5000, m=60_000)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    mix = synth.query_mix(64, dmax=20_000)
    qs = [gg.compile(q) for q in mix]
    want = [og.count(q) for q in mix]
    assert gg.count_batch(qs) == want
    assert gg.count_batch(qs) == want            # graph replay
    assert gg.count_batch(qs[:7]) == want[:7]
    assert [q.count() for q in qs[:10]] == want[:10]


def test_work_counters_match_oracle(tmg):
    """Algorithm-independent work counters (roofline numerator) agree with the oracle's."""
    g = _powerlaw_small(seed=66, n=4000, m=50_000)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    for mo in (synth.cycle(3, 3600), synth.ping_pong(4, 3600), synth.Motif([(0, 1), (2, 3)], 50)):
        _, w = og.count(mo, work=True)
        got = gg.compile(mo).work()
        assert got["roots"] == w["roots"]
        assert got["nodes"] == w["nodes"]
        assert got["entries"] == w["entries"]
        assert got["matches"] == w["matches"]


def test_powerlaw_10m_sampled_roots(tmg):
    """Full 10M-edge power-law workload in the benchmark's launch configuration: totals equal
    the sum of per-root counts, and per-root counts equal the oracle's on sampled root ranges."""
    g = synth.powerlaw_10m()
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    m = g.n_edges
    for mo in synth.powerlaw_queries(3600):
        q = gg.compile(mo)
        pr = pr_tensor(m)
        tot = q.count(per_root=pr)
        prn = pr.cpu().numpy()
        assert int(prn.sum()) == tot
        assert q.count() == tot
        for a in (0, m // 3, m - 20_000):
            _, want = og.count(mo, a, a + 20_000, per_root=True)
            assert np.array_equal(prn[a:a + 20_000].astype(np.uint64), want), (mo.name, a)


def test_hub_skewed_100m_sampled_roots(tmg):
    """Full 100M-edge hub-skewed workload (labels, gaps): total = sum of per-root counts, and
    per-root counts equal the oracle's on sampled root ranges, incl. the busiest hub roots."""
    g = synth.hub_skewed_100m()
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    m = g.n_edges
    for mo in synth.hub_skewed_queries():
        q = gg.compile(mo)
        pr = pr_tensor(m)
        tot = q.count(per_root=pr)
        prn = pr.cpu().numpy()
        assert int(prn.sum()) == tot
        busiest = int(np.argmax(prn))
        for a in (0, m // 2, max(0, min(m - 5000, busiest - 2500))):
            _, want = og.count(mo, a, a + 5000, per_root=True)
            assert np.array_equal(prn[a:a + 5000].astype(np.uint64), want), (mo.name, a)


def test_bounded_wait_reports_timeout_and_context_survives(tmg):
    """A task slot that nothing publishes (host-staged, no GPU fault): the popping warp's
    bounded wait runs out, the call returns TM_E_TIMEOUT, and the next call is correct."""
    g = _powerlaw_small(seed=77, n=2000, m=20_000)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    mo = synth.cycle(3, 3600)
    q = gg.compile(mo)
    q.inject_fault(1)
    with pytest.raises(tmg.TMError) as ei:
        q.count()
    assert ei.value.status == tmg.E_TIMEOUT
    assert q.count() == og.count(mo)


ANTI_MOTIFS = [
    ([(0, 1), (1, 2), (2, 0)], [(0, 2, 0, 300)]),
    ([(0, 1), (1, 2), (2, 0)], [(1, 0, 1, 500), (2, 1, 2, 200)]),
    ([(0, 1), (1, 0)], [(0, 1, 0, 400)]),
    ([(0, 1), (0, 2), (0, 3)], [(1, 2, 2, 600)]),
    ([(0, 1), (1, 2)], [(2, 0, 0, 0)]),
    ([(0, 1), (1, 2), (2, 3), (3, 0)], [(0, 2, 1, 150), (3, 1, 0, 250)]),   # attached to an earlier edge
    ([(0, 1)], [(1, 0, 0, 300)]),
]


def test_anti_edges(tmg):
    """Temporal anti-edges: counts, per-root counts and enumeration equal the oracle's, on a dense
    multigraph (pair-list lookups) and a sparse one (short lists)."""
    rng = np.random.default_rng(31)
    for n, m, tmax in ((40, 6000, 30_000), (400, 6000, 200_000)):
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        t = rng.integers(0, tmax, m).astype(np.int64)
        og = oracle.Graph(n, src, dst, t)
        gg = tmg.Graph.load(n, src, dst, t)
        for edges, anti in ANTI_MOTIFS:
            delta = 400 if len(edges) <= 3 else 200
            mo = synth.Motif(edges, delta, anti=anti, name=f"{edges} anti {anti}")
            check_query(tmg, gg, og, mo, enum_cap="all")


def test_anti_edge_walkthrough_golden(tmg):
    import json, os
    spec = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "walkthrough.json")))
    for case in spec["cases"]:
        e = np.array(case["edges"], np.int64)
        gg = tmg.Graph.load(int(e[:, :2].max()) + 1, e[:, 0].astype(np.int32), e[:, 1].astype(np.int32), e[:, 2])
        mo = synth.Motif([tuple(x) for x in case["motif"]], case["delta"], case["gaps"],
                         anti=[tuple(a) for a in case.get("anti", [])])
        assert gg.compile(mo).count() == case["expected_count"], case["reason"]


def test_baseline_ablation_kernel_counts(tmg):
    """The thread-per-tree baseline kernel (ablation) gives the oracle's counts too."""
    rng = np.random.default_rng(8)
    n, m = 40, 5000
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    t = rng.integers(0, 30_000, m).astype(np.int64)
    el = rng.integers(0, 2, m).astype(np.uint8)
    og = oracle.Graph(n, src, dst, t, el)
    gg = tmg.Graph.load(n, src, dst, t, el)
    for edges in MOTIFS:
        mo = synth.Motif(edges, 300 if len(edges) <= 3 else 120, name=str(edges))
        assert gg.compile(mo).count_baseline()[0] == og.count(mo), edges
    mo = synth.Motif([(0, 1), (1, 2), (2, 0)], 300, [100, 150], elabel=[1, -1, 0])
    assert gg.compile(mo).count_baseline()[0] == og.count(mo)
