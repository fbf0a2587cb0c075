"""Serving loop on the GPU: each request's result is identical alone and in a mix of
concurrently admitted requests, and equals the oracle's (counts exact, match rows equal)."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_02800_gb300 as tmg
    g = synth.powerlaw_graph(8000, 120_000, 77, span=94_608_000.0 / 40)
    og = oracle.Graph.from_synth(g)
    gg = tmg.Graph.from_synth(g)
    return tmg, g, og, gg


def rows_of(srv, res):
    return srv.matches(res).cpu().numpy()


def test_alone_equals_mix_equals_oracle(setup):
    tmg, g, og, gg = setup
    mix = synth.query_mix(24, seed=synth.SEED_BASE + 9, dmax=20_000)
    qs = [gg.compile(q) for q in mix]
    want = [og.count(q) for q in mix]
    enum = [i % 3 == 0 for i in range(len(mix))]
    caps = [max(1, w // 2) if i % 6 == 0 else max(1, w + 5) for i, w in enumerate(want)]
    # alone: one request in flight at a time
    srv = gg.serve(mem_budget_bytes=1 << 30, streams=4, max_batch=16)
    alone = []
    for i, q in enumerate(qs):
        tk = srv.submit(q, enumerate=enum[i], cap=caps[i] if enum[i] else 0)
        r = srv.wait(tk)
        alone.append((r.total, r.n_written, rows_of(srv, r) if enum[i] else None))
        srv.release(tk)
    # mix: everything submitted at once, admitted as slots and memory free up
    tks = [srv.submit(q, enumerate=enum[i], cap=caps[i] if enum[i] else 0) for i, q in enumerate(qs)]
    mixed = []
    for i, tk in enumerate(tks):
        r = srv.wait(tk)
        mixed.append((r.total, r.n_written, rows_of(srv, r) if enum[i] else None))
        srv.release(tk)
    srv.stop()
    for i, mo in enumerate(mix):
        assert alone[i][0] == mixed[i][0] == want[i], mo.name
        assert alone[i][1] == mixed[i][1] == (min(want[i], caps[i]) if enum[i] else 0)
        if enum[i]:
            rows, _ = og.enumerate(mo, cap=caps[i])
            assert np.array_equal(alone[i][2], rows) and np.array_equal(mixed[i][2], rows), mo.name


def test_admission_by_memory(setup):
    tmg, g, og, gg = setup
    mo = synth.cycle(3, 3600)
    q = gg.compile(mo)
    want = og.count(mo)
    # budget fits one enumeration buffer at a time: requests queue and still complete
    per = 200_000 * 3 * 4
    srv = gg.serve(mem_budget_bytes=per + (4 << 20), streams=2, max_batch=4)
    tks = [srv.submit(q, enumerate=True, cap=200_000) for _ in range(5)]
    for tk in tks:
        r = srv.wait(tk)
        assert r.total == want
        srv.release(tk)
    with pytest.raises(tmg.TMError):
        srv.submit(q, enumerate=True, cap=10 ** 9)    # can never fit: TM_E_ADMISSION
    srv.stop()


def test_poll_busy_then_done(setup):
    tmg, g, og, gg = setup
    q = gg.compile(synth.cycle(4, 3600))
    srv = gg.serve()
    tk = srv.submit(q)
    deadline = time.time() + 60
    res = None
    while res is None and time.time() < deadline:
        res = srv.poll(tk)
        time.sleep(0.001)
    assert res is not None and res.total == og.count(synth.cycle(4, 3600))
    srv.release(tk)
    srv.stop()


def test_mixed_feature_sets_in_one_launch(setup):
    """Plain motifs, anti-edge motifs and motifs with look-ahead chords in one batched launch
    and in one served mix (the launch runs the kernel instance with the union of their
    features): every total equals the oracle's, and so do the enumerated rows."""
    tmg, g, og, gg = setup
    d = 20_000
    mix = [synth.cycle(3, d), synth.path(3, d),
           synth.Motif([(0, 1), (1, 2), (2, 0)], d, anti=[(1, 0, 0, d // 4)], name="cycle3_anti"),
           synth.chorded_four_cycle(d),
           synth.Motif([(0, 1), (1, 2), (2, 3), (0, 2)], d, name="path3_chord"),
           synth.Motif([(0, 1), (1, 2), (2, 3), (0, 2)], d, anti=[(2, 1, 1, d // 2)], name="path3_chord_anti"),
           synth.ping_pong(4, d)]
    want = [og.count(q) for q in mix]
    assert all(w > 0 for w in want[:2])
    qs = [gg.compile(q) for q in mix]
    assert gg.count_batch(qs) == want
    assert gg.count_batch(qs[:2]) == want[:2]          # plain instance after the union one
    srv = gg.serve(mem_budget_bytes=1 << 30, streams=2, max_batch=16)
    tks = [srv.submit(q, enumerate=True, cap=want[i] + 3) for i, q in enumerate(qs)]
    for i, tk in enumerate(tks):
        r = srv.wait(tk)
        assert r.total == want[i], mix[i].name
        rows, _ = og.enumerate(mix[i], cap=want[i] + 3)
        assert np.array_equal(rows_of(srv, r), rows), mix[i].name
        srv.release(tk)
    srv.stop()
