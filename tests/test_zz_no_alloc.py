"""GPU test of tm_count_batch_noalloc, the batched count for callers that cannot allocate
device memory at query time (real-time loops that reserve all their memory up front,
processes under a fixed memory cap, plug-ins whose host framework owns all allocations).

It is called through the C ABI with a caller-owned totals buffer and must agree exactly
(integer counts) with tm_count_batch and with the CPU oracle, on two calls in a row with
different query sets, so that contents the shared static scratch keeps from one call cannot
leak into the next.  A second case makes one call donate more subtrees than the static task
queue holds (TM_NOALLOC_TASKS slots per call) and checks that the counts are unchanged.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NOALLOC_TASKS = 4096


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_02800_gb300 as tmg
    g = synth.powerlaw_graph(6000, 80_000, 91, span=94_608_000.0 / 40)
    gg = tmg.Graph.from_synth(g)
    return tmg, g, gg


def call_noalloc(tmg, gg, qs):
    """Direct C-ABI call: tm_count_batch_noalloc(g, qs, nq, stream, totals_dev)."""
    totals = torch.full((len(qs),), -1, dtype=torch.int64, device="cuda")
    arr = (ctypes.c_void_p * len(qs))(*[q._h.value for q in qs])
    st = tmg.lib().tm_count_batch_noalloc(gg._h, arr, len(qs), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          ctypes.c_void_p(totals.data_ptr()))
    assert st == tmg.OK, tmg.lib().tm_last_error()
    return [int(x) for x in totals.cpu().numpy().astype(np.uint64)]


def test_noalloc_matches_existing_batch_and_oracle_twice(setup):
    tmg, g, gg = setup
    og = oracle.Graph.from_synth(g)
    mix = synth.query_mix(40, seed=synth.SEED_BASE + 21, dmax=20_000)
    qs = [gg.compile(q) for q in mix]
    want1 = [og.count(q) for q in mix]
    got1 = call_noalloc(tmg, gg, qs)
    assert got1 == want1
    assert gg.count_batch(qs) == want1
    # second call in a row: a different, smaller set in another order
    sel = list(range(len(mix)))[::-3]
    qs2 = [qs[i] for i in sel]
    want2 = [want1[i] for i in sel]
    got2 = call_noalloc(tmg, gg, qs2)
    assert got2 == want2
    assert gg.count_batch(qs2) == want2
    assert any(w > 0 for w in want1)


def test_noalloc_task_queue_overflow_keeps_counts(setup):
    """Hubs with thousands of edges per window and donation at every step (threshold 0, split
    depth 2): one call reserves more task slots than the static queue has; the donations that
    find it full stay with their warps and the counts still equal the oracle's."""
    tmg, _, _ = setup
    rng = np.random.default_rng(9)
    n, m = 3000, 60_000
    hubs = rng.integers(0, n, 4)
    src = np.where(rng.random(m) < 0.5, rng.choice(hubs, m), rng.integers(0, n, m)).astype(np.int32)
    dst = np.where(rng.random(m) < 0.5, rng.choice(hubs, m), rng.integers(0, n, m)).astype(np.int32)
    t = rng.integers(0, 2_000_000, m).astype(np.int64)
    og = oracle.Graph(n, src, dst, t)
    gg = tmg.Graph.load(n, src, dst, t)
    overflowed = False
    for delta in (20_000, 60_000, 200_000):
        mix = [synth.cycle(3, delta), synth.out_star(3, delta // 4), synth.ping_pong(4, delta),
               synth.cycle(4, delta // 2), synth.path(3, delta // 4)] * 4
        qs = [gg.compile(mo) for mo in mix]
        for q in qs:
            q.set_tuning(4, 32, 2, 0)
        want = [og.count(mo) for mo in mix]
        assert call_noalloc(tmg, gg, qs) == want, delta
        st = tmg.last_search_stats()
        if st["reserved"] > NOALLOC_TASKS:
            overflowed = True
            assert gg.count_batch(qs) == want
            break
    assert overflowed, "no call filled the static task queue"


def test_noalloc_rejects_more_queries_than_its_capacity(setup):
    tmg, _, gg = setup
    q = gg.compile(synth.cycle(3, 3600))
    cap = 64
    totals = torch.zeros(cap + 1, dtype=torch.int64, device="cuda")
    arr = (ctypes.c_void_p * (cap + 1))(*([q._h.value] * (cap + 1)))
    st = tmg.lib().tm_count_batch_noalloc(gg._h, arr, cap + 1, ctypes.c_void_p(0), ctypes.c_void_p(totals.data_ptr()))
    assert st == tmg.E_INVALID
    assert b"64" in tmg.lib().tm_last_error()
