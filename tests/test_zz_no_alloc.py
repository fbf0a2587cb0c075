"""GPU test of tm_count_batch_noalloc, the batched count for callers that cannot allocate
device memory at query time (pre-planned CUDA-graph or real-time loops, processes under a
fixed memory cap, plug-ins whose host framework owns all allocations).

It is called through the C ABI with a caller-owned totals buffer and must agree exactly
(integer counts) with tm_count_batch, on two calls in a row with different query sets, so
that contents the shared static scratch keeps from one call cannot leak into the next.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_02800_gb300 as tmg
    g = synth.powerlaw_graph(6000, 80_000, 91, span=94_608_000.0 / 40)
    gg = tmg.Graph.from_synth(g)
    return tmg, gg


def call_noalloc(tmg, gg, qs):
    """Direct C-ABI call: tm_count_batch_noalloc(g, qs, nq, stream, totals_dev)."""
    totals = torch.full((len(qs),), -1, dtype=torch.int64, device="cuda")
    arr = (ctypes.c_void_p * len(qs))(*[q._h.value for q in qs])
    st = tmg.lib().tm_count_batch_noalloc(gg._h, arr, len(qs), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          ctypes.c_void_p(totals.data_ptr()))
    assert st == tmg.OK, tmg.lib().tm_last_error()
    return [int(x) for x in totals.cpu().numpy().astype(np.uint64)]


def test_noalloc_matches_existing_batch_twice(setup):
    tmg, gg = setup
    mix = synth.query_mix(40, seed=synth.SEED_BASE + 21, dmax=20_000)
    qs = [gg.compile(q) for q in mix]
    want1 = gg.count_batch(qs)
    got1 = call_noalloc(tmg, gg, qs)
    assert got1 == want1
    # second call in a row: a different, smaller set in another order
    qs2 = qs[::-3]
    want2 = gg.count_batch(qs2)
    got2 = call_noalloc(tmg, gg, qs2)
    assert got2 == want2
    assert any(w > 0 for w in want1)


def test_noalloc_rejects_more_queries_than_its_capacity(setup):
    tmg, gg = setup
    q = gg.compile(synth.cycle(3, 3600))
    cap = 64
    totals = torch.zeros(cap + 1, dtype=torch.int64, device="cuda")
    arr = (ctypes.c_void_p * (cap + 1))(*([q._h.value] * (cap + 1)))
    st = tmg.lib().tm_count_batch_noalloc(gg._h, arr, cap + 1, ctypes.c_void_p(0), ctypes.c_void_p(totals.data_ptr()))
    assert st == tmg.E_INVALID
    assert b"64" in tmg.lib().tm_last_error()
