"""Failure handling on the GPU path, every failure made on the host (no GPU fault).

The library's allocation hook (tm_inject_alloc_failure) makes one device or pinned-host
allocation fail as if the device were out of memory: in graph load (first, early and late
allocations of the build), in count and enumerate scratch, and in a served batch.  Each call
must return TM_E_OOM without touching its outputs, and the next call must be exact against
the oracle.  The bounded device wait (a task slot nobody publishes) is covered in
test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_02800_gb300 as tmg
    g = synth.powerlaw_graph(4000, 60_000, 313, span=94_608_000.0 / 50)
    return tmg, g, oracle.Graph.from_synth(g)


def expect_oom(tmg, fn):
    with pytest.raises(tmg.TMError) as e:
        fn()
    tmg.inject_alloc_failure(-1)
    assert e.value.status == tmg.E_OOM, e.value


def test_graph_load_oom_then_exact(env):
    tmg, g, og = env
    # a load makes 11 to 16 allocations (input upload buffers, the graph's one
    # storage block, build temporaries): fail the first, the fourth (the storage
    # block when the input comes from the host), an early and a late temporary
    for after in (0, 3, 7, 10):
        tmg.inject_alloc_failure(after)
        expect_oom(tmg, lambda: tmg.Graph.from_synth(g))
    gg = tmg.Graph.from_synth(g)
    mo = synth.cycle(3, 3600)
    assert gg.compile(mo).count() == og.count(mo)


def test_count_and_enumerate_oom_then_exact(env):
    tmg, g, og = env
    gg = tmg.Graph.from_synth(g)
    mo = synth.cycle(4, 3600)
    want_total = og.count(mo)
    want_rows, _ = og.enumerate(mo)
    for after in range(0, 4):
        q = gg.compile(mo)                     # fresh query: its scratch is allocated on first use
        tmg.inject_alloc_failure(after)
        expect_oom(tmg, lambda: q.count())
        assert q.count() == want_total
        q.free()
    for after in range(0, 6):
        q = gg.compile(mo)
        out = torch.full((want_total + 3, mo.k), -9, dtype=torch.int32, device="cuda")
        tmg.inject_alloc_failure(after)
        try:
            q.enumerate(out)
            failed = False
        except tmg.TMError as e:
            failed = True
            assert e.status == tmg.E_OOM
        tmg.inject_alloc_failure(-1)
        if failed:
            assert bool((out == -9).all())     # outputs untouched on error
        nw, tot, trunc = q.enumerate(out)
        assert (nw, tot, trunc) == (want_total, want_total, False)
        assert np.array_equal(out[:nw].cpu().numpy(), want_rows)
        q.free()


def test_served_batch_oom_then_exact(env):
    tmg, g, og = env
    gg = tmg.Graph.from_synth(g)
    mo = synth.out_star(3, 1800)
    q = gg.compile(mo)
    want_rows, want_total = og.enumerate(mo)
    srv = gg.serve(mem_budget_bytes=1 << 30, streams=2)
    try:
        tmg.inject_alloc_failure(0)
        tk = srv.submit(q, enumerate=True, cap=want_total + 10)
        r = srv.wait(tk, 60_000)
        tmg.inject_alloc_failure(-1)
        assert r.status == tmg.E_OOM and r.n_written == 0 and r.matches_ptr == 0
        srv.release(tk)
        tk = srv.submit(q, enumerate=True, cap=want_total + 10)
        tk2 = srv.submit(q)
        r = srv.wait(tk, 60_000)
        assert r.status == tmg.OK and r.total == want_total and r.n_written == want_total
        assert np.array_equal(srv.matches(r).cpu().numpy(), want_rows)
        assert srv.wait(tk2, 60_000).total == want_total
        srv.release(tk)
        srv.release(tk2)
    finally:
        tmg.inject_alloc_failure(-1)
        srv.stop()
