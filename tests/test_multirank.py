"""World-size-2 gloo ranks on CPU: root-range sharding covers every root exactly once and the
per-rank counts (here from the oracle, as the ranks have no GPU) sum to the whole-graph count."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2310_02800_gb300.shard import my_range, root_ranges


def test_root_ranges_partition():
    for m in (0, 1, 7, 1000, 10 ** 7 + 3):
        for w in (1, 2, 3, 8):
            rr = root_ranges(m, w)
            assert rr[0][0] == 0 and rr[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(rr[:-1], rr[1:]))
            sizes = [b - a for a, b in rr]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    import oracle
    import synth
    g = synth.powerlaw_graph(2000, 30_000, 17, span=3_000_000.0)
    og = oracle.Graph.from_synth(g)
    motif = synth.cycle(3, 3600)
    a, b = my_range(g.n_edges, world, rank)
    part = og.count(motif, a, b)
    t = torch.tensor([part], dtype=torch.int64)
    dist.all_reduce(t)
    if rank == 0:
        q.put((int(t.item()), og.count(motif)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shard_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    got, want = q.get(timeout=60)
    assert got == want and want > 0
