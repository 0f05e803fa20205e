"""Multi-rank path on the CPU: two gloo ranks split a batch of independent
graphs with no data-path collective; together they cover every graph exactly
once, balance the work, and (solving with the oracle) get the same trees as
one rank solving everything.  The timing reduction the benchmark uses
(max over ranks) is checked too."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2005_06913_gb300 import graphgen as gg
from paper_2005_06913_gb300.sharding import shard_graphs, sub_batch


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        import oracle
        b = gg.batched(40, 16, 3000, 8, 7)
        sizes = np.diff(b.edge_off)
        mine = shard_graphs(sizes, world, rank)
        sb = sub_batch(b, mine)
        trees = {}
        for k, g in enumerate(mine):
            gr = sb.graph(k)
            trees[int(g)] = oracle.kruskal(gr.n, gr.src, gr.dst, gr.w).tolist()
        gathered = [None] * world
        dist.all_gather_object(gathered, (mine.tolist(), trees, int(sizes[mine].sum())))
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)  # the benchmark's timing reduction
        if rank == 0:
            q.put((gathered, float(t.item())))
    finally:
        dist.destroy_process_group()


def test_two_rank_split_covers_and_matches():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, tmax = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 2.0
    b = gg.batched(40, 16, 3000, 8, 7)
    sizes = np.diff(b.edge_off)
    all_idx = sorted(i for part, _, _ in gathered for i in part)
    assert all_idx == list(range(b.G))  # disjoint and complete
    loads = [ld for _, _, ld in gathered]
    assert max(loads) - min(loads) <= sizes.max() + 1
    import oracle
    for _, trees, _ in gathered:
        for g, ids in trees.items():
            gr = b.graph(g)
            assert ids == oracle.kruskal(gr.n, gr.src, gr.dst, gr.w).tolist()


def test_shard_single_process_properties():
    rng = np.random.default_rng(0)
    sizes = rng.integers(1, 10000, 333)
    for world in (1, 2, 3, 8):
        parts = [shard_graphs(sizes, world, r) for r in range(world)]
        allp = np.sort(np.concatenate(parts))
        assert np.array_equal(allp, np.arange(333))
        loads = [sizes[p].sum() for p in parts]
        assert max(loads) - min(loads) <= sizes.max() + 1
    with pytest.raises(ValueError):
        shard_graphs(sizes, 2, 2)
