"""Batch sharding over ranks: LPT partition properties, and the multi-rank
path with world_size 2 on the gloo backend (CPU): every rank derives the
same partition without communication, the shards cover the batch exactly
once, and the host-side concatenation maps back to batch order."""
import os

import numpy as np
import pytest

from paper_1604_03703_gb300 import inputs as I
from paper_1604_03703_gb300 import shard


def test_lpt_partition_covers_and_balances():
    sizes = [int(m) for m in I.batch_sizes(4096, 32, 512, 1604037033)]
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        ld = shard.loads(sizes, parts)
        # LPT bound: the heaviest rank exceeds the mean by at most one item
        assert max(ld) <= sum(ld) / world + max(m ** 3 for m in sizes)
    assert shard.lpt_partition([5, 3], 4)[2:] == [[], []]


def test_gather_order_inverts_concatenation():
    sizes = [7, 100, 3, 50, 50, 9]
    parts = shard.lpt_partition(sizes, 2)
    pos = shard.gather_order(parts)
    concat = [i for p in parts for i in p]
    assert [concat[pos[i]] for i in range(len(sizes))] == list(range(len(sizes)))


def _rank_main(rank, world, port, sizes, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = shard.lpt_partition(sizes, world)
    mine = parts[rank]
    # stand-in for the per-rank solve: a result that identifies the matrix
    results = [(i, float(sizes[i])) for i in mine]
    everyone = [None] * world
    dist.all_gather_object(everyone, (parts, results))
    dist.destroy_process_group()
    q.put((rank, everyone))


@pytest.mark.parametrize("world", [2])
def test_sharded_batch_two_ranks_gloo(world):
    import multiprocessing as mp
    import socket

    sizes = [int(m) for m in I.batch_sizes(300, 32, 512, 77)]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        views = out[r]
        # every rank derived the same partition on its own
        assert all(v[0] == views[0][0] for v in views)
        parts = views[0][0]
        results = [res for v in views for res in v[1]]
        assert sorted(i for i, _ in results) == list(range(len(sizes)))
        pos = shard.gather_order(parts)
        ordered = [results[pos[i]] for i in range(len(sizes))]
        assert [i for i, _ in ordered] == list(range(len(sizes)))
        assert all(v == float(sizes[i]) for i, v in ordered)
