"""The multi-GPU path on CPU: world_size-2 gloo process groups check that the
DAG shards of the ranks cover the batch exactly once and that the timing
reduction returns the slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2009_07482_gb300.multi import max_over_ranks, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard(list(range(256)), rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    t = max_over_ranks(1.5 + rank)            # rank r "took" 1.5 + r seconds
    q.put((rank, sorted(x for part in got for x in part), t, len(mine)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_shards_cover_the_batch_once_and_time_is_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, allx, t, n in res:
        assert allx == list(range(256))
        assert t == 1.5 + (world - 1)
        assert n == 256 // world


def test_shard_arguments():
    assert shard([1, 2, 3], 0, 1) == [1, 2, 3]
    with pytest.raises(ValueError):
        shard([1], 2, 2)
