"""Several GPUs of one node: the batched and serving workloads shard at DAG
granularity (independent DAGs), so each rank runs its own share with no
data-path collective; timing takes the max over ranks (torch.distributed,
NCCL on GPUs, gloo on CPU)."""
from __future__ import annotations

import os
from typing import List, Sequence, TypeVar

T = TypeVar("T")


def env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard(items: Sequence[T], rank: int, world: int) -> List[T]:
    """Round-robin share of rank `rank`: items rank, rank+world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return [x for i, x in enumerate(items) if i % world == rank]


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` across the process group (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
