"""Multi-process plumbing for benchmarks and batch runs (one process per GPU).

The learner's hot path has no exchange step between problems, so ranks only
split independent work (problems, seeds) and agree on timings.  Nothing here
touches the learner's arithmetic.
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def env_rank() -> Tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(items: Sequence, rank: int, world: int) -> List:
    """Round-robin share of `items` for `rank` (every item to exactly one rank)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    return [x for i, x in enumerate(items) if i % world == rank]


def init(backend: str = "nccl"):
    """Initialise torch.distributed when launched with world_size > 1."""
    import torch.distributed as dist
    _, _, world = env_rank()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_max(x: float, device=None) -> float:
    """Maximum of x over ranks (x itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
