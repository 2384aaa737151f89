"""Host logic of the multi-GPU runs: one process per GPU, each running the
whole hot path on its own share of independent work (replicas; no
collective on the data path).

The work shards by independent units (whole models of a batched refinement,
or whole replicated steps); the only cross-rank operations are a barrier
around the timed region and a max of the per-rank times.  Everything here
works with the gloo backend on CPU as well as NCCL on GPUs.
"""
from __future__ import annotations

import os
from typing import Tuple


def env_rank_world() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(backend: str | None = None) -> Tuple[int, int]:
    """Join the process group when WORLD_SIZE > 1 (MASTER_ADDR/PORT from the
    environment); bind this process to its GPU when CUDA is present."""
    import torch
    rank, world, local = env_rank_world()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
    return rank, world


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest value of x over all ranks (the timed region ends when the
    slowest rank ends)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous share [begin, end) of n independent units for this rank;
    the shares of all ranks partition [0, n) and differ in size by at most 1."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)
