"""Host-side helpers for running the denoiser on several GPUs of one node.

The method partitions by image: every rank denoises its own images and no
data crosses ranks.  The only collective is the timing reduction of a
benchmark (max over ranks).  Works with the NCCL backend on GPUs and with
gloo on CPU (used by the tests).
"""

from __future__ import annotations

import os


def env_rank() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (defaults 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def image_seed(base_seed: int, rank: int, index: int = 0) -> int:
    """Seed of the `index`-th image of `rank` (distinct across ranks and images)."""
    return base_seed + 10 * (rank * 1000 + index)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
