"""Multi-process plumbing for runs with one process per GPU.

The hot path partitions like the paper's own decomposition (Sec. 6): the
initial k-points (rows of Gamma_nk and of the collision list) are
independent, so ranks split them with no data-path exchange.  This module
holds the host-side pieces: rank discovery, the contiguous partition of a
unit range, and the max/sum reductions used for timing and totals.
"""
from __future__ import annotations

import os


def rank_world():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def partition(n: int, rank: int, world: int):
    """Contiguous block [start, stop) of n units for this rank; sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad partition arguments")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def _tensor(x, device):
    import torch
    return torch.tensor([float(x)], dtype=torch.float64, device=device)


def _device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x: float) -> float:
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = _tensor(x, _device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = _tensor(x, _device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
