"""Data-parallel sharding of the cells over ranks (one process per GPU).

Every (cell, grain) spectrum is independent (Sec. 3 of the paper computes cells in
parallel with no exchange), so ranks take contiguous cell ranges, replicate the grain
tables and need no collective on the data path.  The collectives here are off the hot
path: the max over ranks of a timing, and an optional gather of per-cell outputs (e.g. the
size-integrated J) to one rank.
"""
from __future__ import annotations


def cell_range(rank: int, world: int, n_cells: int, align: int = 32) -> tuple[int, int]:
    """[begin, end) of rank's cells: contiguous, in whole groups of `align` cells (the
    recursion's warp width) except for the last rank, as even as that allows."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    groups = (n_cells + align - 1) // align
    lo = groups * rank // world
    hi = groups * (rank + 1) // world
    return min(n_cells, lo * align), min(n_cells, hi * align)


def max_over_ranks(value: float) -> float:
    """The maximum of a host value over all ranks (a timed region's duration)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local, n_cells: int, dst: int = 0):
    """Assemble the per-cell rows of all ranks (each holding its cell_range rows of a
    [cells, ...] tensor) on rank dst, in cell order; other ranks get None."""
    import torch
    import torch.distributed as dist

    world, rank = dist.get_world_size(), dist.get_rank()
    rows = [cell_range(r, world, n_cells) for r in range(world)]
    width = max(e - b for b, e in rows)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)] if rank == dst else None
    dist.gather(pad, parts, dst=dst)
    if rank != dst:
        return None
    return torch.cat([p[: e - b] for p, (b, e) in zip(parts, rows)])
