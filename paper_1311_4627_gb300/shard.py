"""Data-parallel sharding of the cells over ranks (one process per GPU).

Every (cell, grain) spectrum is independent (Sec. 3 of the paper computes cells in
parallel with no exchange), so ranks take contiguous cell ranges, replicate the grain
tables and need no collective on the data path.  The collectives here are off the hot
path: the max over ranks of a timing, and an optional gather of per-cell outputs (e.g. the
size-integrated J) to one rank.

For devices of unequal speed (the paper's host + coprocessor runs hand chunks of cells to
whichever device is free) ChunkQueue assigns chunks dynamically: each rank claims the next
unclaimed chunk from an atomic counter in a torch.distributed key-value store, so a faster
rank takes more chunks; gather_chunks assembles the results in chunk order.
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


class ChunkQueue:
    """Dynamic assignment of chunks [0, n_chunks) to ranks.  claim() atomically takes the next
    chunk from a counter in `store` (a torch.distributed Store shared by the ranks: TCPStore,
    FileStore, ...) and returns its index, or None once all are taken; every chunk goes to
    exactly one claimant.  `name` keys the counter, so one store can serve several runs."""

    def __init__(self, store, n_chunks: int, name: str = "heat_chunk_queue"):
        if n_chunks < 0:
            raise ValueError("n_chunks must be >= 0")
        self.store, self.n_chunks, self.key = store, int(n_chunks), name

    def claim(self):
        k = int(self.store.add(self.key, 1)) - 1
        return k if k < self.n_chunks else None

    def __iter__(self):
        while True:
            k = self.claim()
            if k is None:
                return
            yield k


def chunk_bounds(k: int, chunk: int, n_cells: int) -> tuple[int, int]:
    """[begin, end) of chunk k of `chunk` cells."""
    return k * chunk, min(n_cells, (k + 1) * chunk)


def gather_chunks(results: dict, n_chunks: int, dst: int = 0):
    """Assemble {chunk index: array of that chunk's rows} held by the ranks into one array in
    chunk order on rank dst (others get None).  Raises if a chunk is missing or held twice."""
    import numpy as np
    import torch.distributed as dist

    world, rank = dist.get_world_size(), dist.get_rank()
    parts = [None] * world if rank == dst else None
    dist.gather_object(results, parts, dst=dst)
    if rank != dst:
        return None
    merged = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise RuntimeError(f"chunk {k} was solved by two ranks")
            merged[k] = v
    missing = [k for k in range(n_chunks) if k not in merged]
    if missing:
        raise RuntimeError(f"chunks {missing} were not solved")
    return np.concatenate([merged[k] for k in range(n_chunks)])
