"""Sharding over ranks, on CPU with the gloo backend (world size 2): the ranges cover the
cells exactly once, and spectra computed per rank (by the oracle) and gathered equal the
single-process result bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1311_4627_gb300 import shard


def test_ranges_partition_the_cells():
    for n in (1, 31, 32, 33, 100, 4096, 4097):
        for world in (1, 2, 3, 8):
            rs = [shard.cell_range(r, world, n) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            for (b0, e0), (b1, e1) in zip(rs, rs[1:]):
                assert e0 == b1
            for b, e in rs[:-1]:
                assert b % 32 == 0 and e % 32 == 0 or e == n
    with pytest.raises(ValueError):
        shard.cell_range(2, 2, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1311_4627_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    full = W.batched(cells=70, n_lambda=128)
    wl = W.grain_subset(full, [0, 40])
    b, e = shard.cell_range(rank, world, wl.n_cells)
    _, j, _, st = oracle.solve_batch(W.field_subset(wl, np.arange(b, e)), oracle.grain_cooling(wl), n_threads=1)
    assert st == oracle.OK
    J = torch.from_numpy(oracle.size_integrate(wl.size_weight, j))
    t = shard.max_over_ranks(float(rank + 1))
    got = shard.gather_rows(J, wl.n_cells)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), got.numpy())
        np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gather_equals_one_process(tmp_path):
    import oracle
    from paper_1311_4627_gb300 import workloads as W

    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    full = W.batched(cells=70, n_lambda=128)
    wl = W.grain_subset(full, [0, 40])
    _, j, _, _ = oracle.solve_batch(wl, oracle.grain_cooling(wl), n_threads=1)
    ref = oracle.size_integrate(wl.size_weight, j)
    got = np.load(os.path.join(tmp_path, "gathered.npy"))
    assert np.array_equal(got, ref)
    assert float(np.load(os.path.join(tmp_path, "tmax.npy"))[0]) == 2.0


def test_chunk_queue_hands_out_every_chunk_once():
    import torch.distributed as dist

    store = dist.HashStore()
    q = shard.ChunkQueue(store, 5, name="t")
    assert [q.claim() for _ in range(7)] == [0, 1, 2, 3, 4, None, None]
    assert list(shard.ChunkQueue(store, 3, name="u")) == [0, 1, 2]
    assert list(shard.ChunkQueue(store, 0, name="v")) == []
    assert shard.chunk_bounds(2, 16, 40) == (32, 40)


def _dyn_worker(rank, world, port, out_dir):
    import time

    import torch.distributed as dist

    import oracle
    from paper_1311_4627_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    store = dist.FileStore(os.path.join(out_dir, "queue"), world)
    full = W.batched(cells=48, n_lambda=64)
    wl = W.grain_subset(full, [0, 40])
    Cf = oracle.grain_cooling(wl)
    chunk, n_chunks = 4, 12
    results = {}
    dist.barrier()  # all ranks start claiming together
    for k in shard.ChunkQueue(store, n_chunks):
        if rank == 0:
            time.sleep(0.5)  # a slow device
        b, e = shard.chunk_bounds(k, chunk, wl.n_cells)
        _, j, _, st = oracle.solve_batch(W.field_subset(wl, np.arange(b, e)), Cf, n_threads=1)
        assert st == oracle.OK
        results[k] = oracle.size_integrate(wl.size_weight, j)
    np.save(os.path.join(out_dir, f"claims{rank}.npy"), np.array(sorted(results), dtype=np.int64))
    got = shard.gather_chunks(results, n_chunks)
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), got)
    dist.barrier()
    dist.destroy_process_group()


def test_dynamic_chunks_over_three_ranks_of_unequal_speed(tmp_path):
    """Three gloo ranks claim 12 chunks from a shared queue; rank 0 is slow.  Every chunk is
    solved once, the slow rank takes fewer chunks, and the gathered result equals the
    single-process one bit for bit."""
    import oracle
    from paper_1311_4627_gb300 import workloads as W

    mp.spawn(_dyn_worker, args=(3, _free_port(), str(tmp_path)), nprocs=3, join=True)
    claims = [np.load(os.path.join(tmp_path, f"claims{r}.npy")) for r in range(3)]
    allc = np.sort(np.concatenate(claims))
    assert np.array_equal(allc, np.arange(12))
    assert len(claims[0]) < (len(claims[1]) + len(claims[2])) / 2
    full = W.batched(cells=48, n_lambda=64)
    wl = W.grain_subset(full, [0, 40])
    _, j, _, _ = oracle.solve_batch(wl, oracle.grain_cooling(wl), n_threads=1)
    ref = oracle.size_integrate(wl.size_weight, j)
    assert np.array_equal(np.load(os.path.join(tmp_path, "gathered.npy")), ref)


def _gather_err_worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    msgs = []
    for results in ({0: np.zeros(2)} if rank == 0 else {2: np.ones(2)},  # chunk 1 missing
                    {0: np.zeros(2), 1: np.ones(2)} if rank == 0 else {1: np.ones(2)}):  # chunk 1 twice
        try:
            shard.gather_chunks(results, 3 if len(msgs) == 0 else 2)
            msgs.append("ok")
        except RuntimeError as e:
            msgs.append(str(e))
    if rank == 0:
        with open(os.path.join(out_dir, "msgs.txt"), "w") as f:
            f.write("\n".join(msgs))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_chunks_refuses_missing_or_duplicated_chunks(tmp_path):
    mp.spawn(_gather_err_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    msgs = open(os.path.join(tmp_path, "msgs.txt")).read().split("\n")
    assert "not solved" in msgs[0] and "two ranks" in msgs[1]
