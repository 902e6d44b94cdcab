"""Volume runs on the host: the Gaussian random fields and the checkpoint manifest
(interrupt, resume, corrupted chunk, configuration mismatch) with a stand-in chunk solver."""
import math
import os

import numpy as np
import pytest

from paper_1311_4627_gb300 import volume as V
from paper_1311_4627_gb300 import workloads as W


def test_grf_moments_and_correlation_length():
    rng = np.random.Generator(np.random.PCG64(7))
    ell = 4.0
    f = W.gaussian_random_field((64, 64, 64), ell, rng)
    assert abs(f.mean()) < 1e-12 and abs(f.std() - 1.0) < 1e-12
    # Gaussian smoothing with standard deviation ell: autocorrelation exp(-r^2 / (4 ell^2))
    for r in (2, 4, 8):
        rho = np.mean([np.mean(f * np.roll(f, r, axis=a)) for a in range(3)])
        assert abs(rho - math.exp(-r * r / (4 * ell * ell))) < 0.06, (r, rho)


def test_rt_volume_field_statistics():
    vol = W.rt_volume((32, 32, 16), corr_cells=4.0, radii_per_composition=2, nbins=64, n_lambda=128)
    assert vol.n_cells == 32 * 32 * 16 and vol.grains.n_grains == 4
    lc = np.log10(vol.chi)
    assert abs(lc.mean()) < 1e-9 and abs(lc.std() - 1.5) < 1e-9
    assert vol.hardness.min() >= -1.0 and vol.hardness.max() <= 1.0
    u = vol.fields(100, 164)
    assert u.shape == (64, 128) and np.all(u > 0) and np.all(np.isfinite(u))
    # chunking of the field generation does not change any cell
    assert np.array_equal(vol.fields(100, 132), u[:32])


class FakeSolver:
    def __init__(self, n_lambda=8):
        self.calls = []
        self.n = n_lambda

    def solve(self, k, b, e, prepared):
        self.calls.append(k)
        assert prepared is None or prepared == (b, e)
        J = (np.arange(b, e)[:, None] * 10 + np.arange(self.n)[None, :]).astype(np.float32)
        return J, {"gpu_ms": 1.0, "spectra": e - b, "energy": {"weighted_ratio": 1.0}}


def _cfg():
    return {"shape": [10, 10, 1], "chunk_cells": 16}


def test_interrupt_and_resume(tmp_path):
    out = str(tmp_path / "run")
    s = FakeSolver()
    r = V.run_chunks(V.ChunkManifest(out, _cfg()), 100, 16, s.solve, stop_after=3,
                     prepare=lambda b, e: (b, e))
    assert r["solved_now"] == 3 and not r["complete"] and s.calls == [0, 1, 2]
    s2 = FakeSolver()
    r = V.run_chunks(V.ChunkManifest(out, _cfg()), 100, 16, s2.solve, prepare=lambda b, e: (b, e))
    assert r["complete"] and s2.calls == [3, 4, 5, 6]
    J = V.load_output(out)
    assert np.array_equal(J, (np.arange(100)[:, None] * 10 + np.arange(8)[None, :]).astype(np.float32))


def test_corrupted_chunk_is_recomputed(tmp_path):
    out = str(tmp_path / "run")
    V.run_chunks(V.ChunkManifest(out, _cfg()), 100, 16, FakeSolver().solve)
    with open(os.path.join(out, "J_00002.npy"), "r+b") as f:
        f.seek(-4, os.SEEK_END)
        f.write(b"\x00\x00\x00\x01")
    os.remove(os.path.join(out, "J_00005.npy"))
    s = FakeSolver()
    r = V.run_chunks(V.ChunkManifest(out, _cfg()), 100, 16, s.solve)
    assert r["complete"] and s.calls == [2, 5]


def test_fresh_run_ignores_old_manifest_and_mismatch_is_refused(tmp_path):
    out = str(tmp_path / "run")
    V.run_chunks(V.ChunkManifest(out, _cfg()), 100, 16, FakeSolver().solve, stop_after=2)
    with pytest.raises(ValueError):
        V.run_chunks(V.ChunkManifest(out, {"shape": [10, 10, 1], "chunk_cells": 32}), 100, 32, FakeSolver().solve)
    s = FakeSolver()
    V.run_chunks(V.ChunkManifest(out, _cfg()), 100, 16, s.solve, resume=False)
    assert s.calls == list(range(7))


def test_energy_summary():
    led = np.zeros((3, 2, 2))
    led[..., 0] = [[1.0, 2.0], [4.0, 0.0], [1.0, 1.0]]
    led[..., 1] = [[1.1, 1.8], [4.0, 0.0], [0.9, 1.0]]
    s = V.energy_summary(led, np.array([1.0, 0.5]))
    assert s["spectra"] == 5
    assert abs(s["ratio_min"] - 0.9) < 1e-12 and abs(s["ratio_max"] - 1.1) < 1e-12
    wa = 1.0 + 1.0 + 4.0 + 1.0 + 0.5
    we = 1.1 + 0.9 + 4.0 + 0.9 + 0.5
    assert abs(s["weighted_ratio"] - we / wa) < 1e-12


def test_write_chunk_hashes_what_it_writes(tmp_path):
    """A chunk file is the .npy of J, written under its final name only when complete, and
    the returned SHA-256 is the file's."""
    J = np.random.default_rng(1).random((300, 16)).astype(np.float32)
    sha = V.write_chunk(str(tmp_path), "J_00000.npy", J)
    p = os.path.join(tmp_path, "J_00000.npy")
    assert np.array_equal(np.load(p), J)
    assert sha == V.sha256_file(p)
    assert not [f for f in os.listdir(tmp_path) if f.endswith(".tmp")]


class OracleChunkSolver:
    """Stand-in for the GPU solver of a volume run: a chunk's size-integrated J from the FP64
    oracle (real spectra, so that a wrong or reordered chunk shows), optionally slow."""

    def __init__(self, vol, delay=0.0):
        import oracle

        self.vol, self.delay = vol, delay
        self.Cf = oracle.grain_cooling(vol.grains)

    def solve(self, k, b, e, prepared):
        import time

        import oracle

        if self.delay:
            time.sleep(self.delay)
        u = prepared[1] if prepared is not None else self.vol.fields(b, e)
        _, j, _, st = oracle.solve_batch(self.vol.grains, self.Cf, u=u, n_threads=1)
        assert st == oracle.OK
        J = oracle.size_integrate(self.vol.grains.size_weight, j).astype(np.float32)
        return J, {"gpu_ms": 0.0, "spectra": (e - b) * self.vol.grains.n_grains, "energy": {"weighted_ratio": 1.0}}

    def prepare(self, b, e):
        return (b, e), self.vol.fields(b, e)


def _tiny_volume():
    return W.rt_volume((8, 8, 4), corr_cells=2.0, radii_per_composition=1, nbins=32, n_lambda=64)


def _dist_volume_worker(rank, world, port, out_dir, stop_after):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vol = _tiny_volume()
    solver = OracleChunkSolver(vol, delay=1.0 if rank == 0 else 0.0)  # rank 0: a slow device
    res = V.run_distributed(out_dir, _cfg(), vol.n_cells, 16, solver.solve, prepare=solver.prepare,
                            stop_after=stop_after)
    np.save(os.path.join(out_dir, f"claimed{rank}.npy"), np.array(res["claimed"], dtype=np.int64))
    dist.destroy_process_group()


def test_distributed_volume_run_with_a_chunk_queue(tmp_path):
    """Three gloo ranks of unequal speed run the volume driver with dynamic chunk claiming:
    first an interrupted run (one chunk per rank), then a resumed one.  Every chunk is solved
    exactly once, the slow rank solves fewer, the merged manifest is complete and the volume
    equals a single-process run's bit for bit."""
    import torch.multiprocessing as mp

    from .test_shard import _free_port

    out = str(tmp_path / "dist")
    os.makedirs(out)
    mp.spawn(_dist_volume_worker, args=(3, _free_port(), out, 1), nprocs=3, join=True)
    first = [np.load(os.path.join(out, f"claimed{r}.npy")) for r in range(3)]
    m = V.ChunkManifest(out, _cfg())
    m.load(resume=True)
    done_first = set(int(k) for k in m.chunks)
    assert done_first == set(int(k) for c in first for k in c) and len(done_first) == 3
    assert not [p for p in os.listdir(out) if p.startswith("manifest.r")]  # shards merged
    mp.spawn(_dist_volume_worker, args=(3, _free_port(), out, None), nprocs=3, join=True)
    second = [np.load(os.path.join(out, f"claimed{r}.npy")) for r in range(3)]
    m.load(resume=True)
    assert sorted(int(k) for k in m.chunks) == list(range(16))
    # the queue hands every chunk to exactly one rank; chunks the first run finished are
    # claimed and skipped, the others solved once
    assert np.array_equal(np.sort(np.concatenate(second)), np.arange(16))
    solved = [set(int(k) for k in c) - done_first for c in second]
    assert sum(len(x) for x in solved) == 13 and set().union(*solved) | done_first == set(range(16))
    assert len(solved[0]) < (len(solved[1]) + len(solved[2])) / 2  # the slow rank takes fewer
    # the output equals one process's
    ref = str(tmp_path / "single")
    vol = _tiny_volume()
    s = OracleChunkSolver(vol)
    r = V.run_chunks(V.ChunkManifest(ref, _cfg()), vol.n_cells, 16, s.solve, prepare=s.prepare)
    assert r["complete"]
    assert np.array_equal(V.load_output(out), V.load_output(ref))
