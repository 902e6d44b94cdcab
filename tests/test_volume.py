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
