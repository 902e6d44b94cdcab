"""A small volume run on the GPU: chunked, interrupted and resumed, the assembled J equal
to one size-integrated solve of all cells, within 1e-3 of the oracle, and an energy
check per chunk."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import volume as V
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, masked_relerr

pytestmark = pytest.mark.gpu


def test_volume_run_resume_and_parity(tmp_path):
    vol = W.rt_volume((16, 16, 8), corr_cells=3.0, radii_per_composition=2, nbins=128, n_lambda=256)
    chunk = 512
    out = str(tmp_path / "vol")
    cfg = V.volume_config(vol, chunk, "bf16x3")
    solver = V.VolumeSolver(vol, chunk)
    try:
        r = V.run_chunks(V.ChunkManifest(out, cfg), vol.n_cells, chunk, solver.solve_chunk, stop_after=2,
                         prepare=solver.prepare)
        assert r["solved_now"] == 2 and not r["complete"]
        r = V.run_chunks(V.ChunkManifest(out, cfg), vol.n_cells, chunk, solver.solve_chunk, prepare=solver.prepare)
        assert r["solved_now"] == 2 and r["complete"]
    finally:
        solver.close()
    J = V.load_output(out)
    # one solve of all cells (same kernels, any chunking gives the same bits)
    g = vol.grains
    u = vol.fields(0, vol.n_cells)
    wl = W.Workload("volume", g.lam, g.radius, g.composition, g.cabs, g.bin_off, g.T, g.E, g.size_weight, u=u)
    lib = Lib(wl)
    try:
        lib.set_fields(u)
        _, J1 = lib.solve(want_P=False, build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3,
                          j_dtype=heat.HEAT_F32, size_integrate=1)
    finally:
        lib.close()
    assert np.array_equal(J.astype(np.float64), J1)
    # the oracle on a few cells: per-grain spectra summed with the size weights
    cells = np.array([0, 77, 1500, 2047])
    sub = W.field_subset(wl, cells)
    _, j_ref, _, _ = oracle.solve_batch(sub, oracle.grain_cooling(wl))
    assert masked_relerr(J[cells], oracle.size_integrate(g.size_weight, j_ref)) <= 1e-3
    # energy check recorded for every chunk
    import json
    import os

    with open(os.path.join(out, V.MANIFEST)) as f:
        m = json.load(f)
    assert len(m["chunks"]) == 4
    for e in m["chunks"].values():
        assert 0.7 < e["energy"]["weighted_ratio"] < 1.5 and e["energy"]["spectra"] > 0
