"""GPU tail pruning (heat_opts.prune_eps): the approximation's error against the unpruned
path and the oracle, its independence of chunking and cell grouping, and option checks."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, masked_relerr

pytestmark = pytest.mark.gpu

EPS = 1e-12
MIXED_TOL = 1e-3  # j, where j > 1e-6 of its peak


@pytest.fixture(scope="module")
def sub():
    """7 grains spanning 128..1024 bins, 45 cells (ragged against 32-cell groups)."""
    full = W.batched(cells=45)
    wl = W.grain_subset(full, [0, 5, 17, 30, 41, 52, 63])
    Cf = oracle.grain_cooling(wl)
    P, j, _, st = oracle.solve_batch(wl, Cf)
    assert st == oracle.OK
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, P, j, lib
    lib.close()


def _spectra(wl, P):
    for g in range(wl.n_grains):
        yield g, P[:, wl.grain_slice(g)]


@pytest.mark.parametrize("build", [heat.HEAT_BUILD_F64, heat.HEAT_BUILD_F32])
def test_pruned_against_unpruned(sub, build):
    """Bins below the cut are computed exactly as without pruning (the same X, a total that
    lacks only the tail): P agrees to ~eps where P is within 1e-6 of its peak, the pruned
    tail is zero, and j (1e-6 mask) moves by far less than the mixed tolerance.  Some
    spectra must actually have been cut."""
    wl, _, _, lib = sub
    P0, j0 = lib.solve(build=build, chunk_cells=32)
    P1, j1 = lib.solve(build=build, chunk_cells=32, prune_eps=EPS)
    cut = 0
    for g, p0 in _spectra(wl, P0):
        p1 = P1[:, wl.grain_slice(g)]
        big = p0 > 1e-6 * p0.max(axis=1, keepdims=True)
        assert np.max(np.abs(p1[big] / p0[big] - 1.0)) < 1e-9, g
        zero = p1 == 0.0
        cut += int(np.sum(zero & (p0 > 0.0)))
        assert np.all((p0 <= 1e-6 * p0.max(axis=1, keepdims=True))[zero]), g
    assert cut > 100, cut
    assert masked_relerr(j1, j0) < 1e-6


@pytest.mark.parametrize("build,tol", [(heat.HEAT_BUILD_F64, 1e-6), (heat.HEAT_BUILD_F32, MIXED_TOL)])
def test_pruned_against_oracle(sub, build, tol):
    """Against the unpruned FP64 oracle: j within the path's tolerance on the 1e-6 mask."""
    wl, _, j, lib = sub
    _, jg = lib.solve(build=build, prune_eps=EPS)
    assert masked_relerr(jg, j) <= tol


def test_pruning_does_not_depend_on_chunks_or_grouping(sub):
    """The cut is decided per cell: chunk sizes and cell ranges give the same bits."""
    wl, _, _, lib = sub
    Pa, ja = lib.solve(build=heat.HEAT_BUILD_F32, prune_eps=EPS, chunk_cells=32)
    Pb, jb = lib.solve(build=heat.HEAT_BUILD_F32, prune_eps=EPS, chunk_cells=0)
    assert np.array_equal(Pa, Pb)
    Pc, _ = lib.solve(build=heat.HEAT_BUILD_F32, prune_eps=EPS, cell_begin=20, cell_count=25, want_j=False)
    assert np.array_equal(Pc, Pa[20:45])


def test_pruned_small_solve(sub):
    """Solves of at most 16 cells (element-parallel kernels) prune with the same test."""
    wl, _, j, lib = sub
    P0, _ = lib.solve(build=heat.HEAT_BUILD_F64, cell_count=5, want_j=False)
    P1, j1 = lib.solve(build=heat.HEAT_BUILD_F64, cell_count=5, prune_eps=EPS)
    assert np.sum((P1 == 0.0) & (P0 > 0.0)) > 10
    for g, p0 in _spectra(wl, P0):
        p1 = P1[:, wl.grain_slice(g)]
        big = p0 > 1e-6 * p0.max(axis=1, keepdims=True)
        assert np.max(np.abs(p1[big] / p0[big] - 1.0)) < 1e-9
    assert masked_relerr(j1, j[:5]) <= 1e-6


def test_prune_option_checks(sub):
    _, _, _, lib = sub
    for bad in (-1e-3, 1.0, 2.0, float("nan")):
        with pytest.raises(heat.HeatError) as e:
            lib.solve(build=heat.HEAT_BUILD_F32, prune_eps=bad)
        assert e.value.status == heat.HEAT_EINVAL


def test_pruned_full_batched_workload_sampled():
    """All 4096 cells x 64 grains on the mixed path with pruning, in the bench's launch
    configuration; sampled spectra against the oracle (j, 1e-6 mask)."""
    import torch

    wl = W.batched()
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        j = torch.empty(wl.n_cells, wl.n_grains, wl.n_lambda, dtype=torch.float32, device="cuda")
        o = heat.heat_default_opts(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32,
                                   prune_eps=EPS)
        heat.heat_solve(lib.ctx, o, None, j, torch.cuda.current_stream().cuda_stream)
        heat.heat_sync(lib.ctx)
        rng = np.random.default_rng(91)
        cells = np.unique(np.concatenate([[0, wl.n_cells - 1], rng.integers(0, wl.n_cells, 6)]))
        grains = np.unique(np.concatenate([[0, wl.n_grains - 1], rng.integers(0, wl.n_grains, 5)]))
        sub_wl = W.grain_subset(wl, list(grains))
        Cf = oracle.grain_cooling(sub_wl)
        _, jo, _, st = oracle.solve_batch(sub_wl, Cf, u=wl.u[cells])
        assert st == oracle.OK
        got = j.cpu().numpy()[cells][:, grains].astype(np.float64)
        assert masked_relerr(got, jo) <= MIXED_TOL
    finally:
        lib.close()
