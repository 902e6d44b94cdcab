"""GPU parity of the point-rule heating (HEAT_HEATING_POINT, Eq. heating at the bin centres)
against the oracle's point mode, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, relerr

pytestmark = pytest.mark.gpu

EXACT_TOL = 1e-10  # FP64 build and recursion: relative, over entries > 1e-280
POINT = heat.HEAT_HEATING_POINT


@pytest.fixture(scope="module")
def single_point():
    wl = W.single_cell()
    Cf = oracle.grain_cooling(wl)
    P, j, led, st = oracle.solve_batch(wl, Cf, want_ledger=True, heating=oracle.HEATING_POINT)
    assert st == oracle.OK
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, Cf, P, j, led, lib
    lib.close()


@pytest.fixture(scope="module")
def batched_point():
    """7 grains spanning 128..1024 bins, 45 cells (ragged against 32-cell groups)."""
    full = W.batched(cells=45)
    wl = W.grain_subset(full, [0, 5, 17, 30, 41, 52, 63])
    Cf = oracle.grain_cooling(wl)
    P, j, led, st = oracle.solve_batch(wl, Cf, want_ledger=True, heating=oracle.HEATING_POINT)
    assert st == oracle.OK
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, Cf, P, j, led, lib
    lib.close()


def test_point_rule_single_cell(single_point):
    """One cell: the element-parallel build (block per spectrum, threads over columns)."""
    wl, _, P, j, _, lib = single_point
    Pg, jg = lib.solve(build=heat.HEAT_BUILD_F64, heating=POINT)
    rP, okP = relerr(Pg, P)
    rj, okj = relerr(jg, j)
    assert okP and okj
    assert rP <= EXACT_TOL, rP
    assert rj <= EXACT_TOL, rj
    for g in range(wl.n_grains):
        assert abs(Pg[0, wl.grain_slice(g)].sum() - 1.0) < 1e-13


@pytest.mark.parametrize("chunk", [32, 0])
def test_point_rule_batched_subset_ragged(batched_point, chunk):
    """45 cells: the lane-per-cell build, in 32-cell chunks (a ragged tail) and in one chunk."""
    wl, _, P, j, _, lib = batched_point
    Pg, jg = lib.solve(build=heat.HEAT_BUILD_F64, heating=POINT, chunk_cells=chunk)
    rP, okP = relerr(Pg, P)
    rj, okj = relerr(jg, j)
    assert okP and okj
    assert rP <= EXACT_TOL, rP
    assert rj <= EXACT_TOL, rj


def test_point_rule_differs_from_the_integral_form(batched_point):
    """The option really switches the matrix: the integral-form solve of the same cells
    differs from the point-rule one by far more than rounding."""
    wl, _, P, _, _, lib = batched_point
    Pi, _ = lib.solve(build=heat.HEAT_BUILD_F64, want_j=False)
    Pp, _ = lib.solve(build=heat.HEAT_BUILD_F64, heating=POINT, want_j=False)
    assert np.max(np.abs(Pp - Pi)) > 1e-3
    assert np.max(np.abs(Pp - P)) < 1e-9


def test_point_rule_energy_check(batched_point):
    """ledger_out with the point rule: [0] is the physical absorbed power (the same bits as
    with the integral form), [1] the model's emitted power, which equals the oracle's
    model absorbed = emitted power; their ratio shows the heating the point rule drops."""
    import torch

    wl, _, _, _, led, lib = batched_point

    def ledger(**kw):
        out = torch.zeros(wl.n_cells, wl.n_grains, 2, dtype=torch.float64, device="cuda")
        o = heat.heat_default_opts(emis=heat.HEAT_EMIS_NONE, ledger_out=out, chunk_cells=32, **kw)
        P = torch.empty(wl.n_cells, wl.total_bins, dtype=torch.float64, device="cuda")
        heat.heat_solve(lib.ctx, o, P, None, torch.cuda.current_stream().cuda_stream)
        heat.heat_sync(lib.ctx)
        return out.cpu().numpy()

    lp = ledger(heating=POINT)
    li = ledger()
    assert np.array_equal(lp[..., 0], li[..., 0])
    r, ok = relerr(lp[..., 1], led[..., 1])
    assert ok and r < 1e-10, r
    # the largest grains absorb nothing under the point rule (every photon is sub-bin): 0 = 0
    r, ok = relerr(led[..., 0], led[..., 1])
    assert ok and r < 1e-11, r
    assert np.any(led[..., 1] == 0.0) and np.any(led[..., 1] > 0.0)


def test_point_rule_option_checks(single_point):
    """The point rule needs the FP64 build; unknown heating values are rejected; the
    surrogate's fallback must use the integral form (all host-side checks)."""
    _, _, _, _, _, lib = single_point
    with pytest.raises(heat.HeatError) as e:
        lib.solve(build=heat.HEAT_BUILD_F32, heating=POINT)
    assert e.value.status == heat.HEAT_EINVAL
    with pytest.raises(heat.HeatError) as e:
        lib.solve(build=heat.HEAT_BUILD_F64, heating=7)
    assert e.value.status == heat.HEAT_EINVAL


def test_point_rule_full_batched_workload_sampled():
    """All 4096 cells x 64 grains (128..1024 bins) in the launch configuration of the timed
    solve, point rule; sampled (cell, grain) spectra against the oracle one by one."""
    import torch

    wl = W.batched()
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        P = torch.empty(wl.n_cells, wl.total_bins, dtype=torch.float64, device="cuda")
        o = heat.heat_default_opts(build=heat.HEAT_BUILD_F64, heating=POINT, emis=heat.HEAT_EMIS_NONE)
        heat.heat_solve(lib.ctx, o, P, None, torch.cuda.current_stream().cuda_stream)
        heat.heat_sync(lib.ctx)
        rng = np.random.default_rng(77)
        cells = np.unique(np.concatenate([[0, wl.n_cells - 1], rng.integers(0, wl.n_cells, 6)]))
        grains = np.unique(np.concatenate([[0, wl.n_grains - 1], rng.integers(0, wl.n_grains, 4)]))
        sub = W.grain_subset(wl, list(grains))
        Cf = oracle.grain_cooling(sub)
        Po, _, _, st = oracle.solve_batch(sub, Cf, want_j=False, u=wl.u[cells], heating=oracle.HEATING_POINT)
        assert st == oracle.OK
        for k, g in enumerate(grains):
            got = P[cells][:, wl.grain_slice(g)].cpu().numpy()
            r, ok = relerr(got, Po[:, sub.grain_slice(k)])
            assert ok and r <= EXACT_TOL, (g, r)
    finally:
        lib.close()
