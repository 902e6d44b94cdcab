"""Thermal-discrete cooling on the GPU (heat_opts.cooling = HEAT_COOLING_DISCRETE) against
the FP64 oracle's thermal-discrete rates and full stationary solve: the downward rate tables,
P, j and the energy check at the exact path's tolerance, on the single cell and a ragged
batched subset; the reduction to the thermal-continuous path when all emission is soft."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, relerr

pytestmark = pytest.mark.gpu

EXACT_TOL = 1e-10
DISCRETE = dict(build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_F64, j_dtype=heat.HEAT_F64,
                cooling=heat.HEAT_COOLING_DISCRETE)


def _case(wl):
    Dg = oracle.grain_cooling_discrete(wl)
    P, j, led, st = oracle.solve_batch_discrete(wl, Dg, want_ledger=True)
    assert st == oracle.OK
    lib = Lib(wl)
    lib.set_fields(wl.u)
    return wl, Dg, P, j, led, lib


@pytest.fixture(scope="module")
def single():
    c = _case(W.single_cell())
    yield c
    c[-1].close()


@pytest.fixture(scope="module")
def ragged():
    """3 batched grains of 128, 160 and 224 bins, 37 cells (ragged groups)."""
    full = W.batched(cells=37, n_lambda=256)
    c = _case(W.grain_subset(full, [0, 2, 6]))
    yield c
    c[-1].close()


@pytest.fixture(scope="module")
def banded():
    """2 cells x the batched workload's grains of 704 and 1024 bins: rates that span few bins
    (the state reduction in device memory, rows and columns limited to the band)."""
    full = W.batched(cells=2, n_lambda=256)
    c = _case(W.grain_subset(full, [42, 63]))
    yield c
    c[-1].close()


@pytest.mark.parametrize("case", ["single", "ragged", "banded"])
def test_downward_rates_match_oracle(case, request):
    wl, Dg, _, _, _, lib = request.getfixturevalue(case)
    got = heat.heat_get_cooling_discrete(lib.ctx, [wl.bins(g) for g in range(wl.n_grains)])
    for g in range(wl.n_grains):
        r, ok = relerr(got[g], Dg[g])
        assert ok and r <= 1e-12, (g, r)


@pytest.mark.parametrize("case", ["single", "ragged", "banded"])
def test_discrete_solve_matches_oracle(case, request):
    import torch

    wl, _, P_ref, j_ref, led_ref, lib = request.getfixturevalue(case)
    led = torch.zeros(wl.n_cells, wl.n_grains, 2, dtype=torch.float64, device="cuda")
    P, j = lib.solve(ledger_out=led.data_ptr(), **DISCRETE)
    r, ok = relerr(P, P_ref)
    assert ok and r <= EXACT_TOL, r
    r, ok = relerr(j, j_ref)
    assert ok and r <= EXACT_TOL, r
    lg = led.cpu().numpy()
    r, ok = relerr(lg[..., 1], led_ref[..., 1])  # emitted power of the discrete model
    assert ok and r <= EXACT_TOL, r
    for g in range(wl.n_grains):
        np.testing.assert_allclose(P[:, wl.grain_slice(g)].sum(axis=1), 1.0, rtol=1e-13)


def test_discrete_differs_from_continuous_for_small_grains(single):
    """The 3.5 A grain's emission skips levels: the two treatments must differ there."""
    wl, _, _, _, _, lib = single
    Pd, _ = lib.solve(want_j=False, **DISCRETE)
    Pc, _ = lib.solve(want_j=False, build=heat.HEAT_BUILD_F64)
    s = wl.grain_slice(0)
    assert np.max(np.abs(Pd[:, s] - Pc[:, s])) > 1e-3


def test_soft_emission_gives_the_continuous_solution():
    """A cross-section that is zero shortward of hc/(1.2 dE) on uniform bins of width dE: the
    discrete rates are the adjacent ones, and both GPU paths give the same P."""
    lam = W.wavelength_grid(256)
    dE = W.H_PLANCK * W.C_LIGHT / (10.0 * W.UM)
    nb = 40
    E = 0.5 * dE + dE * np.arange(nb)
    T = np.geomspace(20.0, 400.0, nb)
    cabs = W.cabs_model(3e-7, lam, "carbonaceous")
    cabs[lam < W.H_PLANCK * W.C_LIGHT / (1.2 * dE)] = 0.0
    u = W.three_bb_fields(lam, np.array([30.0, 3.0]), np.array([0.2, -0.4]), np.array([[0.3, 0.5, 0.2]] * 2))
    wl = W.Workload("soft emission", lam, np.array([3e-7]), ["carbonaceous"], cabs[None, :],
                    np.array([0, nb], dtype=np.int32), T, E, np.ones(1), u=u)
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        Pd, _ = lib.solve(want_j=False, **DISCRETE)
        Pc, _ = lib.solve(want_j=False, build=heat.HEAT_BUILD_F64)
        r, ok = relerr(Pd, Pc)
        assert ok and r <= 1e-10, r
    finally:
        lib.close()


def test_discrete_option_checks(single):
    _, _, _, _, _, lib = single
    for kw in (dict(build=heat.HEAT_BUILD_F32), dict(heating=heat.HEAT_HEATING_POINT), dict(cooling=7)):
        opts = dict(DISCRETE, **kw)
        with pytest.raises(heat.HeatError) as e:
            lib.solve(**opts)
        assert e.value.status == heat.HEAT_EINVAL


def test_discrete_size_limit():
    """More than 2048 bins in a grain: thermal-discrete solves are refused (HEAT_EINVAL), the
    thermal-continuous path still takes the grain."""
    lam = W.wavelength_grid(64)
    nb = 2049
    T = np.geomspace(3.0, 2000.0, nb)
    cabs = W.cabs_model(1e-5, lam, "silicate")[None, :]
    E = W.debye_enthalpy(500.0, W.n_atoms(1e-5, "silicate"), T)
    wl = W.Workload("large grain", lam, np.array([1e-5]), ["silicate"], cabs, np.array([0, nb], dtype=np.int32),
                    T, E, np.ones(1), u=W.three_bb_fields(lam, np.array([1.0]), np.array([0.0]),
                                                          np.array([[0.3, 0.5, 0.2]])))
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        with pytest.raises(heat.HeatError) as e:
            lib.solve(want_j=False, **DISCRETE)
        assert e.value.status == heat.HEAT_EINVAL
        P, _ = lib.solve(want_j=False, build=heat.HEAT_BUILD_F64)
        assert abs(P.sum() - 1.0) < 1e-12
    finally:
        lib.close()
