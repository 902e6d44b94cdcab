"""The few-cell recursion (solves of at most 16 cells: a column sweep, one block per spectrum)
in its launch shapes, against the FP64 oracle at the exact path's tolerance: one warp (every
band row narrower than 32), blocks of one row per thread (the single-cell workload, rows up
to 127 wide; a dense grain of 300 bins) and 1024 threads with up to four rows per thread (a
dense grain of 1100 bins);
with pruning and the energy check; and bit for bit against the lane-per-cell recursion."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, relerr

pytestmark = pytest.mark.gpu

EXACT_TOL = 1e-10
EXACT = dict(build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_F64, j_dtype=heat.HEAT_F64)


def _check(wl, cells=None, **opts):
    Cf = oracle.grain_cooling(wl)
    P, j, led, st = oracle.solve_batch(wl, Cf, want_ledger=True)
    assert st == oracle.OK
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        Pg, jg = lib.solve(**dict(EXACT, **opts))
        rP, okP = relerr(Pg, P)
        rj, okj = relerr(jg, j)
        assert okP and okj and rP <= EXACT_TOL and rj <= EXACT_TOL, (rP, rj)
        for g in range(wl.n_grains):
            np.testing.assert_allclose(Pg[:, wl.grain_slice(g)].sum(axis=1), 1.0, rtol=1e-13)
    finally:
        lib.close()


def test_one_warp_narrow_bands():
    """The three largest grains of the single cell: rows 1-4 wide, so 32 threads."""
    _check(W.grain_subset(W.single_cell(), [5, 6, 7]))


def test_four_warps_single_cell_and_few_cells():
    _check(W.single_cell())
    _check(W.field_subset(W.batched(cells=16, n_lambda=256), np.arange(16)))


def test_block_one_row_per_thread():
    """A 3.5 A grain on 300 bins: rows up to 299 wide, so 320 threads."""
    lam = W.wavelength_grid(256)
    _check(W.custom(lam, np.array([3.5e-8]), ["carbonaceous"], [300], W.single_cell().u))


def test_rows_wider_than_1024():
    """A 3.5 A grain on 1100 bins: every row reaches bin 0, so 1024 threads hold up to two
    rows each at once."""
    lam = W.wavelength_grid(256)
    base = W.single_cell()
    _check(W.custom(lam, np.array([3.5e-8]), ["carbonaceous"], [1100], base.u))


def test_energy_check_and_pruning():
    import torch

    wl = W.single_cell()
    Cf = oracle.grain_cooling(wl)
    _, _, led_ref, _ = oracle.solve_batch(wl, Cf, want_ledger=True)
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        led = torch.zeros(1, wl.n_grains, 2, dtype=torch.float64, device="cuda")
        lib.solve(ledger_out=led.data_ptr(), **EXACT)
        r, ok = relerr(led.cpu().numpy()[..., 1], led_ref[..., 1])
        assert ok and r <= EXACT_TOL, r
        P0, _ = lib.solve(want_j=False, **EXACT)
        Pp, _ = lib.solve(want_j=False, prune_eps=1e-12, **EXACT)
        big = P0 > 1e-6 * P0.max()
        assert np.max(np.abs(Pp[big] / P0[big] - 1.0)) < 1e-9
    finally:
        lib.close()


def test_same_bits_as_the_lane_per_cell_recursion():
    """17 cells take the lane-per-cell kernel, 16 the column sweep; rows are summed in the same
    order over the same B (FP32 build), so the 16 shared cells agree bit for bit."""
    wl = W.field_subset(W.batched(cells=17, n_lambda=256), np.arange(17))
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        opts = dict(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_F64, j_dtype=heat.HEAT_F64)
        P17, _ = lib.solve(want_j=False, **opts)
        P16, _ = lib.solve(want_j=False, cell_count=16, **opts)
        assert np.array_equal(P16, P17[:16])
    finally:
        lib.close()
