"""Tensor-core emissivity (tcgen05) against the FP64 oracle and the FP64 GPU path."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, masked_relerr

pytestmark = pytest.mark.gpu

# Error bounds on j where j > 1e-6 of its peak (per spectrum).  Split modes keep ~16
# (BF16) or ~21 (TF32) mantissa bits per operand; single products keep 8 or 11.
TOL = {heat.HEAT_EMIS_BF16X3: 1e-4, heat.HEAT_EMIS_TF32X3: 1e-5, heat.HEAT_EMIS_BF16: 2e-2,
       heat.HEAT_EMIS_TF32: 3e-3}
MODES = list(TOL)


@pytest.fixture(scope="module")
def single():
    wl = W.single_cell()
    Cf = oracle.grain_cooling(wl)
    P, j, _, _ = oracle.solve_batch(wl, Cf)
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, P, j, lib
    lib.close()


@pytest.fixture(scope="module")
def ragged():
    """Batched grains 0, 7, 20, 45, 63; 77 cells (M tail); 300 wavelengths (N tail)."""
    lam = W.wavelength_grid(300)
    full = W.batched(cells=77, n_lambda=300)
    wl = W.grain_subset(full, [0, 7, 20, 45, 63])
    Cf = oracle.grain_cooling(wl)
    P, j, _, _ = oracle.solve_batch(wl, Cf)
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, P, j, lib
    lib.close()


@pytest.mark.parametrize("mode", MODES)
def test_tc_modes_single_cell(single, mode):
    wl, _, j, lib = single
    _, jg = lib.solve(want_P=False, build=heat.HEAT_BUILD_F64, emis=mode, j_dtype=heat.HEAT_F32)
    err = masked_relerr(jg, j)
    assert err <= TOL[mode], (heat.EMIS_NAMES[mode], err)


@pytest.mark.parametrize("mode", MODES)
def test_tc_modes_ragged_tiles(ragged, mode):
    wl, _, j, lib = ragged
    _, jg = lib.solve(want_P=False, build=heat.HEAT_BUILD_F64, emis=mode, j_dtype=heat.HEAT_F64)
    err = masked_relerr(jg, j)
    assert err <= TOL[mode], (heat.EMIS_NAMES[mode], err)


def test_mixed_path_meets_1e3(ragged):
    """FP32 build + FP64 recursion + BF16x3 tensor-core emissivity: <= 1e-3 on j."""
    wl, _, j, lib = ragged
    _, jg = lib.solve(want_P=False, build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32,
                      chunk_cells=32)
    assert masked_relerr(jg, j) <= 1e-3


def test_tc_matches_f64_path_where_it_matters(ragged):
    wl, _, _, lib = ragged
    _, j64 = lib.solve(want_P=False, build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_F64)
    _, jtc = lib.solve(want_P=False, build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_TF32X3)
    assert masked_relerr(jtc, j64) <= 1e-5


def test_tc_deterministic(ragged):
    wl, _, _, lib = ragged
    a = lib.solve(want_P=False, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32)[1]
    b = lib.solve(want_P=False, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32)[1]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mode", MODES)
def test_tc_size_integrated(ragged, mode):
    """Size-integrated output from one tensor-core GEMM over all grains' bins (Eq. convolution):
    J = sum_g w_g j_g against the oracle's per-grain spectra summed in FP64."""
    wl, _, j, lib = ragged
    Jref = oracle.size_integrate(wl.size_weight, j)
    _, J = lib.solve(want_P=False, build=heat.HEAT_BUILD_F64, emis=mode, j_dtype=heat.HEAT_F32, size_integrate=1)
    assert J.shape == Jref.shape
    err = masked_relerr(J, Jref)
    assert err <= TOL[mode], (heat.EMIS_NAMES[mode], err)


def test_mixed_size_integrated_meets_1e3(ragged):
    wl, _, j, lib = ragged
    Jref = oracle.size_integrate(wl.size_weight, j)
    _, J = lib.solve(want_P=False, build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32,
                     size_integrate=1, chunk_cells=64)
    assert masked_relerr(J, Jref) <= 1e-3
