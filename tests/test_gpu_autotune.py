"""Launch shapes the autotuner chooses among (heat_autotune, heat_get_tuning): each candidate,
forced through heat_opts, against the FP64 oracle at the path's tolerance, and the knobs
that must not change results (the recursion's resident blocks, the fused kernel) bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, masked_relerr

pytestmark = pytest.mark.gpu

MIXED = dict(build=heat.HEAT_BUILD_F32, j_dtype=heat.HEAT_F32)


@pytest.fixture(scope="module")
def sub():
    """7 grains spanning 128..1024 bins, 150 cells (ragged against the 128-cell M tiles), 300
    wavelengths (ragged against both tile widths)."""
    full = W.batched(cells=150, n_lambda=300)
    wl = W.grain_subset(full, [0, 5, 17, 30, 41, 52, 63])
    _, j_ref, _, st = oracle.solve_batch(W.field_subset(wl, np.arange(40)), oracle.grain_cooling(wl))
    assert st == oracle.OK
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, j_ref, lib
    lib.close()


@pytest.mark.parametrize("emis,tol", [(heat.HEAT_EMIS_BF16X3, 1e-4), (heat.HEAT_EMIS_TF32X3, 1e-5),
                                      (heat.HEAT_EMIS_BF16, 2e-2), (heat.HEAT_EMIS_TF32, 3e-3)])
@pytest.mark.parametrize("ntile", [128, 256])
def test_tensor_core_tile_widths_against_oracle(sub, emis, tol, ntile):
    """Each tile width and operand mode on the exact P (FP64 build): the contraction alone
    against the oracle, at the mode's bound (split modes keep ~16 or ~21 mantissa bits)."""
    wl, j_ref, lib = sub
    _, j = lib.solve(want_P=False, build=heat.HEAT_BUILD_F64, emis=emis, j_dtype=heat.HEAT_F64, emis_n_tile=ntile)
    assert masked_relerr(j[:40], j_ref) <= tol


@pytest.mark.parametrize("emis", [heat.HEAT_EMIS_BF16X3, heat.HEAT_EMIS_TF32X3])
def test_tile_widths_agree(sub, emis):
    """The same k order per output element: the two widths agree to FP32 rounding."""
    _, _, lib = sub
    _, a = lib.solve(want_P=False, emis=emis, emis_n_tile=128, **MIXED)
    _, b = lib.solve(want_P=False, emis=emis, emis_n_tile=256, **MIXED)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=0.0)


@pytest.mark.parametrize("bps", [1, 2, 3, 4])
def test_recursion_resident_blocks_do_not_change_results(sub, bps):
    _, _, lib = sub
    a = lib.solve(emis=heat.HEAT_EMIS_BF16X3, **MIXED)
    b = lib.solve(emis=heat.HEAT_EMIS_BF16X3, recur_blocks_per_sm=bps, **MIXED)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("pf", [1, 2])
def test_build_prefetch_does_not_change_results(sub, pf):
    """The FP32 build's pattern prefetch on or off: P and j bit for bit."""
    _, _, lib = sub
    a = lib.solve(emis=heat.HEAT_EMIS_BF16X3, **MIXED)
    b = lib.solve(emis=heat.HEAT_EMIS_BF16X3, build_prefetch=pf, **MIXED)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_launch_shape_option_checks(sub):
    _, _, lib = sub
    for kw in (dict(emis_n_tile=64), dict(recur_blocks_per_sm=5), dict(recur_blocks_per_sm=-1),
               dict(build_prefetch=3), dict(build_prefetch=-1)):
        with pytest.raises(heat.HeatError) as e:
            lib.solve(emis=heat.HEAT_EMIS_BF16X3, **kw, **MIXED)
        assert e.value.status == heat.HEAT_EINVAL


def test_tuned_solve_against_oracle(sub):
    import torch

    wl, j_ref, lib = sub
    j = torch.empty(wl.n_cells, wl.n_grains, wl.n_lambda, dtype=torch.float32, device="cuda")
    heat.heat_autotune(lib.ctx, heat.heat_default_opts(emis=heat.HEAT_EMIS_BF16X3, **MIXED), None, j,
                       torch.cuda.current_stream().cuda_stream)
    t = heat.heat_get_tuning(lib.ctx)
    assert t["streams"] >= 1
    _, jt = lib.solve(want_P=False, emis=heat.HEAT_EMIS_BF16X3, **MIXED)
    assert masked_relerr(jt[:40], j_ref) <= 1e-3
