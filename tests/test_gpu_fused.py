"""The fused build + recursion of the mixed path (heat_opts.fused_build = 1) against the
default two-kernel form (a build kernel writes the B band, the recursion reads it).

The fused kernel makes every B element from the same expressions, sums every prefix in the
same order and runs the recursion's FMAs in the same order, so P, j and the energy check
must agree bit for bit, on ragged cell counts, across chunkings, with tail pruning and at
the full size of the batched workload; and both stay within the mixed tolerance of the
FP64 oracle (the oracle comparisons of the default path live in the parity tests)."""
import numpy as np
import pytest

import oracle
from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, masked_relerr

pytestmark = pytest.mark.gpu

MIXED = dict(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32)


@pytest.fixture(scope="module")
def sub():
    """7 grains spanning 128..1024 bins, 77 cells (ragged against 32-cell groups)."""
    full = W.batched(cells=77)
    wl = W.grain_subset(full, [0, 5, 17, 30, 41, 52, 63])
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, lib
    lib.close()


def _ledger_solve(lib, wl, **opts):
    import torch

    led = torch.zeros(wl.n_cells, wl.n_grains, 2, dtype=torch.float64, device="cuda")
    P, j = lib.solve(ledger_out=led.data_ptr(), **opts)
    return P, j, led.cpu().numpy()


@pytest.mark.parametrize("chunk", [0, 32, 64])
@pytest.mark.parametrize("prune", [0.0, 1e-12])
def test_fused_is_bitwise_the_two_kernel_path(sub, chunk, prune):
    wl, lib = sub
    a = _ledger_solve(lib, wl, chunk_cells=chunk, prune_eps=prune, **MIXED)
    b = _ledger_solve(lib, wl, chunk_cells=chunk, prune_eps=prune, fused_build=1, **MIXED)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_fused_timing_classes(sub):
    """The fused solve launches no separate build kernel."""
    import torch

    wl, lib = sub
    heat.heat_get_timing(lib.ctx, reset=True)
    j = torch.empty(wl.n_cells, wl.n_grains, wl.n_lambda, dtype=torch.float32, device="cuda")
    heat.heat_solve(lib.ctx, heat.heat_default_opts(timing=1, fused_build=1, **MIXED), None, j,
                    torch.cuda.current_stream().cuda_stream)
    heat.heat_sync(lib.ctx)
    t = heat.heat_get_timing(lib.ctx, reset=True)
    assert t["build"][1] == 0 and t["recur"][1] >= 1


def test_fused_full_size_bitwise_and_against_oracle():
    """4096 cells x 64 grains, the benchmark's configuration: fused and two-kernel P agree bit
    for bit; sampled cells within 1e-3 of the oracle (j on the 1e-6 mask)."""
    import torch

    wl = W.batched()
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        st = torch.cuda.current_stream().cuda_stream
        out = []
        for fused in (1, 2):
            P = torch.empty(wl.n_cells, wl.total_bins, dtype=torch.float64, device="cuda")
            j = torch.empty(wl.n_cells, wl.n_grains, wl.n_lambda, dtype=torch.float32, device="cuda")
            heat.heat_solve(lib.ctx, heat.heat_default_opts(fused_build=fused, **MIXED), P, j, st)
            heat.heat_sync(lib.ctx)
            out.append((P, j))
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
        cells = np.array([0, 1000, 2047, 4095])
        Cf = oracle.grain_cooling(wl)
        _, jo, _, st_o = oracle.solve_batch(wl, Cf, u=wl.u[cells])
        assert st_o == oracle.OK
        got = out[0][1][cells].cpu().numpy().astype(np.float64)
        assert masked_relerr(got, jo) <= 1e-3
    finally:
        lib.close()


def test_fused_build_option_checks(sub):
    _, lib = sub
    with pytest.raises(heat.HeatError) as e:
        lib.solve(fused_build=3, **MIXED)
    assert e.value.status == heat.HEAT_EINVAL
