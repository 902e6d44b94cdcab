"""heat_solve_noalloc (no device allocation, static scratch) against heat_solve.

The no-allocation entry point serves callers that cannot allocate device memory in
their loop (a fixed memory budget owned by their own allocator, or a loop that cannot
afford cudaMalloc/cudaFree waiting for the whole device).  It must give the same P as
heat_solve, on every call, although all calls share one static scratch array.
This file sorts last so that a run stopping at the first failure has run the rest.
"""
import numpy as np
import pytest

from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib, relerr

pytestmark = pytest.mark.gpu

EXACT_TOL = 1e-10


@pytest.fixture(scope="module")
def lib200():
    # 7 grains of 128..1024 bins and 200 cells: several 32-cell groups, a ragged last
    # group, and more groups than fit the static scratch at once for the FP64 build.
    wl = W.grain_subset(W.batched(cells=200), [0, 5, 17, 30, 41, 52, 63])
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, lib
    lib.close()


@pytest.mark.parametrize("build", [heat.HEAT_BUILD_F64, heat.HEAT_BUILD_F32])
def test_noalloc_matches_heat_solve_on_two_calls(lib200, build):
    import torch

    wl, lib = lib200
    P_ref, _ = lib.solve(want_j=False, build=build)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        P = torch.full((wl.n_cells, wl.total_bins), float("nan"), dtype=torch.float64, device="cuda")
        heat.heat_solve_noalloc(lib.ctx, build, lib.u, wl.n_cells, P, stream)
        heat.heat_sync(lib.ctx)
        Pg = P.cpu().numpy()
        assert np.all(np.isfinite(Pg)), f"call {call}: unwritten output"
        r, ok = relerr(Pg, P_ref)
        assert ok and r <= EXACT_TOL, (call, r)


@pytest.mark.parametrize("n_cells", [1, 16])
@pytest.mark.parametrize("build", [heat.HEAT_BUILD_F64, heat.HEAT_BUILD_F32])
def test_noalloc_small_solves_match_heat_solve(lib200, build, n_cells):
    """At most 16 cells take the element-parallel build and recursion in both entry points;
    the no-allocation call must pick them too and give heat_solve's P on two calls."""
    import torch

    wl, lib = lib200
    P_ref, _ = lib.solve(want_j=False, build=build, cell_count=n_cells)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        P = torch.full((n_cells, wl.total_bins), float("nan"), dtype=torch.float64, device="cuda")
        heat.heat_solve_noalloc(lib.ctx, build, lib.u, n_cells, P, stream)
        heat.heat_sync(lib.ctx)
        Pg = P.cpu().numpy()
        assert np.all(np.isfinite(Pg)), f"call {call}: unwritten output"
        r, ok = relerr(Pg, P_ref)
        assert ok and r <= EXACT_TOL, (call, r)


def test_noalloc_argument_errors_carry_a_message(lib200):
    import torch

    wl, lib = lib200
    P = torch.zeros((4, wl.total_bins), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(heat.HeatError) as ei:
        heat.heat_solve_noalloc(lib.ctx, 7, lib.u, 4, P, stream)
    assert ei.value.status == heat.HEAT_EINVAL and "build" in str(ei.value)
    with pytest.raises(heat.HeatError) as ei:
        heat.heat_solve_noalloc(lib.ctx, heat.HEAT_BUILD_F64, None, 4, P, stream)
    assert ei.value.status == heat.HEAT_EINVAL and "null" in str(ei.value)


def test_noalloc_rejects_grains_beyond_the_static_scratch():
    import torch

    wl = W.batched(cells=32)  # 64 grains x 1024 wavelengths: one FP64 group needs ~69 MB
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        P = torch.zeros((32, wl.total_bins), dtype=torch.float64, device="cuda")
        with pytest.raises(heat.HeatError) as ei:
            heat.heat_solve_noalloc(lib.ctx, heat.HEAT_BUILD_F64, lib.u, 32, P, torch.cuda.current_stream().cuda_stream)
        assert ei.value.status == heat.HEAT_EINVAL
        assert "HEAT_NOALLOC_SCRATCH_BYTES" in str(ei.value)
        assert float(P.abs().sum()) == 0.0  # nothing was queued
    finally:
        lib.close()
