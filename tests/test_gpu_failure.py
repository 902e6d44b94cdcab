"""Failure detection on the GPU without a fault: bounded waits that give up.

The tensor-core kernels pass tiles between roles through shared-memory barriers, and
every wait on another role is bounded.  heat_set_wait_limit(ctx, 0) makes each such wait
give up at once, as a role whose partner never arrives would after the default limit:
the kernel must record HEAT_ETIMEOUT (reported by heat_sync), let its own copies and MMAs
finish, free its tensor memory and return, and the context must stay usable."""
import numpy as np
import pytest

from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    lam = W.wavelength_grid(256)
    base = W.batched(cells=48, n_lambda=256, grains=8)
    wl = W.custom(lam, base.radius, base.composition, [128] * 8, base.u)
    lib = Lib(wl)
    lib.set_fields(wl.u)
    yield wl, lib
    lib.close()


MIXED = dict(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32)


def test_emissivity_wait_gives_up_and_the_context_recovers(small):
    wl, lib = small
    P0, j0 = lib.solve(**MIXED)
    assert np.all(np.isfinite(j0)) and np.max(j0) > 0.0
    heat.heat_set_wait_limit(lib.ctx, 0)
    try:
        with pytest.raises(heat.HeatError) as ei:
            lib.solve(**MIXED)  # heat_sync inside reports the device status
        assert ei.value.status == heat.HEAT_ETIMEOUT
    finally:
        heat.heat_set_wait_limit(lib.ctx, heat.WAIT_POLLS_DEFAULT)
    # the status word was cleared by heat_sync; the same solve gives the same bits again
    P1, j1 = lib.solve(**MIXED)
    assert np.array_equal(P1, P0) and np.array_equal(j1, j0)


def test_surrogate_gemm_wait_gives_up_and_the_context_recovers(small):
    import torch

    wl, lib = small
    st = torch.cuda.current_stream().cuda_stream
    heat.heat_surrogate_init(lib.ctx, 2, np.zeros(wl.n_grains), seed=1)
    cells = 32
    j = torch.empty(cells, wl.n_grains, wl.n_lambda, dtype=torch.float32, device="cuda")
    heat.heat_solve(lib.ctx, heat.heat_default_opts(cell_count=cells, **MIXED), None, j, st)
    heat.heat_sync(lib.ctx)
    ns = cells * wl.n_grains
    X = torch.empty(ns, heat.SURROGATE_INPUTS, dtype=torch.float32, device="cuda")
    Y = torch.empty(ns, wl.n_lambda, dtype=torch.float32, device="cuda")
    lnp = torch.empty(ns, dtype=torch.float32, device="cuda")
    heat.heat_surrogate_samples(lib.ctx, 0, cells, j, X, Y, lnp, st)
    heat.heat_surrogate_fit_norm(lib.ctx, X, Y, ns, st)
    lnj = torch.empty(ns, wl.n_lambda, dtype=torch.float32, device="cuda")
    sp = torch.empty(ns, dtype=torch.float32, device="cuda")
    heat.heat_surrogate_predict(lib.ctx, X, lnp, ns, lnj, sp, st)
    heat.heat_sync(lib.ctx)
    ref = (lnj.cpu().numpy(), sp.cpu().numpy())
    heat.heat_set_wait_limit(lib.ctx, 0)
    try:
        heat.heat_surrogate_predict(lib.ctx, X, lnp, ns, lnj, sp, st)
        with pytest.raises(heat.HeatError) as ei:
            heat.heat_sync(lib.ctx)
        assert ei.value.status == heat.HEAT_ETIMEOUT
    finally:
        heat.heat_set_wait_limit(lib.ctx, heat.WAIT_POLLS_DEFAULT)
    heat.heat_surrogate_predict(lib.ctx, X, lnp, ns, lnj, sp, st)
    heat.heat_sync(lib.ctx)
    assert np.array_equal(lnj.cpu().numpy(), ref[0]) and np.array_equal(sp.cpu().numpy(), ref[1])


def test_wait_limit_rejects_negative_values(small):
    _, lib = small
    with pytest.raises(heat.HeatError) as ei:
        heat.heat_set_wait_limit(lib.ctx, -1)
    assert ei.value.status == heat.HEAT_EINVAL

