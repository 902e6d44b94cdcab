"""Asynchronous host I/O (heat_opts.host_io = 2): a pipelined loop of solves on host buffers
gives the same bits as synchronous solves, with the two staging sets alternating."""
import numpy as np
import pytest

from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_pipelined_host_solves_match_synchronous_ones():
    """Three consecutive solves on different fields, each into its own pinned host buffers,
    queued without waiting (the copies of one overlap the kernels of the next), then one
    heat_sync: every result equals the synchronous solve of the same fields, bit for bit,
    for j, P and the energy ledger."""
    import torch

    full = W.batched(cells=96)
    wl = W.grain_subset(full, [0, 9, 21, 40, 63])
    G, N, nbt = wl.n_grains, wl.n_lambda, wl.total_bins
    ctx = heat.heat_create_grid(0, wl.lam)
    try:
        heat.heat_set_grains(ctx, wl.radius, wl.cabs, wl.bin_off, wl.T, wl.E, wl.size_weight)
        st = torch.cuda.Stream()
        sh = st.cuda_stream
        rng = np.random.default_rng(3)
        fields = [np.ascontiguousarray(wl.u[rng.permutation(wl.n_cells)]) for _ in range(3)]
        u_pin = [torch.from_numpy(f).pin_memory() for f in fields]
        outs = []
        for k in range(3):
            j = torch.empty(wl.n_cells, G, N, dtype=torch.float32).pin_memory()
            P = torch.empty(wl.n_cells, nbt, dtype=torch.float64).pin_memory()
            L = torch.empty(wl.n_cells, G, 2, dtype=torch.float64).pin_memory()
            outs.append((j, P, L))
        for k in range(3):
            j, P, L = outs[k]
            heat.heat_set_fields(ctx, wl.n_cells, u_pin[k], heat.HEAT_F64, 0, sh)
            o = heat.heat_default_opts(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32,
                                       host_io=2, ledger_out=L.data_ptr())
            heat.heat_solve(ctx, o, P, j, sh)
        heat.heat_sync(ctx)
        for k in range(3):
            j0 = torch.empty(wl.n_cells, G, N, dtype=torch.float32).pin_memory()
            P0 = torch.empty(wl.n_cells, nbt, dtype=torch.float64).pin_memory()
            L0 = torch.empty(wl.n_cells, G, 2, dtype=torch.float64).pin_memory()
            heat.heat_set_fields(ctx, wl.n_cells, u_pin[k], heat.HEAT_F64, 0, sh)
            o = heat.heat_default_opts(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32,
                                       host_io=1, ledger_out=L0.data_ptr())
            heat.heat_solve(ctx, o, P0, j0, sh)
            heat.heat_sync(ctx)
            j, P, L = outs[k]
            assert torch.equal(j, j0) and torch.equal(P, P0) and torch.equal(L, L0), k
        assert not torch.equal(outs[0][0], outs[1][0])
        with pytest.raises(heat.HeatError) as e:
            heat.heat_solve(ctx, heat.heat_default_opts(host_io=3), None, outs[0][0], sh)
        assert e.value.status == heat.HEAT_EINVAL
    finally:
        heat.heat_destroy(ctx)
