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


@pytest.mark.parametrize("streams,chunk,si", [(2, 32, 0), (3, 32, 1)])
def test_pipelined_host_solves_with_chunks_in_flight(streams, chunk, si):
    """Asynchronous host I/O with several chunks in flight on several slots (each with its own
    copy stream and staging sets), per-grain and size-integrated: two queued solves of
    different fields equal their synchronous solves bit for bit."""
    import torch

    full = W.batched(cells=100)
    wl = W.grain_subset(full, [2, 30, 63])
    G, N = wl.n_grains, wl.n_lambda
    ctx = heat.heat_create_grid(0, wl.lam)
    try:
        heat.heat_set_grains(ctx, wl.radius, wl.cabs, wl.bin_off, wl.T, wl.E, wl.size_weight)
        st = torch.cuda.Stream()
        sh = st.cuda_stream
        fields = [torch.from_numpy(np.ascontiguousarray(wl.u[::s])).pin_memory() for s in (1, -1)]
        shape = (wl.n_cells, N) if si else (wl.n_cells, G, N)
        outs = [torch.empty(*shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        kw = dict(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32, streams=streams,
                  chunk_cells=chunk, size_integrate=si)
        for k in range(2):
            heat.heat_set_fields(ctx, wl.n_cells, fields[k], heat.HEAT_F64, 0, sh)
            heat.heat_solve(ctx, heat.heat_default_opts(host_io=2, **kw), None, outs[k], sh)
        heat.heat_sync(ctx)
        for k in range(2):
            ref = torch.empty(*shape, dtype=torch.float32).pin_memory()
            heat.heat_set_fields(ctx, wl.n_cells, fields[k], heat.HEAT_F64, 0, sh)
            heat.heat_solve(ctx, heat.heat_default_opts(host_io=1, **kw), None, ref, sh)
            heat.heat_sync(ctx)
            assert torch.equal(outs[k], ref), k
    finally:
        heat.heat_destroy(ctx)
