"""Solves captured into CUDA graphs: a replay gives the eager solve's bits, follows in-place
field updates, and covers multi-chunk, multi-stream solves."""
import numpy as np
import pytest

from paper_1311_4627_gb300 import heat
from paper_1311_4627_gb300 import workloads as W

from .gpu_helpers import Lib

pytestmark = pytest.mark.gpu


def _run_graph(lib, opts, want_P=True):
    import torch

    wl = lib.wl
    n = lib.u.shape[0]
    s = torch.cuda.Stream()
    P = torch.empty(n, wl.total_bins, dtype=torch.float64, device="cuda") if want_P else None
    j = torch.empty(n, wl.n_grains, wl.n_lambda, dtype=torch.float32, device="cuda")
    g = heat.Graph(lib.ctx, opts, P, j, s.cuda_stream)
    return g, s, P, j


def test_graph_replay_matches_eager_and_follows_fields():
    import torch

    wl = W.single_cell()
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        opts = heat.heat_default_opts(build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_F64, j_dtype=heat.HEAT_F32)
        P0, j0 = lib.solve(build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_F64, j_dtype=heat.HEAT_F32)
        g, s, P, j = _run_graph(lib, opts)
        assert g.kernel_nodes() >= 4
        P.zero_()
        j.zero_()
        torch.cuda.synchronize()  # the zeroing ran on torch's stream, the replay runs on s
        g.launch(s.cuda_stream)
        s.synchronize()
        heat.heat_sync(lib.ctx)
        assert np.array_equal(P.cpu().numpy(), P0) and np.array_equal(j.cpu().numpy().astype(np.float64), j0)
        # in-place field update: the replay reads the new values
        lib.u.mul_(3.0)
        torch.cuda.synchronize()
        g.launch(s.cuda_stream)
        s.synchronize()
        heat.heat_sync(lib.ctx)
        P3, j3 = P.cpu().numpy().copy(), j.cpu().numpy().astype(np.float64)
        torch.cuda.synchronize()
        heat.heat_set_fields(lib.ctx, 1, lib.u, heat.HEAT_F64, 1, torch.cuda.current_stream().cuda_stream)
        Pe, je = lib.solve(build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_F64, j_dtype=heat.HEAT_F32)
        assert np.array_equal(P3, Pe) and np.array_equal(j3, je)
        assert not np.array_equal(P3, P0)
        g.close()
    finally:
        lib.close()


def test_graph_of_pipelined_mixed_solve():
    full = W.batched(cells=160)
    wl = W.grain_subset(full, [3, 30, 60])
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        kw = dict(build=heat.HEAT_BUILD_F32, emis=heat.HEAT_EMIS_BF16X3, j_dtype=heat.HEAT_F32, streams=2,
                  chunk_cells=64)
        Pe, je = lib.solve(**kw)
        g, s, P, j = _run_graph(lib, heat.heat_default_opts(**kw))
        P.zero_()
        j.zero_()
        import torch

        torch.cuda.synchronize()
        for _ in range(3):
            g.launch(s.cuda_stream)
        s.synchronize()
        heat.heat_sync(lib.ctx)
        assert np.array_equal(P.cpu().numpy(), Pe) and np.array_equal(j.cpu().numpy().astype(np.float64), je)
        g.close()
    finally:
        lib.close()


def test_graph_rejects_timing_and_host_io():
    import torch

    wl = W.single_cell()
    lib = Lib(wl)
    try:
        lib.set_fields(wl.u)
        s = torch.cuda.Stream()
        for kw in (dict(timing=1), dict(host_io=1)):
            with pytest.raises(heat.HeatError):
                heat.Graph(lib.ctx, heat.heat_default_opts(**kw), None, None, s.cuda_stream)
    finally:
        lib.close()
