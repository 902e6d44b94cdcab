"""Drive libheat through its C ABI from the tests (device buffers from torch)."""
import numpy as np

from paper_1311_4627_gb300 import heat


def relerr(got, ref, floor=1e-280):
    """Max relative error over |ref| > floor; entries below must agree to 1e-290 absolute."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    big = np.abs(ref) > floor
    small_ok = np.all(np.abs(got[~big] - ref[~big]) <= 1e-290) if np.any(~big) else True
    r = np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big])) if np.any(big) else 0.0
    return float(r), bool(small_ok)


def masked_relerr(got, ref, rel_floor=1e-6):
    """Max relative error of j over lambda where ref > rel_floor * max_lambda(ref), per spectrum."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    peak = ref.max(axis=-1, keepdims=True)
    m = ref > rel_floor * peak
    return float(np.max(np.abs(got[m] - ref[m]) / ref[m]))


class Lib:
    """One context per workload; solve() returns numpy results."""

    def __init__(self, wl, device=0):
        import torch

        self.torch = torch
        self.wl = wl
        self.ctx = heat.heat_create_grid(device, wl.lam)
        heat.heat_set_grains(self.ctx, wl.radius, wl.cabs, wl.bin_off, wl.T, wl.E, wl.size_weight)
        self.u = None

    def set_fields(self, u, dtype=heat.HEAT_F64):
        torch = self.torch
        tdt = torch.float64 if dtype == heat.HEAT_F64 else torch.float32
        self.u = torch.from_numpy(np.ascontiguousarray(u)).to(device="cuda", dtype=tdt)
        heat.heat_set_fields(self.ctx, self.u.shape[0], self.u, dtype, 1, torch.cuda.current_stream().cuda_stream)

    def solve(self, want_P=True, want_j=True, **opts):
        torch = self.torch
        o = heat.heat_default_opts(**opts)
        wl = self.wl
        cells = (o.cell_count if o.cell_count > 0 else self.u.shape[0] - o.cell_begin)
        P = torch.empty(cells, wl.total_bins, dtype=torch.float64, device="cuda") if want_P else None
        jdt = torch.float64 if o.j_dtype == heat.HEAT_F64 else torch.float32
        jshape = (cells, wl.n_lambda) if o.size_integrate else (cells, wl.n_grains, wl.n_lambda)
        j = torch.empty(*jshape, dtype=jdt, device="cuda") if want_j else None
        if not want_j:
            o.emis = heat.HEAT_EMIS_NONE
        heat.heat_solve(self.ctx, o, P, j, torch.cuda.current_stream().cuda_stream)
        heat.heat_sync(self.ctx)
        return (None if P is None else P.cpu().numpy(), None if j is None else j.cpu().numpy().astype(np.float64))

    def cooling(self):
        return heat.heat_get_cooling(self.ctx, self.wl.total_bins)

    def close(self):
        heat.heat_destroy(self.ctx)
        self.ctx = None
