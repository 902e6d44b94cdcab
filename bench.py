#!/usr/bin/env python
"""Benchmark: cell x grain emissivity spectra/s on one GB300.

Workload (the batched configuration): 4096 cells x 64 grain radii (3.5 A - 1 um,
alternating carbonaceous / silicate), 128-1024 enthalpy bins per grain, 1024
wavelengths, three-blackbody fields with chi log-uniform in [1e-2, 1e4] and hardness
in [-1, 1] (seeded, synthetic).  One step = one heat_solve over all cells: field
tables, B-matrix build, FP64 recursion, renormalisation and the emissivity of every
(cell, grain) pair, with inputs resident in HBM.

Paths (``--path``):
  ``mixed``      FP32 matrix build, FP64 recursion, BF16x3 tensor-core emissivity (default)
  (``surrogate`` is measured after them: an MLP ensemble trained, untimed, on 1M
  spectra of other cells, with the mixed path as fallback for uncertain cells)
  ``mixed_tf32`` FP32 matrix build, FP64 recursion, TF32x3 tensor-core emissivity
  ``batched``    FP32 matrix build, FP64 recursion, FP64 emissivity
  ``exact``      FP64 everywhere (the plain path)
  ``mixed_pruned`` the mixed path with tail pruning (bins whose probability and emission
                 stay below 1e-12 of the spectrum's are not solved)
The headline line reports ``--path``; the other exact-method paths are timed after it
for the plain-vs-mixed comparison (``paths``), each with its error against the oracle.
The JSON line adds the roofline of the dominant kernel, an end-to-end number
through the C ABI with host buffers, the oracle timed on the host cores, and the
SM clocks sampled during the timed region.

``--impl reference`` times the FP64 oracle (plain C, OpenMP over spectra) on the
host cores on a bounded sample of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell×grain emissivity spectra/s on 1 GB300: plain vs mixed vs surrogate @ rel err"
UNIT = "spectra/s"
FP64_PEAK_TFLOPS = 1.25  # nominal dense FP64 of a GB300 (no measured figure in the peaks file)
PATHS = {  # name: (build, emissivity, description, dtype)
    "mixed": ("f32", "bf16x3", "FP32 build, FP64 recursion, BF16x3 tensor-core emissivity", "f32+f64+bf16"),
    "mixed_tf32": ("f32", "tf32x3", "FP32 build, FP64 recursion, TF32x3 tensor-core emissivity", "f32+f64+tf32"),
    "batched": ("f32", "f64", "FP32 build, FP64 recursion, FP64 emissivity", "f32+f64"),
    "exact": ("f64", "f64", "FP64 build, FP64 recursion, FP64 emissivity", "f64"),
    "mixed_pruned": ("f32", "bf16x3", "mixed, with tail pruning at eps = 1e-12 (heat_opts.prune_eps)", "f32+f64+bf16"),
}
PRUNE_EPS = {"mixed_pruned": 1e-12}
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="mixed", choices=list(PATHS))
    ap.add_argument("--cells", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="time only --path")
    ap.add_argument("--no-surrogate", action="store_true", help="skip training and timing the surrogate path")
    ap.add_argument("--sur-cells", type=int, default=16384, help="training cells for the surrogate (x 64 grains)")
    ap.add_argument("--sur-epochs", type=int, default=30)
    ap.add_argument("--sur-tol", type=float, default=1e-2, help="ensemble spread (ln j) above which a cell falls back")
    ap.add_argument("--oracle-cells", type=int, default=96, help="cells in the oracle sample (about 12 s on 16 cores)")
    ap.add_argument("--no-single-cell", action="store_true", help="skip the single-cell latency section")
    ap.add_argument("--no-point", action="store_true", help="skip the point-rule heating section")
    ap.add_argument("--no-emis-heavy", action="store_true",
                    help="skip the emissivity-heavy workload (65536 cells x 32 grains x 512 bins x 2048 wavelengths)")
    ap.add_argument("--no-rt-volume", action="store_true", help="skip the RT-volume chunks section")
    ap.add_argument("--no-discrete", action="store_true", help="skip the thermal-discrete cooling section")
    ap.add_argument("--emis-heavy-oracle-cells", type=int, default=256,
                    help="cells of the emissivity-heavy workload checked against the oracle")
    return ap.parse_args()


# ---------------------------------------------------------------------------- utils
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def recorded_traffic(kernel, cells, launches_per_step):
    """DRAM bytes per launch of `kernel` from the committed ncu record (profiles/traffic.json),
    or None when there is none for this kernel and size or the kernel's source changed since."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "traffic.json")
    name = {"recur": "k_recur"}.get(kernel)
    if not name or not os.path.exists(p) or cells != 4096 or launches_per_step != 1:
        return None
    with open(p) as f:
        rec = json.load(f).get(name)
    if not rec:
        return None
    with open(os.path.join(ROOT, rec["source"]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != rec["source_sha256_prefix"]:
            return None
    return rec["bytes_per_launch_4096_cells"]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------- oracle leg
def oracle_sample(wl, n_cells, Cf=None):
    """Time the FP64 oracle on the first n_cells cells x all grains (cooling untimed)."""
    import oracle

    from paper_1311_4627_gb300 import workloads as W

    if Cf is None:
        Cf = oracle.grain_cooling(wl)
    sub = W.field_subset(wl, np.arange(n_cells))
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    P, j, _, st = oracle.solve_batch(sub, Cf)
    dt = time.perf_counter() - t0
    spectra = n_cells * wl.n_grains
    # one core: the first cell's spectra on a single thread
    sub1 = W.field_subset(wl, np.arange(1))
    t1 = time.perf_counter()
    oracle.solve_batch(sub1, Cf, n_threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": spectra / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_cells} cells x {wl.n_grains} grains of the workload ({spectra} spectra, "
                      f"{dt:.1f} s, OpenMP over spectra; cooling set-up untimed)",
            "one_core": {"value": wl.n_grains / dt1, "unit": UNIT,
                         "sample": f"1 cell x {wl.n_grains} grains on one thread ({dt1:.1f} s)"},
            "status": st}, P, j, Cf


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    from paper_1311_4627_gb300 import workloads as W

    wl = W.batched(cells=args.cells)
    Cf = oracle.grain_cooling(wl)
    per_step = 2  # cells per step: a bounded sample of the workload (~1 s of CPU work)
    times = []
    for s in range(args.warmup + args.steps):
        cells = np.arange(s * per_step, (s + 1) * per_step) % wl.n_cells
        sub = W.field_subset(wl, cells)
        t0 = time.perf_counter()
        oracle.solve_batch(sub, Cf)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    spectra = per_step * wl.n_grains
    ms = 1e3 * float(np.mean(times))
    value = spectra / (ms / 1e3)
    cores = oracle.max_threads()
    sample = f"{per_step} cells x {wl.n_grains} grains per step (of {wl.n_cells} cells)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, "oracle FP64 (CPU)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def workload_config(wl, path):
    nb = np.diff(wl.bin_off)
    return {"workload": f"batched: {wl.n_cells} cells x {wl.n_grains} grains (3.5 A-1 um), "
                        f"{int(nb.min())}-{int(nb.max())} bins, {wl.n_lambda} wavelengths",
            "cells": wl.n_cells, "grains": wl.n_grains, "bins_total": int(wl.total_bins), "n_lambda": wl.n_lambda,
            "path": path}


# ---------------------------------------------------------------------------- single-cell latency
def point_rule_section(args, wl, ctx, heat, timed_run, opts_for, dev, sh, Cf_oracle):
    """The paper's point-rule heating (Eq. heating at the bin centres) against the integral
    form on the same workload: exact path timing, error against the oracle's point mode on a
    small sample, and the energy check (model emitted / physical absorbed power) by grain
    size, which shows the heating the point rule drops for grains whose bins are wider than
    the photons."""
    import torch

    import oracle

    cells, G, nbt = wl.n_cells, wl.n_grains, wl.total_bins
    k2 = max(2, args.steps // 2)
    ms_p, _, kt_p, _, _ = timed_run("exact", k2, 1, heating=heat.HEAT_HEATING_POINT)
    out = {"spectra_per_s": cells * G / (ms_p / 1e3), "ms_per_step": ms_p,
           "kernels_ms_per_step": {k: v[0] / k2 for k, v in kt_p.items()},
           "precision": "FP64 point-rule build, FP64 recursion, FP64 emissivity"}
    led = {}
    for name, h in (("point", heat.HEAT_HEATING_POINT), ("integral", heat.HEAT_HEATING_INTEGRAL)):
        lg = torch.zeros(cells, G, 2, dtype=torch.float64, device=dev)
        heat.heat_solve(ctx, heat.heat_default_opts(emis=heat.HEAT_EMIS_NONE, heating=h, ledger_out=lg), None, None, sh)
        heat.heat_sync(ctx)
        led[name] = lg.cpu().numpy()
    classes = {"a<25A": wl.radius < 25e-8, "25A<=a<100A": (wl.radius >= 25e-8) & (wl.radius < 100e-8),
               "a>=100A": wl.radius >= 100e-8}
    ratio = {}
    for name, lg in led.items():
        r = lg[..., 1] / lg[..., 0]
        ratio[name] = {c: float(np.median(r[:, m])) for c, m in classes.items() if m.any()}
    out["median_emitted_over_absorbed"] = ratio
    if args.no_cpu_baseline:  # the oracle runs only in the CPU-baseline leg
        return out
    nsub = min(4, cells)
    sub_P = torch.empty(nsub, nbt, dtype=torch.float64, device=dev)
    o = opts_for("exact", cell_count=nsub, heating=heat.HEAT_HEATING_POINT)
    o.emis = heat.HEAT_EMIS_NONE
    heat.heat_solve(ctx, o, sub_P, None, sh)
    heat.heat_sync(ctx)
    P_ref, _, _, st = oracle.solve_batch(wl, Cf_oracle, want_j=False, u=wl.u[:nsub], heating=oracle.HEATING_POINT)
    Pg = sub_P.cpu().numpy()
    m = np.abs(P_ref) > 1e-280
    out["max_rel_err"] = {"P": float(np.max(np.abs(Pg[m] - P_ref[m]) / np.abs(P_ref[m]))), "oracle_status": int(st),
                          "sample": f"{nsub} cells x {G} grains vs the FP64 oracle's point mode"}
    return out


def single_cell_section(dev, stream):
    """One cell x 8 carbonaceous grains x 128 bins x 256 wavelengths: microseconds per
    heat_solve, launched eagerly and replayed from a CUDA graph, for the exact and the
    mixed path (a latency-bound solve: the roofline does not apply)."""
    import torch

    from paper_1311_4627_gb300 import heat
    from paper_1311_4627_gb300 import workloads as W

    wl = W.single_cell()
    ctx = heat.heat_create_grid(dev.index, wl.lam)
    heat.heat_set_grains(ctx, wl.radius, wl.cabs, wl.bin_off, wl.T, wl.E, wl.size_weight)
    s = torch.cuda.Stream(dev)
    sh = s.cuda_stream
    u = torch.from_numpy(wl.u).to(dev)
    heat.heat_set_fields(ctx, 1, u, heat.HEAT_F64, 1, sh)
    P = torch.empty(1, wl.total_bins, dtype=torch.float64, device=dev)
    j = torch.empty(1, wl.n_grains, wl.n_lambda, dtype=torch.float32, device=dev)
    out = {"workload": f"single cell x {wl.n_grains} grains, 128 bins, {wl.n_lambda} wavelengths", "paths": {}}
    reps = 200
    for name, b, e in (("exact", heat.HEAT_BUILD_F64, heat.HEAT_EMIS_F64),
                       ("mixed", heat.HEAT_BUILD_F32, heat.HEAT_EMIS_BF16X3)):
        o = heat.heat_default_opts(build=b, emis=e, j_dtype=heat.HEAT_F32)
        for _ in range(5):
            heat.heat_solve(ctx, o, P, j, sh)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            heat.heat_solve(ctx, o, P, j, sh)
        e1.record(s)
        torch.cuda.synchronize(dev)
        eager_us = e0.elapsed_time(e1) * 1e3 / reps
        g = heat.Graph(ctx, o, P, j, sh)
        for _ in range(5):
            g.launch(sh)
        torch.cuda.synchronize(dev)
        e0.record(s)
        for _ in range(reps):
            g.launch(sh)
        e1.record(s)
        torch.cuda.synchronize(dev)
        graph_us = e0.elapsed_time(e1) * 1e3 / reps
        nodes = g.kernel_nodes()
        g.close()
        heat.heat_get_timing(ctx, reset=True)  # per-kernel-class times of eager solves
        for _ in range(reps):
            heat.heat_solve(ctx, heat.heat_default_opts(build=b, emis=e, j_dtype=heat.HEAT_F32, timing=1), P, j, sh)
        heat.heat_sync(ctx)
        kt = heat.heat_get_timing(ctx, reset=True)
        out["paths"][name] = {"eager_us_per_solve": eager_us, "graph_us_per_solve": graph_us,
                              "graph_kernel_nodes": nodes,
                              "spectra_per_s_graph": wl.n_grains / (graph_us * 1e-6),
                              "kernels_us_per_solve": {k: v[0] * 1e3 / reps for k, v in kt.items() if v[1]}}
    heat.heat_sync(ctx)
    heat.heat_destroy(ctx)
    return out


# ---------------------------------------------------------------------------- thermal-discrete cooling
def thermal_discrete_section(dev):
    """Thermal-discrete cooling (heat_opts.cooling = HEAT_COOLING_DISCRETE, exact FP64 path):
    the single cell (8 grains x 128 bins, latency), 32 cells of the batched workload (64
    grains, 128-1024 bins; their rate matrices are banded for the larger grains) and a dense
    case for the state reduction's roofline (the 3.5 A grain, 128 bins, 87 % of its upward and
    all its downward rates non-zero, dense after fill-in; 1216 cells = 8 spectra per SM).  Each solve is timed with CUDA events, the kernels with the
    library's per-class events (build = rate matrices, recur = state reduction); P and j are
    compared with the FP64 oracle's thermal-discrete solve on every spectrum of the single cell
    and on 2 cells x 4 grains of the batched case."""
    import torch

    import oracle
    from paper_1311_4627_gb300 import heat
    from paper_1311_4627_gb300 import workloads as W

    def solve(wl, reps):
        ctx = heat.heat_create_grid(dev.index, wl.lam)
        heat.heat_set_grains(ctx, wl.radius, wl.cabs, wl.bin_off, wl.T, wl.E, wl.size_weight)
        s = torch.cuda.Stream(dev)
        sh = s.cuda_stream
        u = torch.from_numpy(wl.u).to(dev)  # the library keeps this pointer: u lives until the ctx is gone
        heat.heat_set_fields(ctx, wl.n_cells, u, heat.HEAT_F64, 1, sh)
        P = torch.empty(wl.n_cells, wl.total_bins, dtype=torch.float64, device=dev)
        j = torch.empty(wl.n_cells, wl.n_grains, wl.n_lambda, dtype=torch.float64, device=dev)
        kw = dict(build=heat.HEAT_BUILD_F64, emis=heat.HEAT_EMIS_F64, j_dtype=heat.HEAT_F64,
                  cooling=heat.HEAT_COOLING_DISCRETE)
        for _ in range(3):
            heat.heat_solve(ctx, heat.heat_default_opts(**kw), P, j, sh)
        heat.heat_sync(ctx)
        heat.heat_get_timing(ctx, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(s)
        for _ in range(reps):
            heat.heat_solve(ctx, heat.heat_default_opts(timing=1, **kw), P, j, sh)
        e1.record(s)
        torch.cuda.synchronize(dev)
        heat.heat_sync(ctx)
        ms = e0.elapsed_time(e1) / reps
        kt = heat.heat_get_timing(ctx, reset=True)
        out = P.cpu().numpy(), j.cpu().numpy()
        heat.heat_destroy(ctx)
        return ms, {k: v[0] / reps for k, v in kt.items() if v[1]}, out

    def errors(wl_ref, Pg, jg):
        P_ref, j_ref = oracle.solve_batch_discrete(wl_ref)[:2]
        okP = P_ref > 1e-280
        okj = np.abs(j_ref) > 1e-280
        return {"P": float(np.max(np.abs(Pg[okP] - P_ref[okP]) / P_ref[okP])),
                "j": float(np.max(np.abs(jg[okj] - j_ref[okj]) / np.abs(j_ref[okj])))}

    out = {"path": "exact FP64 (FP64 rate matrices, state reduction, FP64 emissivity)"}
    wl = W.single_cell()
    ms, kt, (Pg, jg) = solve(wl, 20)
    out["single_cell"] = {"workload": f"single cell x {wl.n_grains} grains, 128 bins, {wl.n_lambda} wavelengths",
                          "us_per_solve": ms * 1e3, "kernels_us_per_solve": {k: v * 1e3 for k, v in kt.items()},
                          "max_rel_err": errors(wl, Pg, jg),
                          "err_sample": "all 8 spectra vs the FP64 oracle (P > 1e-280, |j| > 1e-280)"}

    full = W.batched(cells=32)
    ms, kt, (Pg, jg) = solve(full, 2)
    cells, grains = [0, 31], [0, 21, 42, 63]
    sub = W.grain_subset(W.field_subset(full, cells), grains)
    cols = np.concatenate([np.arange(full.bin_off[g], full.bin_off[g + 1]) for g in grains])
    out["batched_32_cells"] = {
        "workload": "32 cells x 64 grains (3.5 A - 1 um), 128-1024 bins, 1024 wavelengths",
        "ms_per_solve": ms, "spectra_per_s": 32 * full.n_grains / (ms * 1e-3),
        "kernels_ms_per_solve": kt,
        "max_rel_err": errors(sub, Pg[cells][:, cols], jg[cells][:, grains]),
        "err_sample": "cells 0 and 31 x grains 0, 21, 42, 63 (128, 416, 704, 1024 bins) vs the FP64 oracle"}

    dense = W.grain_subset(W.batched(cells=1216, n_lambda=256), [0])
    M = dense.bins(0)
    ms, kt, (Pg, jg) = solve(dense, 5)
    fma_red = (M - 2) * (M - 1) * M / 3.0  # removing state n updates n(n-1) rates, n = 1..M-1
    work = 2.0 * dense.n_cells * (fma_red + M * (M - 1) / 2.0)
    ach = work / (kt["recur"] * 1e-3) / 1e12
    out["dense_roofline"] = {
        "workload": f"{dense.n_cells} cells x the 3.5 A grain ({M} bins, dense after fill-in), 256 wavelengths",
        "ms_per_solve": ms, "kernels_ms_per_solve": kt,
        "roofline": {"kernel": "state reduction (k_gth)", "bound": "alu", "unit": "TFLOP/s",
                     "achieved": ach, "peak": FP64_PEAK_TFLOPS, "frac": ach / FP64_PEAK_TFLOPS,
                     "frac_of_measured": ach / heat.heat_measure_fma_peak(dev.index, True),
                     "peak_source": "nominal dense FP64 1.25 TFLOP/s (profiling recipe table)",
                     "algorithmic_work": f"2 x cells x ((M-2)(M-1)M/3 + M(M-1)/2) = {work:.3e} FP64 flop per solve "
                                         "(reduction updates + back substitution)"}}
    return out


# ---------------------------------------------------------------------------- emissivity-heavy workload
def emissivity_heavy_section(args, dev, stream, peaks, peaks_src):
    """65536 cells x 32 carbonaceous grains x 512 bins x 2048 wavelengths, per-grain FP32
    output (17 GB): the BF16x3 and TF32x3 tensor-core paths timed, their error measured on
    a seeded subsample against the oracle, and the emissivity kernel's roofline."""
    import torch

    import oracle
    from paper_1311_4627_gb300 import heat
    from paper_1311_4627_gb300 import workloads as W

    sh = stream.cuda_stream
    wl = W.emissivity_heavy()
    cells, G, N, nbt = wl.n_cells, wl.n_grains, wl.n_lambda, wl.total_bins
    ctx = heat.heat_create_grid(dev.index, wl.lam)
    heat.heat_set_grains(ctx, wl.radius, wl.cabs, wl.bin_off, wl.T, wl.E, wl.size_weight)
    u = torch.from_numpy(wl.u).to(dev)
    heat.heat_set_fields(ctx, cells, u, heat.HEAT_F64, 1, sh)
    j = torch.empty(cells, G, N, dtype=torch.float32, device=dev)
    out = {"workload": f"emissivity-heavy: {cells} cells x {G} grains (3.5 A-1 um, carbonaceous), 512 bins, "
                       f"{N} wavelengths; per-grain FP32 j ({j.numel() * 4 / 1e9:.1f} GB written per step)",
           "band_elements_per_cell": heat.heat_band_elements(ctx), "paths": {}}
    nsub = args.emis_heavy_oracle_cells
    # the error subsample: seeded cells spread over the whole workload
    sub_cells = np.sort(np.random.default_rng(1003).choice(cells, size=nsub, replace=False))
    Cf = oracle.grain_cooling(wl)
    t0 = time.perf_counter()
    _, j_ref, _, _ = oracle.solve_batch(W.field_subset(wl, sub_cells), Cf)
    ot = time.perf_counter() - t0
    out["oracle"] = {"spectra_per_s": nsub * G / ot, "cores": oracle.max_threads(),
                     "sample": f"{nsub} seeded cells (PCG64 seed 1003) x {G} grains"}
    for name, emis in (("mixed", heat.HEAT_EMIS_BF16X3), ("mixed_tf32", heat.HEAT_EMIS_TF32X3)):
        o = heat.heat_default_opts(build=heat.HEAT_BUILD_F32, emis=emis, j_dtype=heat.HEAT_F32)
        heat.heat_solve(ctx, o, None, j, sh)
        heat.heat_sync(ctx)
        heat.heat_get_timing(ctx, reset=True)
        steps = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            heat.heat_solve(ctx, heat.heat_default_opts(build=heat.HEAT_BUILD_F32, emis=emis, j_dtype=heat.HEAT_F32,
                                                        timing=1), None, j, sh)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        heat.heat_sync(ctx)
        ms = e0.elapsed_time(e1) / steps
        kt = heat.heat_get_timing(ctx, reset=True)
        emis_ms, emis_n = kt["emis"]
        flop = 2.0 * cells * nbt * N
        tf32 = emis == heat.HEAT_EMIS_TF32X3
        pk = peaks["bf16_tflops"] / (2.0 if tf32 else 1.0)
        step_emis_s = emis_ms / steps / 1e3  # all emissivity launches of one step (chunks x launches)
        ach = flop / step_emis_s / 1e12
        bytes_out = 4.0 * cells * G * N
        gbs = bytes_out / step_emis_s / 1e9
        # the subsample's spectra from the timed solve's output (the whole workload, FP32 j)
        jg = j[torch.from_numpy(sub_cells).to(dev)].double().cpu().numpy()
        peak = j_ref.max(axis=-1, keepdims=True)
        m = j_ref > 1e-6 * peak
        err = float(np.max(np.abs(jg[m] - j_ref[m]) / j_ref[m]))
        out["paths"][name] = {
            "spectra_per_s": cells * G / (ms / 1e3), "ms_per_step": ms,
            "kernels_ms_per_step": {k: v[0] / steps for k, v in kt.items()},
            "emis_roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": pk, "frac": ach / pk,
                              "launches_per_step": emis_n / steps,
                              "peak_source": ("measured bf16 burst" + (" x 1/2 (nominal tf32:bf16)" if tf32 else "")
                                              + f" ({peaks_src})"),
                              "algorithmic_work": f"2 x cells x bins x wavelengths = {flop:.3e} flop per step",
                              "output_write_gbs": gbs, "output_write_frac_of_hbm": gbs / peaks["hbm_gbs"]},
            "max_rel_err_j_masked_1e-6_peak": err,
            "error_sample": f"{nsub} seeded cells x {G} grains of the timed solve's j against the FP64 oracle"}
    heat.heat_destroy(ctx)
    del j, u
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------- RT-volume chunks
def rt_volume_section(dev):
    """RT-volume workload (128 x 128 x 64 cells of Gaussian-random-field chi and hardness, 2
    compositions x 40 radii, 512 bins, 1024 wavelengths), run as the volume driver runs it:
    chunks of 65536 cells, fields copied in from pinned host memory, the mixed path with
    size-integrated output and the energy ledger, J copied back.  One warm-up chunk, then two
    timed chunks (device events around copies and solve; the fields are made on the host
    beforehand, as the driver makes them a chunk ahead)."""
    from paper_1311_4627_gb300 import volume as V
    from paper_1311_4627_gb300 import workloads as W

    t0 = time.perf_counter()
    vol = W.rt_volume((128, 128, 64), radii_per_composition=40, nbins=512, n_lambda=1024)
    chunk = 65536
    solver = V.VolumeSolver(vol, chunk, device=dev.index)
    setup_s = time.perf_counter() - t0
    solver.solve_chunk(0, 0, chunk, solver.prepare(0, chunk))
    infos = []
    for k in (1, 2):
        prep = solver.prepare(k * chunk, (k + 1) * chunk)
        _, info = solver.solve_chunk(k, k * chunk, (k + 1) * chunk, prep)
        infos.append(info)
    solver.close()
    gpu_s = sum(i["gpu_ms"] for i in infos) / 1e3
    spectra = sum(i["spectra"] for i in infos)
    return {"workload": f"RT volume 128x128x64 cells, {vol.grains.n_grains} grains, 512 bins, 1024 wavelengths; "
                        f"2 timed chunks of {chunk} cells (after one warm-up chunk)",
            "spectra_per_s": spectra / gpu_s, "gpu_ms_per_chunk": [i["gpu_ms"] for i in infos],
            "path": "mixed (FP32 build, FP64 recursion, BF16x3 tcgen05), size-integrated J, energy ledger",
            "energy_check": [i["energy"] for i in infos], "setup_s": round(setup_s, 2),
            "timing": "device events around field copy-in, solve and J copy-out of each chunk"}


# ---------------------------------------------------------------------------- GPU leg
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    import __graft_entry__

    __graft_entry__.build()
    from paper_1311_4627_gb300 import heat
    from paper_1311_4627_gb300 import workloads as W

    wl = W.batched(cells=args.cells)
    if rank > 0:  # each rank solves its own cells (weak scaling): a seeded permutation of the fields
        rng = np.random.Generator(np.random.PCG64(5000 + rank))
        wl.u = np.ascontiguousarray(wl.u[rng.permutation(wl.n_cells)])
    G, N, cells = wl.n_grains, wl.n_lambda, wl.n_cells
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream

    t0 = time.perf_counter()
    ctx = heat.heat_create_grid(local, wl.lam)
    heat.heat_set_grains(ctx, wl.radius, wl.cabs, wl.bin_off, wl.T, wl.E, wl.size_weight)
    setup_s = time.perf_counter() - t0
    band = heat.heat_band_elements(ctx)

    u = torch.from_numpy(wl.u).to(dev)
    heat.heat_set_fields(ctx, cells, u, heat.HEAT_F64, 1, sh)
    j = torch.empty(cells, G, N, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    emis_code = {"f64": heat.HEAT_EMIS_F64, "bf16x3": heat.HEAT_EMIS_BF16X3, "tf32x3": heat.HEAT_EMIS_TF32X3}

    def opts_for(path, timing=0, host_io=0, **kw):
        b, e, _, _ = PATHS[path]
        if path in PRUNE_EPS:
            kw.setdefault("prune_eps", PRUNE_EPS[path])
        return heat.heat_default_opts(build=heat.HEAT_BUILD_F32 if b == "f32" else heat.HEAT_BUILD_F64,
                                      emis=emis_code[e], j_dtype=heat.HEAT_F32, timing=timing, host_io=host_io, **kw)

    def timed_run(path, steps, warmup, sample_clocks=False, **kw):
        for _ in range(warmup):
            heat.heat_solve(ctx, opts_for(path, **kw), None, j, sh)
        heat.heat_sync(ctx)
        heat.heat_get_timing(ctx, reset=True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        for s in range(steps):
            flush.zero_()  # evict L2 between steps (outside the per-step events)
            evs[s][0].record(stream)
            heat.heat_solve(ctx, opts_for(path, timing=1, **kw), None, j, sh)
            evs[s][1].record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - w0
        clocks = sampler.stop() if sampler else None
        heat.heat_sync(ctx)
        step_ms = [a.elapsed_time(b) for a, b in evs]
        kt = heat.heat_get_timing(ctx, reset=True)
        return float(np.mean(step_ms)), step_ms, kt, clocks, wall

    ms, step_ms, kt, clocks, wall = timed_run(args.path, args.steps, args.warmup, sample_clocks=True)
    total_ms = float(np.sum(step_ms))
    if ws > 1:
        from paper_1311_4627_gb300 import shard

        total_ms = shard.max_over_ranks(total_ms)
    value = ws * cells * G * args.steps / (total_ms / 1e3)
    # kernel launches: one per timed region (the per-grain tensor-core emissivity's operand is
    # packed by the recursion's epilogue, so its region holds the GEMM alone)
    gpu_launches = int(sum(n for _, (_, n) in kt.items()))

    # roofline of every kernel class, the dominant one as "roofline"; the FP64-bound ones also
    # against the FP64 FMA rate measured on this device now (the peaks file has none)
    nbt = wl.total_bins
    peaks, peaks_src = measured_peaks()
    fp64_measured = heat.heat_measure_fma_peak(dev.index, True)
    fp32_measured = heat.heat_measure_fma_peak(dev.index, False)
    rooflines = {}
    for name, (tot_ms, n_launch) in kt.items():
        if n_launch == 0:
            continue
        per_step = n_launch / args.steps
        launch_ms = tot_ms / n_launch
        if name == "recur":
            work = 2.0 * cells * (band + nbt)
            r = {"bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                 "peak_source": "nominal dense FP64 1.25 TFLOP/s (profiling recipe table)",
                 "algorithmic_work": f"2 x cells x (band elements + rows) = {work:.3e} FP64 flop per step"}
        elif name == "emis" and PATHS[args.path][1] == "f64":
            work = 2.0 * cells * nbt * N
            r = {"bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                 "peak_source": "nominal dense FP64 1.25 TFLOP/s (profiling recipe table)",
                 "algorithmic_work": f"2 x cells x total bins x wavelengths = {work:.3e} FP64 flop per step"}
        elif name == "emis":
            work = 2.0 * cells * nbt * N
            tf32 = PATHS[args.path][1].startswith("tf32")
            pk = peaks["bf16_tflops"] / (2.0 if tf32 else 1.0)
            r = {"bound": "tensor", "unit": "TFLOP/s", "peak": pk,
                 "peak_source": ("measured bf16 burst" + (" x 1/2 (nominal tf32:bf16 ratio)" if tf32 else "")
                                 + f" ({peaks_src})"),
                 "algorithmic_work": f"2 x cells x total bins x wavelengths = {work:.3e} flop per step "
                                     f"(the split executes 3x this on the tensor pipe, plus operand packing)"}
        else:
            continue
        ach = work / per_step / (launch_ms / 1e3) / 1e12
        r.update({"kernel": name, "achieved": ach, "frac": ach / r["peak"], "traffic": None})
        if r["bound"] == "alu" and fp64_measured:
            r.update({"measured_peak": fp64_measured, "frac_of_measured": ach / fp64_measured,
                      "measured_peak_source": "heat_measure_fma_peak: independent DFMA chains on every SM, this run"})
        rooflines[name] = r
    dom = max(rooflines, key=lambda k: kt[k][0])
    roofline = dict(rooflines[dom])
    roofline["traffic"] = recorded_traffic(dom, cells, kt[dom][1] / args.steps)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": PATHS[args.path][3], "data": "synthetic",
            "config": dict(workload_config(wl, PATHS[args.path][2]),
                           l2="flushed between steps (256 MiB write outside the per-step events)",
                           band_elements_per_cell=band, grain_setup_s=round(setup_s, 3)),
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kt.items()},
            "roofline": roofline, "kernel_rooflines": rooflines, "clocks": clocks, "gpu_launches": gpu_launches,
            "wall_s_timed_region": wall,
            "measured_fma_peaks_tflops": {"fp64": fp64_measured, "fp32": fp32_measured,
                                          "how": "heat_measure_fma_peak (8 independent FMA chains per thread, "
                                                 "full occupancy, fastest of 4 timed launches)"}}

    # the same solve captured once into a CUDA graph and replayed (heat_graph_*), L2 flushed
    # between replays as above
    if ws == 1:
        gs = torch.cuda.Stream(dev)  # stream capture needs a stream other than the legacy default
        torch.cuda.synchronize(dev)
        g = heat.Graph(ctx, opts_for(args.path), None, j, gs.cuda_stream)
        for _ in range(2):
            g.launch(gs.cuda_stream)
        torch.cuda.synchronize(dev)
        gms = []
        for _ in range(args.steps):
            with torch.cuda.stream(gs):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(gs)
            g.launch(gs.cuda_stream)
            e1.record(gs)
            torch.cuda.synchronize(dev)
            gms.append(e0.elapsed_time(e1))
        heat.heat_sync(ctx)
        line["graph"] = {"ms_per_step": float(np.mean(gms)), "spectra_per_s": cells * G / (np.mean(gms) / 1e3),
                         "kernel_nodes": g.kernel_nodes(),
                         "note": "the headline solve replayed from one captured CUDA graph"}
        g.close()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    if not args.no_e2e:
        u_host = torch.from_numpy(wl.u).pin_memory()
        j_host = [torch.empty(cells, G, N, dtype=torch.float32).pin_memory() for _ in range(2)]

        def e2e_run(host_io):
            # every step copies its fields in and its spectra out; with host_io = 2 the calls
            # return once queued and a step's copies out overlap the next step's kernels
            oe = opts_for(args.path, host_io=host_io)
            for k in range(2):
                heat.heat_set_fields(ctx, cells, u_host, heat.HEAT_F64, 0, sh)
                heat.heat_solve(ctx, oe, None, j_host[k % 2], sh)
            heat.heat_sync(ctx)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for k in range(args.steps):
                heat.heat_set_fields(ctx, cells, u_host, heat.HEAT_F64, 0, sh)
                heat.heat_solve(ctx, oe, None, j_host[k % 2], sh)
            torch.cuda.synchronize(dev)
            dt = (time.perf_counter() - t0) / args.steps
            heat.heat_sync(ctx)
            return ws * cells * G / dt

        v_async = e2e_run(2)
        v_sync = e2e_run(1)
        # the copies alone, as plain pinned-memory copies on a side stream (3 of each, CUDA events):
        # with the two directions on their own copy engines, the slower one bounds a step from below
        j_dev = torch.empty(cells, G, N, dtype=torch.float32, device=dev)
        u_dev2 = torch.empty_like(u)
        cs = torch.cuda.Stream(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(cs):
            j_host[0].copy_(j_dev, non_blocking=True)
            u_dev2.copy_(u_host, non_blocking=True)
            ev[0].record(cs)
            for _ in range(3):
                j_host[0].copy_(j_dev, non_blocking=True)
            ev[1].record(cs)
            for _ in range(3):
                u_dev2.copy_(u_host, non_blocking=True)
            ev[2].record(cs)
        cs.synchronize()
        d2h_b, h2d_b = j_host[0].numel() * 4, u_host.numel() * 8
        d2h_gbs = 3 * d2h_b / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e9
        h2d_gbs = 3 * h2d_b / (ev[1].elapsed_time(ev[2]) * 1e-3) / 1e9
        floor_ms = max(d2h_b / d2h_gbs, h2d_b / h2d_gbs) / 1e6
        del j_dev, u_dev2
        line["e2e"] = {"value": v_async, "unit": UNIT, "h2d_bytes_per_step": int(h2d_b),
                       "d2h_bytes_per_step": int(d2h_b),
                       "mode": "heat_solve with host_io = 2 (pinned host buffers, copies in and out every step, "
                               "queued without waiting; timed to the device's completion)",
                       "synchronous_value": v_sync,
                       "copies_alone": {"d2h_gbs": d2h_gbs, "h2d_gbs": h2d_gbs, "floor_ms_per_step": floor_ms,
                                        "note": "plain pinned-memory copies of one step's j out and u in; the "
                                                "slower direction bounds an overlapped step from below"}}
        heat.heat_set_fields(ctx, cells, u, heat.HEAT_F64, 1, sh)

    # the other exact-method paths, for the plain-vs-mixed comparison
    paths = {args.path: {"spectra_per_s": value, "ms_per_step": ms, "precision": PATHS[args.path][2]}}
    if not args.no_compare:
        for other in PATHS:
            if other == args.path:
                continue
            k2 = max(2, args.steps // 2)
            ms_o, _, kt_o, _, _ = timed_run(other, k2, 1)
            paths[other] = {"spectra_per_s": cells * G / (ms_o / 1e3), "ms_per_step": ms_o,
                            "precision": PATHS[other][2],
                            "kernels_ms_per_step": {k: v[0] / k2 for k, v in kt_o.items()}}
        base = paths["exact"]["spectra_per_s"]
        for v in paths.values():
            v["x_plain_exact"] = v["spectra_per_s"] / base

    # the learned surrogate with exact fallback (trained untimed on other cells)
    sur_j = None
    Cf_oracle = None
    if not args.no_surrogate:
        tw = W.batched(cells=args.sur_cells, seed=2002)
        t0 = time.perf_counter()
        heat.heat_surrogate_init(ctx, 4, W.composition_flags(wl), seed=7)
        ut = torch.from_numpy(tw.u).to(dev)
        heat.heat_set_fields(ctx, tw.n_cells, ut, heat.HEAT_F64, 1, sh)
        jt = torch.empty(tw.n_cells, G, N, dtype=torch.float32, device=dev)
        heat.heat_solve(ctx, opts_for("mixed"), None, jt, sh)
        heat.heat_sync(ctx)
        ns = tw.n_cells * G
        Xt = torch.empty(ns, heat.SURROGATE_INPUTS, dtype=torch.float32, device=dev)
        Yt = torch.empty(ns, N, dtype=torch.float32, device=dev)
        heat.heat_surrogate_samples(ctx, 0, tw.n_cells, jt, Xt, Yt, None, sh)
        del jt
        gen_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        heat.heat_surrogate_fit_norm(ctx, Xt, Yt, ns, sh)
        hist = heat.heat_surrogate_train(ctx, Xt, Yt, ns, 8192, args.sur_epochs, 1e-3, seed=9, stream=sh)
        train_s = time.perf_counter() - t0
        # inference on the ns training samples (2^20 by default: one (field, grain) each)
        lnp_t = torch.zeros(ns, dtype=torch.float32, device=dev)
        lnj_t = torch.empty(ns, N, dtype=torch.float32, device=dev)
        sp_t = torch.empty(ns, dtype=torch.float32, device=dev)
        heat.heat_surrogate_predict(ctx, Xt[:8192], lnp_t[:8192], 8192, lnj_t[:8192], sp_t[:8192], sh)
        e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e_a.record(stream)
        heat.heat_surrogate_predict(ctx, Xt, lnp_t, ns, lnj_t, sp_t, sh)
        e_b.record(stream)
        torch.cuda.synchronize(dev)
        infer_ms = e_a.elapsed_time(e_b)
        del Xt, Yt, ut, lnp_t, lnj_t, sp_t
        heat.heat_set_fields(ctx, cells, u, heat.HEAT_F64, 1, sh)
        fo = opts_for("mixed")
        for _ in range(2):
            heat.heat_solve_surrogate(ctx, fo, args.sur_tol, j, sh)
        heat.heat_sync(ctx)
        ks = max(2, args.steps // 2)
        nfb = 0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(ks):
            nfb = heat.heat_solve_surrogate(ctx, fo, args.sur_tol, j, sh)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_s = ev0.elapsed_time(ev1) / ks
        sur_j = j[: args.oracle_cells].double().cpu().numpy()
        # the network alone: features + ensemble inference over the workload, and its raw
        # accuracy (max relative error over the 1e-6 mask, per spectrum) against the mixed path
        nsm = cells * G
        Xs = torch.empty(nsm, heat.SURROGATE_INPUTS, dtype=torch.float32, device=dev)
        lnp = torch.empty(nsm, dtype=torch.float32, device=dev)
        lnj = torch.empty(nsm, N, dtype=torch.float32, device=dev)
        spr = torch.empty(nsm, dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        heat.heat_surrogate_samples(ctx, 0, cells, None, Xs, None, lnp, sh)
        heat.heat_surrogate_predict(ctx, Xs, lnp, nsm, lnj, spr, sh)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_inf = ev0.elapsed_time(ev1)
        nchk = min(cells, 512)
        jm = torch.empty(nchk, G, N, dtype=torch.float32, device=dev)
        heat.heat_solve(ctx, opts_for("mixed", cell_count=nchk), None, jm, sh)
        heat.heat_sync(ctx)
        ref = jm.reshape(nchk * G, N).double()
        got = torch.exp(lnj[: nchk * G].double())
        pk = ref.max(dim=1, keepdim=True).values
        msk = ref > 1e-6 * pk
        rel = torch.where(msk, (got - ref).abs() / ref.clamp_min(1e-300), torch.zeros_like(ref)).max(dim=1).values
        rel = rel.cpu().numpy()
        spq = spr[: nchk * G].cpu().numpy()
        # calibration: per tolerance, the cells whose every grain's spread is within it (fallback
        # is per cell) and the error of the spectra those cells would take from the network
        cell_sp = spq.reshape(nchk, G).max(axis=1)
        rel_c = rel.reshape(nchk, G)
        calib = {}
        for t in (0.01, 0.03, 0.1, 0.3, 1.0):
            acc = cell_sp <= t
            ea = rel_c[acc].ravel()
            calib[str(t)] = {"accepted_cells": float(np.mean(acc)), "accepted_spectra": float(np.mean(spq <= t)),
                             "err_accepted_median": float(np.median(ea)) if ea.size else None,
                             "err_accepted_max": float(np.max(ea)) if ea.size else None}
        mixed_ms = paths["mixed"]["ms_per_step"] if "mixed" in paths else ms
        raw = {"inference_spectra_per_s": nsm / (ms_inf / 1e3), "inference_ms": ms_inf,
               "max_rel_err_per_spectrum_quantiles": {q: float(np.quantile(rel, float(q))) for q in ("0.1", "0.5", "0.9")},
               "spread_quantiles": {q: float(np.quantile(spq, float(q))) for q in ("0.1", "0.5", "0.9")},
               "accepted_fraction_at_tol": float(np.mean(spq <= args.sur_tol)),
               "calibration_by_tol": calib,
               "break_even_accepted_cells": ms_inf / mixed_ms,
               "break_even_note": "the surrogate path beats the mixed path only if the accepted fraction of cells "
                                  "exceeds network time / mixed time (above 1: never)",
               "sample": f"{nchk} cells x {G} grains vs the mixed path"}
        del Xs, lnp, lnj, spr, jm
        paths["surrogate"] = {"spectra_per_s": cells * G / (ms_s / 1e3), "ms_per_step": ms_s,
                              "precision": "MLP ensemble (4 x 128-512x4-1024, BF16 tensor cores) + mixed-path fallback",
                              "fallback_cells": nfb, "fallback_fraction": nfb / cells, "tol_spread": args.sur_tol,
                              "network_alone": raw,
                              "inference_samples": {"samples": ns, "ms": infer_ms,
                                                    "samples_per_s": ns / (infer_ms / 1e3),
                                                    "flop_per_sample": 4 * 2 * (128 * 512 + 3 * 512 * 512 + 512 * N)},
                              "training": {"samples": ns, "epochs": args.sur_epochs, "data_s": round(gen_s, 2),
                                           "train_s": round(train_s, 2), "loss_first": float(hist[0]),
                                           "loss_last": float(hist[-1])}}
        if "exact" in paths:
            paths["surrogate"]["x_plain_exact"] = paths["surrogate"]["spectra_per_s"] / paths["exact"]["spectra_per_s"]

    # oracle on the host cores (rank 0, N = 1), its outputs double as the error reference
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, P_ref, j_ref, Cf = oracle_sample(wl, args.oracle_cells)
        Cf_oracle = Cf
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "one_core")}
        nsub = args.oracle_cells
        for path in [q for q in paths if q in PATHS]:
            P_sub = torch.empty(nsub, nbt, dtype=torch.float64, device=dev)
            j_sub = torch.empty(nsub, G, N, dtype=torch.float64, device=dev)
            o_sub = opts_for(path, cell_count=nsub)
            o_sub.j_dtype = heat.HEAT_F64
            heat.heat_solve(ctx, o_sub, P_sub, j_sub, sh)
            heat.heat_sync(ctx)
            Pg, jg = P_sub.cpu().numpy(), j_sub.cpu().numpy()
            m = np.abs(P_ref) > 1e-280
            rel_P = float(np.max(np.abs(Pg[m] - P_ref[m]) / np.abs(P_ref[m])))
            # P where it is within 1e-6 of its spectrum's peak (the pruned path zeroes the tail)
            pk = np.concatenate([np.repeat(P_ref[:, wl.grain_slice(g)].max(axis=1, keepdims=True), wl.bins(g), axis=1)
                                 for g in range(G)], axis=1)
            mb = P_ref > 1e-6 * pk
            rel_P_big = float(np.max(np.abs(Pg[mb] - P_ref[mb]) / P_ref[mb]))
            peak = j_ref.max(axis=-1, keepdims=True)
            mj = j_ref > 1e-6 * peak
            rel_j = float(np.max(np.abs(jg[mj] - j_ref[mj]) / j_ref[mj]))
            mj_all = np.abs(j_ref) > 1e-280
            rel_j_all = float(np.max(np.abs(jg[mj_all] - j_ref[mj_all]) / np.abs(j_ref[mj_all])))
            paths[path]["max_rel_err"] = {"P": rel_P, "P_above_1e-6_peak": rel_P_big,
                                          "j_masked_1e-6_peak": rel_j, "j_all_above_1e-280": rel_j_all,
                                          "sample": f"{nsub} cells x {G} grains vs the FP64 oracle"}
        if sur_j is not None:
            peak = j_ref.max(axis=-1, keepdims=True)
            mj = j_ref > 1e-6 * peak
            paths["surrogate"]["max_rel_err"] = {
                "j_masked_1e-6_peak": float(np.max(np.abs(sur_j[mj] - j_ref[mj]) / j_ref[mj])),
                "sample": f"{nsub} cells x {G} grains vs the FP64 oracle"}
    line["paths"] = paths
    if rank == 0 and ws == 1 and not args.no_point:
        line["point_rule"] = point_rule_section(args, wl, ctx, heat, timed_run, opts_for, dev, sh, Cf_oracle)
    if rank == 0 and ws == 1 and not args.no_single_cell:
        line["single_cell"] = single_cell_section(dev, stream)
    if rank == 0 and ws == 1 and not args.no_discrete:
        line["thermal_discrete"] = thermal_discrete_section(dev)
    if rank == 0 and ws == 1 and not args.no_rt_volume:
        line["rt_volume"] = rt_volume_section(dev)
    if rank == 0 and ws == 1 and not args.no_emis_heavy:
        del j
        torch.cuda.empty_cache()
        line["emissivity_heavy"] = emissivity_heavy_section(args, dev, stream, peaks, peaks_src)
    if rank == 0:
        print(json.dumps(line))
    heat.heat_destroy(ctx)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
