"""Radiative-transfer volume run: every cell of a volume solved chunk by chunk through the
C ABI (mixed path, size-integrated emissivity J_c = sum_g w_g j_{c,g}, Eq. convolution),
an energy check per chunk, and a checkpoint manifest so that an interrupted run resumes
where it stopped.

The manifest (``manifest.json`` in the output directory) records the run's configuration
and, per finished chunk, its output file, the file's SHA-256, the cell range and the
energy check.  A resumed run must have the same configuration; a chunk whose file is
missing or whose checksum does not match is computed again.  The manifest is replaced
atomically (written to a temporary file, then renamed).

    python -m paper_1311_4627_gb300.volume --out DIR [--shape 128 128 64] [--chunk 65536]

Several GPUs (one process each, launched by torchrun): the ranks take chunks from a shared
queue (shard.ChunkQueue) as they become free, so a faster device solves more of them (the
paper's host + coprocessor scheduling, Appendix B), each rank records its chunks in its own
manifest shard, and rank 0 merges the shards into the manifest at the end.

    torchrun --nproc-per-node N -m paper_1311_4627_gb300.volume --out DIR ...
"""
from __future__ import annotations

import argparse
import hashlib
import io
import json
import os
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

MANIFEST = "manifest.json"


def sha256_file(path: str) -> str:
    h = hashlib.sha256()
    with open(path, "rb") as f:
        for block in iter(lambda: f.read(1 << 22), b""):
            h.update(block)
    return h.hexdigest()


def energy_summary(ledger: np.ndarray, weights: np.ndarray) -> dict:
    """Energy check of one chunk from the solve's ledger [cells][grains][2] (absorbed power on
    the grid, emitted power of the discrete model, erg/s per grain): the spread of the
    per-spectrum ratio emitted / absorbed and the size-weighted totals."""
    absorbed, emitted = ledger[..., 0], ledger[..., 1]
    ok = absorbed > 0
    r = emitted[ok] / absorbed[ok]
    tot_a = float(np.sum(absorbed * weights[None, :]))
    tot_e = float(np.sum(emitted * weights[None, :]))
    return {"spectra": int(ok.sum()), "ratio_min": float(r.min()) if r.size else None,
            "ratio_median": float(np.median(r)) if r.size else None, "ratio_max": float(r.max()) if r.size else None,
            "weighted_absorbed": tot_a, "weighted_emitted": tot_e,
            "weighted_ratio": tot_e / tot_a if tot_a > 0 else None}


def _write_json_atomic(out_dir: str, path: str, obj: dict) -> None:
    fd, tmp = tempfile.mkstemp(dir=out_dir, prefix=".manifest.", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(obj, f, indent=1, sort_keys=True)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def _shard_files(out_dir: str) -> list[str]:
    return sorted(os.path.join(out_dir, f) for f in os.listdir(out_dir)
                  if f.startswith("manifest.") and f.endswith(".json") and f != MANIFEST)


class ChunkManifest:
    """Checkpoint state of a chunked run (host logic only).  With `shard` (a rank's name in a
    run of several processes) the records this process makes go to manifest.<shard>.json, so
    that no two processes write one file; load() sees the manifest and every shard, and
    merge() folds the shards into the manifest."""

    def __init__(self, out_dir: str, config: dict, shard: str | None = None):
        self.out_dir = out_dir
        self.config = config
        self.path = os.path.join(out_dir, MANIFEST if shard is None else f"manifest.{shard}.json")
        self.shard = shard
        self.chunks: dict[str, dict] = {}  # every record seen (manifest and shards)
        self.own: dict[str, dict] = {}     # records written by this process's file

    def _read(self, path: str) -> dict:
        with open(path) as f:
            m = json.load(f)
        if m.get("config") != self.config:
            raise ValueError(f"{path}: written by a run with another configuration")
        return m.get("chunks", {})

    def load(self, resume: bool) -> None:
        os.makedirs(self.out_dir, exist_ok=True)
        main = os.path.join(self.out_dir, MANIFEST)
        if self.shard is None and (not resume or not os.path.exists(main)):
            for p in _shard_files(self.out_dir):  # shards of an earlier run do not count
                os.remove(p)
            self.chunks, self.own = {}, {}
            self.save()
            return
        self.chunks = {}
        for p in ([main] if os.path.exists(main) else []) + _shard_files(self.out_dir):
            self.chunks.update(self._read(p))
        self.own = dict(self._read(self.path)) if self.shard is not None and os.path.exists(self.path) else \
            (dict(self.chunks) if self.shard is None else {})

    def save(self) -> None:
        _write_json_atomic(self.out_dir, self.path, {"version": 1, "config": self.config, "chunks": self.own})

    def merge(self) -> None:
        """Fold every shard into the manifest (one process, after all shards are written)."""
        main = os.path.join(self.out_dir, MANIFEST)
        chunks = self._read(main) if os.path.exists(main) else {}
        shards = _shard_files(self.out_dir)
        for p in shards:
            chunks.update(self._read(p))
        _write_json_atomic(self.out_dir, main, {"version": 1, "config": self.config, "chunks": chunks})
        for p in shards:
            os.remove(p)
        self.chunks = dict(chunks)

    def done(self, k: int) -> bool:
        """Chunk k finished and its file intact."""
        e = self.chunks.get(str(k))
        if not e:
            return False
        p = os.path.join(self.out_dir, e["file"])
        return os.path.exists(p) and sha256_file(p) == e["sha256"]

    def record(self, k: int, fname: str, info: dict, sha256: str | None = None) -> None:
        p = os.path.join(self.out_dir, fname)
        e = dict(info, file=fname, sha256=sha256 if sha256 is not None else sha256_file(p))
        self.chunks[str(k)] = e
        self.own[str(k)] = e
        self.save()


def write_chunk(out_dir: str, fname: str, J: np.ndarray) -> str:
    """Write J as .npy under its final name atomically (temporary file, then rename) and
    return the file's SHA-256, hashed from the bytes written rather than read back (the
    array is written from its own memory, without an intermediate copy)."""
    J = np.ascontiguousarray(J, dtype=np.float32)
    head = io.BytesIO()
    np.lib.format.write_array_header_1_0(head, np.lib.format.header_data_from_array_1_0(J))
    header = head.getvalue()
    body = memoryview(J).cast("B")
    h = hashlib.sha256(header)
    h.update(body)
    fd, tmp = tempfile.mkstemp(dir=out_dir, prefix=".chunk.", suffix=".tmp")
    with os.fdopen(fd, "wb") as f:
        f.write(header)
        f.write(body)
    os.replace(tmp, os.path.join(out_dir, fname))
    return h.hexdigest()


def run_chunks(manifest: ChunkManifest, n_cells: int, chunk: int, solve_chunk, resume: bool = True,
               stop_after: int | None = None, prepare=None, log=None, claim=None) -> dict:
    """Drive the chunks of [0, n_cells): skip the finished ones, solve the others with
    solve_chunk(k, begin, end, prepared) -> (J float32 [cells][n_lambda], info dict), write
    J_k.npy and record it.  prepare(begin, end), if given, runs one chunk ahead in a host
    thread (e.g. making the next chunk's fields while the GPU works); the file of a solved
    chunk is written and hashed in another host thread while the next chunk is solved, and
    recorded in the manifest once it is complete.  stop_after: return after that many
    chunks were solved in this call (an interrupted run).  claim: an iterable of chunk
    indices handed to this process (a shard.ChunkQueue shared by several), taken one chunk
    ahead of the solve; without it every chunk is this process's."""
    manifest.load(resume)
    n_all = (n_cells + chunk - 1) // chunk
    if claim is None:
        todo = iter([k for k in range(n_all) if not manifest.done(k)])
    else:  # claimed chunks that an earlier run finished are skipped
        todo = (k for k in claim if not manifest.done(k))
    todo = _lookahead(todo)
    solved = 0
    pending = None  # (k, fname, info, future) of the chunk being written

    def finish(p):
        k, fname, info, fut = p
        manifest.record(k, fname, info, sha256=fut.result())
        if log:
            log(f"chunk {k}: cells {info['cells']} {json.dumps(info)}")

    with ThreadPoolExecutor(1) as pool, ThreadPoolExecutor(1) as writer:
        nxt = None
        first = todo.peek()
        if prepare and first is not None:
            b = first * chunk
            nxt = pool.submit(prepare, b, min(n_cells, b + chunk))
        while stop_after is None or solved < stop_after:  # no chunk is claimed past the stop
            k = next(todo, None)
            if k is None:
                break
            b, e = k * chunk, min(n_cells, (k + 1) * chunk)
            prepared = nxt.result() if nxt is not None else None
            nxt = None
            k2 = todo.peek() if (stop_after is None or solved + 1 < stop_after) else None
            if prepare and k2 is not None:
                b2 = k2 * chunk
                nxt = pool.submit(prepare, b2, min(n_cells, b2 + chunk))
            J, info = solve_chunk(k, b, e, prepared)
            if pending is not None:  # at most one chunk waits for the disk
                finish(pending)
            fname = f"J_{k:05d}.npy"
            pending = (k, fname, dict(info, cells=[b, e]), writer.submit(write_chunk, manifest.out_dir, fname, J))
            solved += 1
        if pending is not None:
            finish(pending)
    return {"chunks": n_all, "solved_now": solved, "complete": all(manifest.done(k) for k in range(n_all))}


class _lookahead:
    """An iterator with peek(): the next item, taken from the source one step early (so a
    claimed chunk's fields can be prepared while the previous chunk is solved)."""

    _END = object()

    def __init__(self, it):
        self.it = iter(it)
        self.buf = self._END
        self.buffered = False

    def peek(self):
        if not self.buffered:
            self.buf = next(self.it, self._END)
            self.buffered = True
        return None if self.buf is self._END else self.buf

    def __iter__(self):
        return self

    def __next__(self):
        v = self.peek()
        self.buffered = False
        if v is None:
            raise StopIteration
        return v


def run_distributed(out_dir: str, config: dict, n_cells: int, chunk: int, solve_chunk, resume: bool = True,
                    stop_after: int | None = None, prepare=None, log=None) -> dict:
    """run_chunks on every rank of an initialised torch.distributed process group (any
    backend: only barriers and one broadcast of a path pass through it), the chunks handed out
    by a ChunkQueue on a FileStore in the output directory.  Each rank records its chunks in
    its manifest shard; rank 0 resets or checks the manifest first and merges the shards at
    the end.  Returns this rank's run_chunks result plus the chunks it solved and, on rank 0,
    whether the merged run is complete."""
    import shutil

    import torch.distributed as dist

    from .shard import ChunkQueue

    rank, world = dist.get_rank(), dist.get_world_size()
    n_all = (n_cells + chunk - 1) // chunk
    qdir = [None]
    if rank == 0:
        ChunkManifest(out_dir, config).load(resume)  # start a run or check the one resumed
        qdir = [tempfile.mkdtemp(dir=out_dir, prefix=".queue.")]
    dist.broadcast_object_list(qdir, src=0)
    store = dist.FileStore(os.path.join(qdir[0], "store"), world)
    dist.barrier()
    man = ChunkManifest(out_dir, config, shard=f"r{rank}")
    mine = []

    def claim():
        for k in ChunkQueue(store, n_all, name="volume"):
            mine.append(k)
            yield k

    claims = claim()
    res = run_chunks(man, n_cells, chunk, solve_chunk, resume=True, stop_after=stop_after, prepare=prepare, log=log,
                     claim=claims)
    dist.barrier()
    if rank == 0:
        m = ChunkManifest(out_dir, config)
        m.merge()
        res["complete"] = all(m.done(k) for k in range(n_all))
    # every rank closes its store (the queue iterator of an interrupted run holds it too)
    # before rank 0 removes the store's directory: a FileStore touches its file when it closes
    claims.close()
    del claims, claim, store
    dist.barrier()
    if rank == 0:
        shutil.rmtree(qdir[0], ignore_errors=True)
    res["claimed"] = mine
    return res


def load_output(manifest_dir: str) -> np.ndarray:
    """The volume's J [cells][n_lambda] assembled from the chunk files."""
    with open(os.path.join(manifest_dir, MANIFEST)) as f:
        m = json.load(f)
    parts = sorted(m["chunks"].values(), key=lambda e: e["cells"][0])
    return np.concatenate([np.load(os.path.join(manifest_dir, e["file"])) for e in parts])


class VolumeSolver:
    """GPU side of a volume run: one ctx with the volume's grains; per chunk the fields are
    made straight into one of two pinned host buffers (the next chunk's while this one is
    solved), copied to the device, solved on the mixed path with size-integrated output and
    the energy ledger, and J is read back into one of two pinned buffers (the other may still
    be being written to disk)."""

    def __init__(self, vol, chunk: int, device: int = 0, emis: str = "bf16x3"):
        import torch

        from . import heat

        self.torch, self.heat, self.vol = torch, heat, vol
        g = vol.grains
        self.dev = torch.device(f"cuda:{device}")
        torch.cuda.set_device(self.dev)
        self.stream = torch.cuda.Stream(self.dev)
        self.ctx = heat.heat_create_grid(device, g.lam)
        heat.heat_set_grains(self.ctx, g.radius, g.cabs, g.bin_off, g.T, g.E, g.size_weight)
        self.emis = {"bf16x3": heat.HEAT_EMIS_BF16X3, "tf32x3": heat.HEAT_EMIS_TF32X3}[emis]
        N, G = g.n_lambda, g.n_grains
        self.u_dev = torch.empty(chunk, N, dtype=torch.float64, device=self.dev)
        self.J_dev = torch.empty(chunk, N, dtype=torch.float32, device=self.dev)
        self.led_dev = torch.empty(chunk, G, 2, dtype=torch.float64, device=self.dev)
        self.u_pin = [torch.empty(chunk, N, dtype=torch.float64).pin_memory() for _ in range(2)]
        self.J_pin = [torch.empty(chunk, N, dtype=torch.float32).pin_memory() for _ in range(2)]
        self.led_pin = torch.empty(chunk, G, 2, dtype=torch.float64).pin_memory()
        self.prep_slot = 0  # pinned field buffer of the next prepare (alternates per call)
        self.solve_slot = 0  # pinned J buffer of the next solve (alternates per call)

    def prepare(self, begin: int, end: int):
        """Make the fields of [begin, end) in the next pinned buffer: (buffer index, array)."""
        s = self.prep_slot
        self.prep_slot ^= 1
        buf = self.u_pin[s][: end - begin].numpy()
        return s, self.vol.fields(begin, end, out=buf)

    def solve_chunk(self, k: int, begin: int, end: int, prepared=None):
        torch, heat = self.torch, self.heat
        n = end - begin
        if prepared is None:
            prepared = self.prepare(begin, end)
        s_in, _ = prepared
        s_out = self.solve_slot
        self.solve_slot ^= 1
        sh = self.stream.cuda_stream
        t0 = time.perf_counter()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(self.stream):
            ev[0].record(self.stream)
            self.u_dev[:n].copy_(self.u_pin[s_in][:n], non_blocking=True)
            heat.heat_set_fields(self.ctx, n, self.u_dev, heat.HEAT_F64, 1, sh)
            o = heat.heat_default_opts(build=heat.HEAT_BUILD_F32, emis=self.emis, j_dtype=heat.HEAT_F32,
                                       size_integrate=1, cell_count=n, ledger_out=self.led_dev)
            heat.heat_solve(self.ctx, o, None, self.J_dev, sh)
            self.J_pin[s_out][:n].copy_(self.J_dev[:n], non_blocking=True)
            self.led_pin[:n].copy_(self.led_dev[:n], non_blocking=True)
            ev[1].record(self.stream)
        self.stream.synchronize()
        heat.heat_sync(self.ctx)
        gpu_ms = ev[0].elapsed_time(ev[1])
        # a view, not a copy: this buffer is filled again two solves later, after the chunk's
        # file has been written (run_chunks keeps at most one chunk waiting for the disk)
        J = self.J_pin[s_out][:n].numpy()
        info = {"gpu_ms": round(gpu_ms, 3), "wall_s": round(time.perf_counter() - t0, 3),
                "spectra": n * self.vol.grains.n_grains,
                "energy": energy_summary(self.led_pin[:n].numpy(), self.vol.grains.size_weight)}
        return J, info

    def close(self):
        self.heat.heat_destroy(self.ctx)


def volume_config(vol, chunk: int, emis: str) -> dict:
    g = vol.grains
    return {"shape": list(vol.shape), "seed": vol.seed, "grains": g.n_grains, "bins": int(g.total_bins),
            "n_lambda": g.n_lambda, "chunk_cells": chunk, "path": f"mixed ({emis}), size-integrated"}


def main(argv=None):
    from . import workloads as W

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--shape", type=int, nargs=3, default=[128, 128, 64])
    ap.add_argument("--chunk", type=int, default=65536)
    ap.add_argument("--radii", type=int, default=40, help="radii per composition")
    ap.add_argument("--bins", type=int, default=512)
    ap.add_argument("--n-lambda", type=int, default=1024)
    ap.add_argument("--emis", default="bf16x3", choices=["bf16x3", "tf32x3"])
    ap.add_argument("--no-resume", action="store_true")
    ap.add_argument("--stop-after", type=int, default=None)
    args = ap.parse_args(argv)
    t0 = time.perf_counter()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    device, rank = 0, 0
    if world > 1:  # one process per GPU (torchrun); the process group only coordinates
        import torch.distributed as dist

        dist.init_process_group("gloo")
        device, rank = int(os.environ.get("LOCAL_RANK", "0")), dist.get_rank()
    vol = W.rt_volume(tuple(args.shape), radii_per_composition=args.radii, nbins=args.bins, n_lambda=args.n_lambda)
    solver = VolumeSolver(vol, args.chunk, device=device, emis=args.emis)
    setup_s = time.perf_counter() - t0
    config = volume_config(vol, args.chunk, args.emis)
    log = (lambda m: print(f"[rank {rank}] {m}")) if world > 1 else print
    if world > 1:
        res = run_distributed(args.out, config, vol.n_cells, args.chunk, solver.solve_chunk, resume=not args.no_resume,
                              stop_after=args.stop_after, prepare=solver.prepare, log=log)
    else:
        res = run_chunks(ChunkManifest(args.out, config), vol.n_cells, args.chunk, solver.solve_chunk,
                         resume=not args.no_resume, stop_after=args.stop_after, prepare=solver.prepare, log=log)
    solver.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
        if rank != 0:
            return
    man = ChunkManifest(args.out, config)
    man.load(resume=True)
    ch = [man.chunks[k] for k in sorted(man.chunks, key=int)]
    gpu_s = sum(c["gpu_ms"] for c in ch) / 1e3
    spectra = sum(c["spectra"] for c in ch)
    ratios = [c["energy"]["weighted_ratio"] for c in ch if c["energy"]["weighted_ratio"] is not None]
    res.update({"cells": vol.n_cells, "spectra": spectra, "gpu_s": round(gpu_s, 3),
                "spectra_per_s_gpu": spectra / gpu_s if gpu_s > 0 else None,
                "wall_s": round(time.perf_counter() - t0, 2), "setup_s": round(setup_s, 2),
                "energy_weighted_ratio_range": [min(ratios), max(ratios)] if ratios else None,
                "config": man.config})
    print(json.dumps(res))


if __name__ == "__main__":
    main()
