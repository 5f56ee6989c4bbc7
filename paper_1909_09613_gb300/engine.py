"""Host-side orchestration of many runs: autotuning, batching and serving.

Everything here is scheduling and bookkeeping on the host; every step of every run executes in
libpic's kernels (pic_step for a run on its own, pic_batch_step for a batch).

* `Autotuner` picks the particle-tile extent and the sort interval of a run by timing short
  probe runs of the same spline order and particle density and keeping the fastest full step
  (sort cost included).
* `make_run` builds a run from a request and loads its seeded particles on the device.
* `Server` is a continuous-batching request loop: requests (NCI-scan runs: grid, c dt, drift
  gamma, particles per cell) arrive over time, are admitted when the device-memory budget has
  room, stay resident until their last step, and are advanced in chunks of steps -- every 2D
  run of the FP32 form in one batch (one persistent particle kernel per step), every 3D run on
  its own stream, all concurrently.  When runs finish or arrive, the batch is rebuilt at the
  next chunk boundary.  It reports the latency (completion - arrival) of every request.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import paper_1909_09613_gb300 as pic


@dataclass
class Request:
    rid: int
    grid: Tuple[int, int, int]
    dt: float
    l: int
    gamma: float
    u_th: float
    ppc: int
    steps: int
    arrival: float = 0.0          # seconds after the serving clock starts
    scheme: int = pic.PIC_SCHEME_WT
    seed: int = 0

    @property
    def dim(self):
        return 3 if self.grid[2] > 1 else 2

    @property
    def particles(self):
        return self.grid[0] * self.grid[1] * self.grid[2] * self.ppc


def _default_interval(dt: float, dim: int) -> int:
    return int(math.floor(2.0 / dt)) + 1 if dim == 2 else 8


class Autotuner:
    """Chooses (tile, sort interval) per (spline order, particles per cell) by timing probe runs.

    The probe is a 512x256 run (2D, FP32 form) of the same order and density at c dt = 0.4,
    large enough that launch latency does not decide; candidates are the tile extents below
    crossed with the default sort interval and half of it (a smaller shared-memory halo, more
    frequent sorts).  The measured quantity is the time of whole steps (particle kernel, Yee
    and the amortised sort) over two sort intervals, per particle."""

    TILES = ((16, 8), (32, 8), (32, 16), (64, 8), (64, 16), (32, 32))

    def __init__(self, probe_grid=(512, 256), probe_dt=0.4):
        self.probe_grid = probe_grid
        self.probe_dt = probe_dt
        self.cache: Dict[Tuple[int, int], Tuple[Tuple[int, int], float]] = {}
        self.log: List[dict] = []

    def choose(self, l: int, ppc: int, dt: float) -> Tuple[Tuple[int, int, int], int]:
        key = (int(l), int(ppc))
        if key not in self.cache:
            self.cache[key] = self._tune(*key)
        tile, frac = self.cache[key]
        si = max(1, int(round(_default_interval(dt, 2) * frac)))
        return (tile[0], tile[1], 1), si

    def _tune(self, l: int, ppc: int):
        import torch
        import workloads
        best = None
        wl = workloads.pair_plasma(self.probe_grid, (1.0, 1.0), self.probe_dt, l, 1, 20.0, 0.01,
                                   ppc, device="cuda", seed=12345)
        caps = [int(s.x.shape[1]) for s in wl.species]
        base_si = _default_interval(self.probe_dt, 2)
        for tile in self.TILES:
            for frac in (1.0, 0.5):
                si = max(1, int(round(base_si * frac)))
                try:
                    run = pic.Run(wl.grid, wl.dx, wl.dt, l, 1, precision=pic.PIC_FP32_MIXED,
                                  capacity=caps, tile=(tile[0], tile[1], 1), sort_interval=si)
                except pic.PicError:
                    continue
                for i, s in enumerate(wl.species):
                    run.load(i, s.q, s.m, s.w, s.x, s.u)
                run.step(2)
                torch.cuda.synchronize()
                n = 2 * si
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(run.stream)
                run.step(n)
                e1.record(run.stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / n / sum(caps)
                self.log.append({"l": l, "ppc": ppc, "tile": tile, "sort_interval": si,
                                 "ns_per_particle_step": t * 1e6})
                if best is None or t < best[0]:
                    best = (t, tile, frac)
                run.close()
        return best[1], best[2]


def make_run(req: Request, precision=pic.PIC_FP32_MIXED, tuner: Optional[Autotuner] = None,
             stream=None, device="cuda"):
    """Create, bind and load one run for a request (seeded drifting pair plasma)."""
    import workloads
    dx = (1.0, 1.0, 1.0)
    wl = workloads.pair_plasma(req.grid if req.dim == 3 else req.grid[:2], dx[:req.dim], req.dt,
                               req.l, req.scheme, req.gamma, req.u_th, req.ppc, seed=req.seed,
                               run=req.rid, device=device)
    tile, si = (None, 0)
    if tuner is not None and req.dim == 2 and precision == pic.PIC_FP32_MIXED:
        tile, si = tuner.choose(req.l, req.ppc, req.dt)
        tile = (min(tile[0], req.grid[0]), min(tile[1], req.grid[1]), 1)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=precision, capacity=caps,
                  tile=tile, sort_interval=si, stream=stream)
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, s.u)
    del wl
    return run


def footprint_estimate(req: Request, precision=pic.PIC_FP32_MIXED) -> int:
    """Device bytes a request will hold (libpic's own footprint query, without device work)."""
    dim = req.dim
    grid = req.grid
    n = grid[0] * grid[1] * grid[2] * req.ppc // 2
    opt = pic.pic_options()
    opt.precision = precision
    opt.n_species = 2
    opt.capacity[0] = n
    opt.capacity[1] = n
    ctx = pic.pic_create(grid, (1.0, 1.0, 1.0), req.dt, req.l, req.scheme, opt)
    try:
        b = pic.pic_footprint(ctx)
    finally:
        pic.pic_destroy(ctx)
    # the seeded FP64 input arrays are created on the device while loading
    return b + n * 2 * (dim + 3) * 8


@dataclass
class Served:
    rid: int
    arrival: float
    admitted: float
    done: float
    steps: int
    particles: int
    dim: int
    diag: dict = field(default_factory=dict)

    @property
    def latency(self):
        return self.done - self.arrival


class Server:
    """Continuous-batching request loop (see module docstring)."""

    def __init__(self, budget_bytes: float = 150e9, chunk: int = 10,
                 tuner: Optional[Autotuner] = None, keep_runs: bool = False):
        self.budget = float(budget_bytes)
        self.chunk = int(chunk)
        self.tuner = tuner
        self.keep_runs = keep_runs
        self.results: List[Served] = []
        self.finished_runs = {}
        self.peak_bytes = 0
        self.max_active = 0
        self.chunks = 0

    def serve(self, requests: List[Request]) -> List[Served]:
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        active = {}      # rid -> dict(run, req, done_steps, admitted, bytes, stream)
        used = 0
        batch = None
        batch_ids: Tuple[int, ...] = ()
        t0 = time.perf_counter()
        s3d = [torch.cuda.Stream() for _ in range(4)]
        while pending or active:
            now = time.perf_counter() - t0
            # admit arrived requests while the budget has room (arrival order)
            while pending and pending[0].arrival <= now:
                req = pending[0]
                need = footprint_estimate(req)
                if used + need > self.budget and active:
                    break
                pending.pop(0)
                stream = s3d[req.rid % len(s3d)] if req.dim == 3 else None
                run = make_run(req, tuner=self.tuner, stream=stream)
                active[req.rid] = {"run": run, "req": req, "done": 0, "bytes": need,
                                   "admitted": time.perf_counter() - t0}
                used += need
                self.peak_bytes = max(self.peak_bytes, used)
            if not active:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            # the 2D runs form the batch; rebuild it when the set changed
            ids2d = tuple(sorted(r for r, a in active.items() if a["req"].dim == 2))
            if ids2d != batch_ids:
                if batch is not None:
                    batch.sync()
                    batch.close()
                batch = pic.Batch([active[r]["run"] for r in ids2d]) if ids2d else None
                batch_ids = ids2d
            self.max_active = max(self.max_active, len(active))
            self.chunks += 1
            # one chunk: as many steps as the nearest-finishing active run still needs
            k = min(self.chunk, min(a["req"].steps - a["done"] for a in active.values()))
            if batch is not None:
                batch.step(k)
            for rid, a in active.items():
                if a["req"].dim == 3:
                    a["run"].step(k)
            torch.cuda.synchronize()
            for a in active.values():
                a["done"] += k
            finished = [r for r, a in active.items() if a["done"] >= a["req"].steps]
            if finished:
                if batch is not None:
                    batch.sync()
                    if any(r in batch_ids for r in finished):
                        batch.close()
                        batch = None
                        batch_ids = ()
                for rid in finished:
                    a = active.pop(rid)
                    d = a["run"].diag()
                    done_t = time.perf_counter() - t0
                    self.results.append(Served(rid, a["req"].arrival, a["admitted"], done_t,
                                               a["req"].steps, a["req"].particles, a["req"].dim, d))
                    used -= a["bytes"]
                    if self.keep_runs:
                        self.finished_runs[rid] = a["run"]
                    else:
                        a["run"].close()
        if batch is not None:
            batch.close()
        return self.results


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return v[lo] + (v[hi] - v[lo]) * (k - lo)
