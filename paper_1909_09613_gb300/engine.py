"""Host-side orchestration of many runs: autotuning, batching and serving.

Everything here is scheduling and bookkeeping on the host; every step of every run executes in
libpic's kernels (pic_step for a run on its own, pic_batch_step for a batch).

* `Autotuner` picks the particle-tile extent and the sort interval of a run by timing short
  probe runs of the same spline order and particle density and keeping the fastest full step
  (sort cost included).
* `make_run` builds a run from a request and generates its seeded drifting pair plasma in HBM
  with the library's device loader (pic_load_drifting_plasma: App. D's flip and boost of
  Gaussian co-moving momenta); for a batchable run `fit_batch_tile` keeps the tuned tile only
  if its shared-memory stage still lets the batched kernel hold two CTAs per SM (a batch runs
  at the largest stage of its runs).
* `Server` is a continuous-batching request loop: requests (NCI-scan runs: grid, c dt, drift
  gamma, particles per cell) arrive over time, are admitted when the device-memory budget has
  room, stay resident until their last step, and are advanced in chunks of steps -- every 2D
  quadratic or cubic run of the FP32 form in one of two batches, small runs and larger ones
  (one persistent particle kernel per step each), every other run (3D, quartic, plain FP64)
  on a side stream, all concurrently.  When runs finish or arrive, a batch's run set changes
  at its next chunk boundary.  Short requests go first (the other lanes wait at chunk
  boundaries while the batch of small runs holds runs), and runs that each fill the GPU take
  turns in arrival order.  It reports the latency (completion - arrival) of every request and,
  for requests that ask for it, the field-energy history (E/E0 of the Table 1 scan).
* `table1_requests` builds the requests of the paper's Table 1 NCI scan.
"""
from __future__ import annotations

import collections
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
    solver: int = pic.PIC_SOLVER_YEE
    record_every: int = 0         # steps between field-energy samples (0: none)
    rng_run: int = -1             # random stream of the initial plasma (-1: the request id)
    precision: int = pic.PIC_FP32_MIXED
    colocated: bool = False       # positrons start at the electrons' positions (neutral start)

    @property
    def batchable(self):
        """Runs the batched kernel serves (2D FP32 form, quadratic or cubic); others step on
        their own streams."""
        return self.dim == 2 and self.l in (2, 3) and self.precision == pic.PIC_FP32_MIXED

    @property
    def dim(self):
        return 3 if self.grid[2] > 1 else 2

    @property
    def particles(self):
        return self.grid[0] * self.grid[1] * self.grid[2] * self.ppc


def _default_interval(dt: float, dim: int) -> int:
    return int(math.floor(2.0 / dt)) + 1 if dim == 2 else 8


def species_constants(req: Request, s: int):
    """(q, m, w, particles per cell, position species) of species s (0 = e-, 1 = e+) of a
    request's pair plasma.  The weight gives the drifting plasma 16 cells per relativistic skin
    depth (c / omega_p = 16 dx with dx = 1, as in Table 1): omega_p^2 = n q^2 / (gamma m) with
    n = (ppc / 2) w / V_c, so w = omega_p^2 gamma V_c / (ppc / 2)."""
    per = req.ppc // 2
    omega_p = 1.0 / 16.0
    w = omega_p * omega_p * req.gamma / per if per > 0 else 0.0
    return (-1.0 if s == 0 else 1.0, 1.0, w, per, 0 if req.colocated else s)


def load_request(run, req: Request, rng_run: Optional[int] = None):
    """Generate the request's pair plasma in the run's particle stores on the device."""
    rr = req.rid if req.rng_run < 0 else req.rng_run
    if rng_run is not None:
        rr = rng_run
    for s in range(2):
        q, m, w, per, pos = species_constants(req, s)
        run.load_drifting_plasma(s, q, m, w, per, req.gamma, req.u_th, req.seed, rr, pos)


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
        best = None
        probe = Request(rid=0, grid=(self.probe_grid[0], self.probe_grid[1], 1), dt=self.probe_dt,
                        l=l, gamma=20.0, u_th=0.01, ppc=ppc, steps=0, seed=12345)
        n = self.probe_grid[0] * self.probe_grid[1] * (ppc // 2)
        caps = [n, n]
        base_si = _default_interval(self.probe_dt, 2)
        for tile in self.TILES:
            for frac in (1.0, 0.5):
                si = max(1, int(round(base_si * frac)))
                try:
                    run = pic.Run(probe.grid, (1.0, 1.0), probe.dt, l, 1,
                                  precision=pic.PIC_FP32_MIXED, capacity=caps,
                                  tile=(tile[0], tile[1], 1), sort_interval=si)
                except pic.PicError:
                    continue
                load_request(run, probe)
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


# Tiles tried, in order, when the tuned tile of a batchable run would give its batched work
# items more shared memory than two CTAs per SM leave (a batch runs at the largest of its runs)
BATCH_FALLBACK_TILES = ((32, 16), (32, 8), (16, 16), (16, 8))


def fit_batch_tile(req: Request, tile, si):
    """The tuned (tile, sort interval) of a batchable request, or the first of the fallback
    tiles (then with half the sort interval, a narrower drift halo) whose stage keeps two CTAs
    per SM in the batched kernel (pic_smem_info; a host query, no device memory)."""
    def fits(t, k):
        opt = pic.pic_options()
        opt.precision = pic.PIC_FP32_MIXED
        opt.n_species = 2
        n = req.grid[0] * req.grid[1] * req.ppc // 2
        opt.capacity[0] = n
        opt.capacity[1] = n
        opt.tile[0], opt.tile[1], opt.tile[2] = t[0], t[1], 1
        opt.sort_interval = k
        try:
            ctx = pic.pic_create(req.grid, (1.0, 1.0, 1.0), req.dt, req.l, req.scheme, opt)
        except pic.PicError:
            return False
        try:
            _, batched, two = pic.pic_smem_info(ctx)
        finally:
            pic.pic_destroy(ctx)
        return two == 0 or batched <= two
    if fits(tile, si):
        return tile, si
    for k in (si, max(1, si // 2)):
        for t in BATCH_FALLBACK_TILES:
            t = (min(t[0], req.grid[0]), min(t[1], req.grid[1]), 1)
            if fits(t, k):
                return t, k
    return tile, si


def request_tile(req: Request, tuner: Optional[Autotuner] = None, precision=None):
    """(tile, sort interval) a run of this request uses ((None, 0): the library's defaults)."""
    if precision is None:
        precision = req.precision
    if tuner is not None and req.batchable and precision == pic.PIC_FP32_MIXED:
        tile, si = tuner.choose(req.l, req.ppc, req.dt)
        tile = (min(tile[0], req.grid[0]), min(tile[1], req.grid[1]), 1)
        return fit_batch_tile(req, tile, si)
    return None, 0


def make_run(req: Request, precision=None, tuner: Optional[Autotuner] = None,
             stream=None, device="cuda"):
    """Create, bind and load one run for a request: its seeded drifting pair plasma is
    generated on the device (App. D; load_request)."""
    if precision is None:
        precision = req.precision
    tile, si = request_tile(req, tuner, precision)
    n = req.grid[0] * req.grid[1] * req.grid[2] * (req.ppc // 2)
    run = pic.Run(req.grid, (1.0, 1.0, 1.0), req.dt, req.l, req.scheme, precision=precision,
                  capacity=[n, n], tile=tile, sort_interval=si, stream=stream,
                  device=device, solver=req.solver)
    load_request(run, req)
    return run


def footprint_estimate(req: Request, precision=None, tuner: Optional[Autotuner] = None) -> int:
    """Device bytes a request will hold: libpic's own footprint query (no device work) with
    the tile and sort interval the run will use (the sort scratch depends on the tile)."""
    grid = req.grid
    n = grid[0] * grid[1] * grid[2] * req.ppc // 2
    if precision is None:
        precision = req.precision
    tile, si = request_tile(req, tuner, precision)
    opt = pic.pic_options()
    opt.precision = precision
    opt.n_species = 2
    opt.capacity[0] = n
    opt.capacity[1] = n
    opt.solver = req.solver
    if tile is not None:
        opt.tile[0], opt.tile[1], opt.tile[2] = tile
    opt.sort_interval = si
    ctx = pic.pic_create(grid, (1.0, 1.0, 1.0), req.dt, req.l, req.scheme, opt)
    try:
        return pic.pic_footprint(ctx)
    finally:
        pic.pic_destroy(ctx)


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
    # (step, t omega_p, field energy, kinetic energy) every record_every steps, from step 0
    history: list = field(default_factory=list)

    @property
    def latency(self):
        return self.done - self.arrival


class HoldPolicy:
    """Whether the server holds its other lanes for short requests: while short requests run
    (`urgent`), hold, except that a hold longer than `max_hold_s` is released for one round
    (then holding starts over), so that a steady stream of short requests cannot starve the
    others."""

    def __init__(self, max_hold_s: float):
        self.max_hold_s = float(max_hold_s)
        self.since = None
        self.releases = 0

    def hold(self, urgent: bool, now: float) -> bool:
        if not urgent:
            self.since = None
            return False
        if self.since is None:
            self.since = now
        elif now - self.since > self.max_hold_s:
            self.since = now
            self.releases += 1
            return False
        return True


class _BatchLane:
    """One batch of the server: its stream, the pic batch, the runs it holds and the chunk of
    steps it has on the GPU."""

    def __init__(self, stream):
        self.stream = stream
        self.batch = None
        self.bytes = 0
        self.ids: Tuple[int, ...] = ()
        self.inflight = collections.deque()   # (end event, steps, start event) of the chunks on the GPU
        self.captured = False  # the batch's first step (its graph capture) has been issued


class Server:
    """Continuous-batching request loop (see module docstring).

    The batchable runs live in long-lived pic batches whose run sets are replaced with
    pic_batch_set_runs when runs arrive or finish: the batch's launches walk device tables of
    any set that fits its capacities, so its captured CUDA graph is kept (a batch is rebuilt,
    with doubled capacities, only when a set outgrows them).  Two batches, by size: runs of
    fewer than `small_particles` particles share one, larger runs the other, so that a short
    request is not paced by the step of a large run (a batch advances all its runs one step at
    a time, so its step lasts as long as its total work).  Each lane waits for its own streams
    (events), not for the whole device.  The batches' device tables count against the memory
    budget.

    Streams carry priorities, so that short requests are not queued behind the thread blocks of
    a large one: the batch of small runs runs on the highest-priority stream, the batch of the
    larger 2D runs next, other runs of fewer than `large_particles` particles on
    medium-priority side streams, larger runs on low-priority ones.  The GPU's block scheduler
    then starts a waiting block of a higher-priority stream before more blocks of a lower one.

    Priorities order only the start of thread blocks; the particle kernels of a 2D batch need a
    large share of an SM each (256 threads of 128 registers, about 100 KB of shared memory), and
    beside 3D runs and a batch of larger runs, whose blocks fill the SMs, they wait for room
    (measured: the batch of small runs took 0.49 ms per step with 1.07 runs on average, against
    0.1-0.2 ms for one such run alone).  So short requests go first (`preempt`): while the batch
    of small runs holds runs, the other lanes get no new chunks, and their chunks are sized to
    about `chunk_ms` of GPU time, which bounds how long a short request shares the GPU with
    them (a hold longer than `max_hold_s` releases one round of their chunks, so that a steady
    stream of short requests cannot starve them); the persistent particle kernel of the batch of larger runs takes one CTA per SM
    (`large_lane_ctas_per_sm`), leaving the other slot to the batch of small runs.  Side runs of
    `large_particles` and more take turns (`max_large` at a time, in arrival order)."""

    def __init__(self, budget_bytes: float = 150e9, chunk: int = 10,
                 tuner: Optional[Autotuner] = None, keep_runs: bool = False,
                 large_particles: int = 1 << 24, small_particles: int = 1 << 20,
                 depth: int = 2, batch_reserve_bytes: int = 1 << 21,
                 large_lane_ctas_per_sm: int = 1, preempt: bool = True,
                 chunk_ms: float = 4.0, max_large: int = 1, max_hold_s: float = 0.5):
        self.budget = float(budget_bytes)
        self.depth = max(1, int(depth))   # chunks a batch lane keeps queued on its stream
        # budget held for the device tables of a batch lane that has none yet (its first
        # request is admitted before the batch exists); the batch's own bytes replace it
        self.batch_reserve = int(batch_reserve_bytes)
        # the persistent particle kernel of the batch of larger runs holds its SM slots for the
        # whole pass (stream priorities only order the start of CTAs): one CTA per SM leaves
        # the other slot to the batch of small runs
        self.large_lane_ctas_per_sm = int(large_lane_ctas_per_sm)
        # short requests first: while the batch of small runs has runs, the other lanes finish
        # the chunks they have queued but get no new ones, and their chunks are sized to about
        # chunk_ms of GPU time (from their measured step time), so that a short request waits
        # at most about that long for the GPU
        self.preempt = bool(preempt)
        self.chunk_ms = float(chunk_ms)
        # side runs of large_particles and more step max_large at a time, in arrival order: one
        # such run already fills the GPU, so several at once only share it (each finishing as
        # late as the last) where turns let the earlier ones finish first
        self.max_large = max(1, int(max_large))
        self.max_hold_s = float(max_hold_s)
        self.hold_releases = 0   # rounds released by the hold limit in the last serve
        self.large_particles = int(large_particles)
        self.small_particles = int(small_particles)
        self.chunk = int(chunk)
        self.tuner = tuner
        self.keep_runs = keep_runs
        self.results: List[Served] = []
        self.finished_runs = {}
        self.peak_bytes = 0
        self.max_active = 0
        self.chunks = 0
        self.batch_builds = 0
        self.set_changes = 0
        self.lane_runs = [0, 0]   # runs served by the batch of small runs, of larger runs
        self.host_block_s = 0.0   # longest end-of-run read on the loop thread
        # per batch lane: chunks, steps, run-steps and the GPU time of its chunks (events on the
        # lane's stream around each chunk)
        self.lane_stats = [dict(chunks=0, steps=0, run_steps=0, gpu_ms=0.0) for _ in range(2)]

    @staticmethod
    def _capacity(runs, factor=2.0, ctas_per_sm=0):
        """Batch capacities: `factor` times the totals of `runs`, the largest batched stage
        that still lets two CTAs share an SM, and the persistent kernel's CTAs per SM."""
        cap = pic.pic_batch_capacity()
        n = len(runs)
        cap.runs = max(8, int(factor * n))
        cells = tiles = 0
        stage = 0
        for r in runs:
            cells += r.ncell
            tiles += r.ntiles
            _, batched, two = pic.pic_smem_info(r.ctx)
            stage = max(stage, batched, two)
        cap.cells = int(factor * max(cells, 1 << 18))
        # work items: a small set splits its heavier tiles into up to 8 items
        cap.tiles = int(factor * max(8 * tiles, 1 << 12))
        cap.stage_bytes = int(stage)
        cap.ctas_per_sm = int(ctas_per_sm)
        return cap

    def lane_of(self, req: Request) -> int:
        """Batch lane of a batchable request: 0 (small runs) or 1 (larger runs)."""
        return 0 if req.particles < self.small_particles else 1

    def serve(self, requests: List[Request]) -> List[Served]:
        """Serve the requests at their arrival times; returns one Served record per request.

        Lanes advance independently: each batch (its runs, one graph replay per step) and every
        other run on its own side stream.  A lane gets its next chunk of steps as soon as its
        previous chunk's event has completed, so small runs never wait for a large run's
        steps; run sets change, and finished runs are reported, at a lane's chunk boundary."""
        import concurrent.futures as cf
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        # preempting (and time-sized chunks) only matters when short requests are to come
        preempt = self.preempt and any(r.batchable and self.lane_of(r) == 0 for r in requests)
        active = {}      # rid -> dict(run, req, done, admitted, bytes, stream, history, lane)
        # admitted requests whose run is being created and loaded by the loader thread (the
        # library's calls release the interpreter, so the loop keeps the lanes fed meanwhile):
        # rid -> (future, request, bytes, lane)
        loading = {}
        loader = cf.ThreadPoolExecutor(max_workers=1)
        used = 0
        side_inflight = {}      # rid -> (end event, steps, start event) of a side run's chunk
        t0 = time.perf_counter()
        # priorities: lower numbers are served first (torch clamps them to the device's range)
        lanes = [_BatchLane(torch.cuda.Stream(priority=-3)),   # batch of small 2D runs
                 _BatchLane(torch.cuda.Stream(priority=-2))]   # batch of larger 2D runs

        reserved = set()   # lanes whose batch tables are held in the budget by batch_reserve
        hold = HoldPolicy(self.max_hold_s)

        def install(li, ids):
            """Make lane li's batch hold the runs `ids` (a new batch when none fits)."""
            nonlocal used
            lane = lanes[li]
            runs = [active[r]["run"] for r in ids]
            if lane.batch is not None and lane.batch.set_runs(runs):
                self.set_changes += 1
                lane.ids = ids
                return
            if lane.batch is not None:
                lane.batch.set_runs([])   # write every run's state back before the batch goes
                lane.batch.close()
                used -= lane.bytes
                lane.batch, lane.bytes = None, 0
            if runs:
                lane.batch = pic.Batch(runs, capacity=self._capacity(
                    runs, ctas_per_sm=self.large_lane_ctas_per_sm if li == 1 else 0))
                lane.captured = False
                lane.bytes = int(lane.batch.mem.numel())
                used += lane.bytes
                if li in reserved:
                    reserved.discard(li)
                    used -= self.batch_reserve
                self.peak_bytes = max(self.peak_bytes, used)
                self.batch_builds += 1
            lane.ids = ids

        def chunk_steps(ids, ahead=0, ms_per_step=0.0):
            """Steps of the next chunk of runs `ids`, `ahead` steps past their completed ones
            (at most about chunk_ms of GPU time when preempting and the step time is known)."""
            k = self.chunk
            if preempt and ms_per_step > 0.0:
                k = max(1, min(k, int(self.chunk_ms / ms_per_step)))
            k = min(k, min(active[r]["req"].steps - active[r]["done"] - ahead for r in ids))
            for r in ids:  # stop at the next field-energy sample
                ev = active[r]["req"].record_every
                if ev > 0:
                    k = min(k, ev - (active[r]["done"] + ahead) % ev)
            return k

        def stops(ids, ahead):
            """A run of `ids` samples its field energy or ends `ahead` steps past its completed
            steps (the host must act there before more steps are queued)."""
            for r in ids:
                a = active[r]
                n = a["done"] + ahead
                ev = a["req"].record_every
                if n >= a["req"].steps or (ev > 0 and n % ev == 0):
                    return True
            return False

        def finish(rid):
            nonlocal used
            a = active.pop(rid)
            tb = time.perf_counter()
            d = a["run"].diag()
            self.host_block_s = max(self.host_block_s, time.perf_counter() - tb)
            done_t = time.perf_counter() - t0
            self.results.append(Served(rid, a["req"].arrival, a["admitted"], done_t,
                                       a["req"].steps, a["req"].particles, a["req"].dim, d,
                                       a["history"]))
            used -= a["bytes"]
            if self.keep_runs:
                self.finished_runs[rid] = a["run"]
            else:
                a["run"].close()

        def recorded(a):
            ev = a["req"].record_every
            return ev > 0 and a["done"] % ev == 0

        while pending or active or loading:
            progressed = False
            now = time.perf_counter() - t0
            # admit arrived requests while the budget has room (arrival order)
            while pending and pending[0].arrival <= now:
                req = pending[0]
                need = footprint_estimate(req, tuner=self.tuner)
                lane = self.lane_of(req) if req.batchable else -1
                extra = (self.batch_reserve if lane >= 0 and lanes[lane].batch is None
                         and lane not in reserved else 0)
                if used + need + extra > self.budget and (active or loading):
                    break
                pending.pop(0)
                if extra:
                    reserved.add(lane)
                    used += extra
                if lane >= 0:
                    stream = lanes[lane].stream
                    self.lane_runs[lane] += 1
                else:
                    # a side run has a stream of its own: loading it (and reading its
                    # diagnostics when it ends) waits for that stream only, not for the chunk
                    # another run has in flight
                    stream = torch.cuda.Stream(priority=-1 if req.particles < self.large_particles
                                               else 0)
                loading[req.rid] = (loader.submit(make_run, req, tuner=self.tuner, stream=stream),
                                    req, need, lane)
                used += need
                self.peak_bytes = max(self.peak_bytes, used)
                progressed = True
            # runs the loader thread has finished join the lanes
            for rid in [r for r, v in loading.items() if v[0].done()]:
                fut, req, need, lane = loading.pop(rid)
                run = fut.result()
                active[rid] = {"run": run, "req": req, "done": 0, "bytes": need,
                               "admitted": time.perf_counter() - t0, "history": [],
                               "stream": run.stream, "lane": lane}
                if req.record_every > 0:
                    self._record(active[rid])
                progressed = True
            self.max_active = max(self.max_active, len(active))
            # the batch lanes: account finished chunks, change the run set, keep up to
            # `depth` chunks queued on the lane's stream (the GPU does not wait for the host
            # between chunks) as long as no run of the set reaches a field-energy sample or its
            # last step and no admitted run waits to join
            urgent = preempt and (any(a["lane"] == 0 for a in active.values())
                                        or any(v[3] == 0 for v in loading.values()))
            urgent = hold.hold(urgent, time.perf_counter())
            for li, lane in enumerate(lanes):
                done_chunk = False
                while lane.inflight and lane.inflight[0][0].query():
                    ev, k, ev0 = lane.inflight.popleft()
                    for r in lane.ids:
                        active[r]["done"] += k
                    st = self.lane_stats[li]
                    st["chunks"] += 1
                    st["steps"] += k
                    st["run_steps"] += k * len(lane.ids)
                    st["gpu_ms"] += ev0.elapsed_time(ev)
                    done_chunk = True
                if lane.inflight:
                    if done_chunk:
                        progressed = True
                else:
                    if done_chunk:
                        rec = [active[r] for r in lane.ids if recorded(active[r])]
                        fin = [r for r in lane.ids if active[r]["done"] >= active[r]["req"].steps]
                        if rec and not fin:
                            lane.batch.sync()
                        if fin:  # the finished runs leave the batch (their state written back)
                            install(li, tuple(r for r in lane.ids if r not in fin))
                        for a in rec:
                            self._record(a)
                        for r in fin:
                            finish(r)
                        progressed = True
                    ids = tuple(sorted(r for r, a in active.items() if a["lane"] == li))
                    if ids != lane.ids:
                        install(li, ids)
                if lane.batch is None or not lane.ids:
                    continue
                if li > 0 and urgent:
                    continue
                joining = any(a["lane"] == li and r not in lane.ids for r, a in active.items())
                st = self.lane_stats[li]
                msps = st["gpu_ms"] / st["steps"] if li > 0 and st["steps"] else 0.0
                while len(lane.inflight) < self.depth:
                    ahead = sum(c[1] for c in lane.inflight)
                    if lane.inflight and (joining or stops(lane.ids, ahead)):
                        break
                    k = chunk_steps(lane.ids, ahead, msps)
                    if not lane.captured:
                        # the first step captures the batch's graph on the lane's stream, on
                        # which the loader thread also loads the lane's new runs: let it finish
                        cf.wait([v[0] for v in loading.values()])
                        lane.captured = True
                    ev0 = torch.cuda.Event(enable_timing=True)
                    ev0.record(lane.stream)
                    lane.batch.step(k)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(lane.stream)
                    lane.inflight.append((ev, k, ev0))
                    self.chunks += 1
                    progressed = True
            # the side lanes: every other run on its own stream; the runs of large_particles
            # and more (each one fills the GPU) take turns in arrival order, max_large at once
            large = sorted((a["req"].arrival, r) for r, a in active.items()
                           if a["lane"] < 0 and a["req"].particles >= self.large_particles)
            large_turn = {r for _, r in large[:self.max_large]}
            for rid in [r for r, a in active.items() if a["lane"] < 0]:
                a = active[rid]
                inf = side_inflight.get(rid)
                if inf is not None and not inf[0].query():
                    continue
                if inf is not None:
                    a["done"] += inf[1]
                    a["ms_per_step"] = inf[2].elapsed_time(inf[0]) / inf[1]
                    del side_inflight[rid]
                    if recorded(a):
                        self._record(a)
                    if a["done"] >= a["req"].steps:
                        finish(rid)
                        progressed = True
                        continue
                if urgent:
                    continue
                if a["req"].particles >= self.large_particles and rid not in large_turn:
                    continue
                # the first chunk of a side run is one step, which measures its step time
                k = chunk_steps([rid], 0, a.get("ms_per_step", 1e9 if preempt else 0.0))
                ev0 = torch.cuda.Event(enable_timing=True)
                ev0.record(a["stream"])
                a["run"].step(k)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(a["stream"])
                side_inflight[rid] = (ev, k, ev0)
                self.chunks += 1
                progressed = True
            if not progressed:
                if not active and not loading and pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - (time.perf_counter() - t0))))
                else:
                    time.sleep(0.0002)
        self.hold_releases = hold.releases
        loader.shutdown()
        for lane in lanes:
            if lane.batch is not None:
                lane.batch.close()
        return self.results

    @staticmethod
    def _record(a):
        req = a["req"]
        d = a["run"].diag()
        wp = 1.0 / 16.0  # omega_p of the drifting plasma (16 cells per skin depth, dx = 1)
        a["history"].append((a["done"], a["done"] * req.dt * wp, d["field_energy"],
                             d["kinetic_energy"]))


# The drifting pair-plasma NCI test of Table 1: 256 x 128 cells (16 x 8 skin depths), 64
# particles per cell, gamma0 = 1000, k T = 0.01 m c^2 in the co-moving frame (Gaussian momenta
# of spread sqrt(kT / m c^2) = 0.1, boosted with the App. D flip), l = 4, and
# dt / dt_CFL in {0.1, 0.3, 0.5, 0.7, 1/sqrt(2)} with dt_CFL = dx / (sqrt(2) c).
TABLE1_RATIOS = (0.1, 0.3, 0.5, 0.7, 1.0 / math.sqrt(2.0))


def table1_requests(t_end: float, record_dt: float = 1.0, schemes=(pic.PIC_SCHEME_MC, pic.PIC_SCHEME_WT),
                    solvers=(pic.PIC_SOLVER_YEE, pic.PIC_SOLVER_M4), ratios=TABLE1_RATIOS,
                    grid=(256, 128, 1), ppc=64, seed=1909096130, precision=pic.PIC_FP32_MIXED,
                    only=None, colocated=True):
    """One request per (scheme, solver, dt) of Table 1, run to t_end (in 1/omega_pe), sampling
    the field energy every record_dt; every run starts from the same seeded plasma.  `only`
    keeps the (scheme, solver, ratio index) triples listed.

    The start is neutral by default (positrons at the electrons' positions): with independent
    positions the initial charge noise, with zero fields, stays in the system as a frozen
    background (D.E - rho is conserved) through which the plasma streams at ~c, and that
    drives field growth unrelated to the interpolation scheme."""
    reqs = []
    for scheme in schemes:
        for solver in solvers:
            for ri, ratio in enumerate(ratios):
                if only is not None and (scheme, solver, ri) not in only:
                    continue
                # c dt / dx = ratio / sqrt(2); the last ratio is exactly dx / 2 (WT = MC there)
                dt = 0.5 if abs(ratio * math.sqrt(2.0) - 1.0) < 1e-12 else ratio / math.sqrt(2.0)
                steps = int(math.ceil(t_end * 16.0 / dt))
                every = max(1, int(round(record_dt * 16.0 / dt)))
                steps = (steps + every - 1) // every * every
                reqs.append(Request(rid=len(reqs), grid=grid, dt=dt, l=4, gamma=1000.0, u_th=0.1,
                                    ppc=ppc, steps=steps, scheme=scheme, seed=seed, solver=solver,
                                    record_every=every, rng_run=0, precision=precision,
                                    colocated=colocated))
    return reqs


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return v[lo] + (v[hi] - v[lo]) * (k - lo)
