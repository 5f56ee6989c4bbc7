#!/usr/bin/env python
"""Benchmark of the WT-scheme PIC step on GB300 (one JSON line on rank 0).

Workload (default): the 2048x1024 periodic drifting pair plasma, cubic B-splines, WT gather,
gamma = 50, u_th = 0.01 (App. D loading, generated in HBM by the library's device loader),
64 particles per cell = 134,217,728 particles, c dt = 0.25 dx, in the plain FP64 single-run
form.  A step is one full PIC step through
pic_step: gather + Boris + move + Esirkepov deposit (the fused particle kernel), the periodic
Yee update, and the tile sort every sort_interval steps.  The same workload in the precision
form (int32 cell + FP32 offset, FP32 push/gather/tile current, FP64 fields) is reported under
"precision_form".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the run (independent runs, no
collective on the data path); value = particle-steps of all ranks / max-over-ranks time.
--impl reference times the FP64 CPU oracle (its OpenMP timing build, all host cores) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit), batched vs plain; p50/p99 run latency"
UNIT = "particle-steps/s"
WORKLOAD = "pair_2048x1024_l3_WT_g50_uth0.01_ppc64_cdt0.25"

# Algorithmic bytes of the fused particle kernel (per particle-step, per cell-step):
#   FP64 form: particle read + write 2 x (2 x 8 position + 3 x 8 momentum) = 80 B per
#              particle-step (the method's bytes); grid: E, B read once (6 x 8 B) + J written
#              (3 x 8 B) = 72 B per cell.  The kernel also reads and writes the B-spline
#              weights of the stored positions, 2 x 2 (l + 1) x 8 B = 128 B for l = 3, a cache
#              that spends HBM bytes to save FP64 instructions (the form is bound by its FP64
#              pipe), reported beside the roofline as extra traffic.
#   FP32 form: 2 x (4 cell + 2 x 4 offset + 3 x 4 momentum) = 48 B;
#              grid: FP32 shadow of E, B (6 x 4 B) + FP64 J (3 x 8 B) = 48 B per cell.
# Algorithmic bytes per particle-step and per cell-step of each form (the method's per-unit
# figures): the particle state read and written once, and the grid traffic of a whole step per
# cell (FP64: gather 48 + J 72 + Yee 120; FP32: FP64 Yee 192 + FP32 shadows 24 + gather 24 +
# J 72), amortised over the particles.  KERNEL_GRID_BYTES: the particle kernel's own grid bytes
# (fields read, current written), for the kernel-only view reported beside the roofline.
BYTES = {"fp64": (80.0, 240.0), "fp32": (48.0, 310.0)}
KERNEL_GRID_BYTES = {"fp64": 72.0, "fp32": 48.0}
WEIGHT_CACHE_BYTES_FP64_L3 = 128.0
SCHEDULERS_PER_SM = 4
# The particle kernel's sources: the counts of profiles/counts.txt (from one ncu capture) are
# used only while these files hash to the digest recorded with them.
KERNEL_SOURCES = ("pic_common.cuh", "pic_gpp.cuh", "pic_gpp_kernels.cuh", "pic_gpp_f32.cu",
                  "pic_gpp_f64.cu")


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_digest():
    """sha256 (16 hex digits) of the particle kernel's source files with comments and blank
    space left out: an edit of a comment does not change the kernel the counts describe."""
    import hashlib
    import re
    from paper_1909_09613_gb300 import _build
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        txt = open(os.path.join(_build.CSRC, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        txt = "\n".join(line.strip() for line in txt.splitlines() if line.strip())
        h.update(txt.encode())
    return h.hexdigest()[:16]


def profile_counts(kernel: str):
    """The counts recorded from an ncu capture of `kernel` (profiles/counts.txt: kernel, source
    digest, key=value ...), if the kernel sources still hash to the recorded digest; else {}
    (the numbers no longer describe the code)."""
    path = os.path.join(ROOT, "profiles", "counts.txt")
    try:
        digest = kernel_digest()
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
                return {k: float(v) for k, v in (p.split("=") for p in parts[2:])}
    except Exception:
        pass
    return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = max(smax, float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _barrier(dist_on):
    if dist_on:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(v, dist_on):
    """Largest value over the ranks (the slowest replica's time); NCCL on the GPUs, or gloo on
    the host."""
    if not dist_on:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(particles_per_rank, world, steps, ms_max):
    """Whole-job particle-steps/s of `world` independent replicas that each advance
    `particles_per_rank` particles `steps` steps, the slowest taking ms_max milliseconds."""
    return particles_per_rank * world * steps / (ms_max * 1e-3)


def load_device(run, wl):
    """Generate the workload's plasma in the run's stores with the device loader (App. D)."""
    for i, s in enumerate(wl.species):
        if wl.theta > 0.0:
            run.load_drifting_juttner(i, s.q, s.m, s.w, s.per_cell, wl.gamma, wl.theta,
                                      seed=wl.seed, run=wl.run, pos_species=s.pos_species)
        else:
            run.load_drifting_plasma(i, s.q, s.m, s.w, s.per_cell, wl.gamma, wl.u_th,
                                     seed=wl.seed, run=wl.run, pos_species=s.pos_species)


def time_form(wl, prec, steps, warmup, dist_on, clocks=True):
    """Load the workload on the device (inputs resident in HBM), warm up, time `steps` full
    steps with CUDA events on the run's stream."""
    import torch
    import paper_1909_09613_gb300 as pic
    caps = [wl.ncell * s.per_cell for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps)
    load_device(run, wl)
    run.step(warmup)
    run.sync()
    stream = run.stream
    sampler = ClockSampler(torch.cuda.current_device()) if clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    k0 = run.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    _barrier(dist_on)
    torch.cuda.synchronize()
    e0.record(stream)
    run.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(dist_on)
    ms = e0.elapsed_time(e1)
    gpp_ms, gpp_n = run.gpp_ms()
    launches = run.kernel_launches() - k0
    clk = sampler.stop() if sampler else None
    run.sync()
    d = run.diag()
    run.step(1)
    d1 = run.diag()  # one step after the previous pic_diag: the continuity residual
    out = {"ms": _max_over_ranks(ms, dist_on), "gpp_ms": gpp_ms, "gpp_launches": gpp_n,
           "launches": launches, "clocks": clk, "n": sum(caps), "ncell": wl.ncell,
           "sort_interval": run.sort_interval, "tile": run.tile, "diag_status": d["status"],
           "charge_conservation": {
               "max_continuity_residual": d1["max_continuity_residual"],
               "max_gauss_residual_drift": d1["max_gauss_residual_drift"],
               "rho_scale": abs(wl.species[0].q * wl.species[0].w) * wl.species[0].per_cell},
           "run": run}
    return out


def e2e_form(run, wl, steps):
    """Same metric through the public C-ABI from pinned host buffers: load (H2D, pack, sort) +
    steps + diagnostics read-back (D2H), every byte counted.  The host arrays are the run's
    own initial state, read back once before timing (the same plasma the device loader drew)."""
    import torch
    import paper_1909_09613_gb300 as pic
    xs, us = [], []
    for i in range(len(wl.species)):
        x, u, _ = run.particles(i)
        xs.append(torch.from_numpy(x).pin_memory())
        us.append(torch.from_numpy(u).pin_memory())
        del x, u
    h2d = sum(x.numel() * 8 + u.numel() * 8 for x, u in zip(xs, us))

    def load():
        for i, s in enumerate(wl.species):
            st = pic.load_library().pic_load_particles(
                run.ctx, i, s.q, s.m, s.w, int(xs[i].shape[1]),
                pic.ctypes.cast(pic.ctypes.c_void_p(xs[i].data_ptr()), pic._c_dp),
                pic.ctypes.cast(pic.ctypes.c_void_p(us[i].data_ptr()), pic._c_dp))
            if st != 0:
                raise pic.PicError(st, "pic_load_particles")

    # warm-up: untimed passes through the same calls until two successive loads agree within
    # 15% (at most 6): the host-to-device rate from freshly pinned pages, and while the host is
    # still settling after earlier processes, varies several-fold for a few seconds
    warm = []
    for _ in range(6):
        torch.cuda.synchronize()
        tw = time.perf_counter()
        load()
        warm.append(time.perf_counter() - tw)
        if len(warm) >= 2 and abs(warm[-1] - warm[-2]) <= 0.15 * warm[-1]:
            break
    run.step(1)
    run.diag()
    # three timed passes (load + steps + diagnostics); the median one is reported, since a
    # single host-to-device load now and then takes several times its usual time
    passes = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        load()
        tl = time.perf_counter()  # pic_load_particles returns after its sort has completed
        run.step(steps)
        d = run.diag()
        t1 = time.perf_counter()
        passes.append((t1 - t0, tl - t0, t1 - tl, d["status"]))
    passes.sort()
    tot, tload, tsteps, status = passes[1]
    d2h = 72  # pic_diag_t
    n = sum(int(x.shape[1]) for x in xs)
    return {"value": n * steps / tot, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d / steps), "d2h_bytes_per_step": int(math.ceil(d2h / steps)),
            "status": status, "load_s": tload, "steps_and_diag_s": tsteps,
            "passes_s": [round(p[0], 4) for p in passes],
            "timing": "median of three timed passes (load + steps + pic_diag)",
            "warmup": "untimed loads until two agree within 15%, then a step and pic_diag",
            "warmup_load_s": [round(w, 4) for w in warm]}


def cpu_baseline(budget_s=8.0, one_core=True):
    """The FP64 oracle as it stands (its OpenMP timing build: particles split over threads,
    per-thread current buffers added at the end), on all host cores and on one core, over a
    bounded sample of the large workload: the particle pass (gather + push + deposit) of the
    same plasma on a 256x128 section of the grid (64 per cell, the same per-particle work;
    the oracle's cost is per particle).  Returns a dict for the bench line."""
    import oracle
    import workloads
    oracle.build(timing=True)
    wl = workloads.config_large(scheme=1, scale=8)
    ncores = os.cpu_count() or 1
    try:
        nproc = int(subprocess.run(["nproc"], capture_output=True, text=True).stdout.strip())
    except Exception:
        nproc = ncores
    sim = oracle.Sim(wl.grid[:2], wl.dx[:2], wl.dt, wl.l, wl.scheme, timing=True)
    n_per = wl.ncell * wl.species[0].per_cell
    for i, s in enumerate(wl.species):
        x, u, _ = oracle.load_drifting(wl.grid, wl.dx, s.per_cell, wl.gamma, wl.u_th, 0.0,
                                       wl.seed, wl.run, i, s.pos_species)
        sim.add_species(s.q, s.m, s.w, x, u)
        del x, u
    out = {"unit": UNIT, "kind": "oracle", "nproc": nproc}
    modes = [("all_cores", nproc, n_per)]
    if one_core:
        modes.append(("one_core", 1, max(1, n_per // 32)))
    for name, threads, count in modes:
        t0 = time.perf_counter()
        used = sim.particle_pass_threads(0, count, threads)
        one = time.perf_counter() - t0
        reps = max(1, int(budget_s / max(one, 1e-6)))
        t0 = time.perf_counter()
        for _ in range(reps):
            sim.particle_pass_threads(0, count, threads)
        t = time.perf_counter() - t0
        out[name] = {"value": 2 * count * reps / t, "cores": used,
                     "sample": "%d particle passes over %d particles (%d per species) of the "
                               "256x128 section (64 per cell) of the large workload"
                               % (reps, 2 * count, count)}
    sim.close()
    out["value"] = out["all_cores"]["value"]
    out["cores"] = out["all_cores"]["cores"]
    out["sample"] = out["all_cores"]["sample"]
    return out


def batched_form(steps, warmup, n_runs=256, max_nx=512, baselines=True):
    """Config 4: 256 uneven 2D runs (FP32 form, WT, autotuned tiles) in one persistent particle
    kernel per step, replayed from a CUDA graph; against the same runs stepped one after another
    through pic_step (FP32 form, and the plain FP64 form)."""
    import torch
    import workloads
    import paper_1909_09613_gb300 as pic
    from paper_1909_09613_gb300 import engine
    specs = workloads.batched_runs(n_runs, max_nx=max_nx)
    reqs = [engine.Request(rid=i, grid=sp["grid"], dt=sp["dt"], l=sp["l"], gamma=sp["gamma"],
                           u_th=sp["u_th"], ppc=sp["ppc"], steps=sp["steps"], seed=workloads.BASE_SEED)
            for i, sp in enumerate(specs)]
    tuner = engine.Autotuner()
    t0 = time.perf_counter()
    runs = [engine.make_run(r, tuner=tuner) for r in reqs]
    setup_s = time.perf_counter() - t0
    n_part = sum(r.particles for r in reqs)
    b = pic.Batch(runs)
    b.step(warmup)
    gpp_ms = b.time_gpp()
    torch.cuda.synchronize()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    b.step(steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t1) * 1e3
    b.sync()
    items, launches = b.info()
    b.close()
    flags = sum(r.diag()["error_flags"] for r in runs)
    # the persistent particle kernel against the measured HBM copy rate, with the precision
    # form's algorithmic bytes (particle state read and written, fields read and current written)
    ncell = sum(int(math.prod(r.grid)) for r in reqs)
    pb, gb = BYTES["fp32"]
    alg = n_part * pb + ncell * gb
    peaks, peak_kind = _peaks()
    ach = alg / (gpp_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None,
                "kernel": "k_b_gpp (persistent, every run's tiles)", "kernel_ms": gpp_ms,
                "algorithmic_bytes": alg, "bytes_per_unit": {"particle": pb, "cell": gb},
                "peak_source": "%s hbm_gbs" % peak_kind}
    if not baselines:
        for r in runs:
            r.close()
        return {"value": n_part * steps / (ms * 1e-3), "unit": UNIT, "runs": n_runs,
                "particles": n_part, "ms_per_step": ms / steps, "gpp_ms_per_step": gpp_ms,
                "roofline": roofline, "error_flags": flags}
    # the same runs one after another, each through pic_step (FP32 form)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for r in runs:
        r.step(1)
    torch.cuda.synchronize()
    seq32_ms = (time.perf_counter() - t1) * 1e3
    for r in runs:
        r.close()
    del runs
    torch.cuda.empty_cache()
    # plain FP64 form, one after another (a step of each run)
    seq64 = []
    t64 = 0.0
    for r in reqs:
        run = engine.make_run(r, precision=pic.PIC_FP64)
        run.step(1)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        run.step(1)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - ta
        run.close()
    torch.cuda.empty_cache()
    return {"value": n_part * steps / (ms * 1e-3), "unit": UNIT, "runs": n_runs,
            "particles": n_part, "steps": steps, "ms_per_step": ms / steps,
            "gpp_ms_per_step": gpp_ms, "work_items": items, "launches_per_step": launches,
            "roofline": roofline,
            "graph": "one CUDA graph per batch step, replayed",
            "sequential_fp32_particle_steps_per_s": n_part / (seq32_ms * 1e-3),
            "sequential_fp64_plain_particle_steps_per_s": n_part / t64,
            "speedup_vs_sequential_fp32": (n_part * steps / (ms * 1e-3)) / (n_part / (seq32_ms * 1e-3)),
            "speedup_vs_sequential_fp64_plain": (n_part * steps / (ms * 1e-3)) / (n_part / t64),
            "autotuned": {"%d_%d" % k: {"tile": v[0], "sort_interval_factor": v[1]}
                          for k, v in tuner.cache.items()},
            "setup_s": setup_s, "error_flags": flags}


def table1_form(t_end=300.0, record_dt=1.0, history_path=None, precision="fp32", only=None,
                colocated=True):
    """The Table 1 NCI scan (MC4 / WT4 x Yee / M4 x five time steps, 256x128, 64 particles per
    cell, gamma0 = 1000) served as 20 concurrent NCI-scan requests in the FP32 form, each
    recording E/E0 (field energy over the initial kinetic energy) every record_dt / omega_pe."""
    import numpy as np
    import paper_1909_09613_gb300 as pic
    from paper_1909_09613_gb300 import engine
    prec = pic.PIC_FP64 if precision == "fp64" else pic.PIC_FP32_MIXED
    sel = None
    if only:
        # "WT4:Yee:0,MC4:M4:4": scheme, solver, index into the Table 1 time steps
        sel = set()
        for item in only.split(","):
            sc, so, ri = item.split(":")
            sel.add((pic.PIC_SCHEME_WT if sc == "WT4" else pic.PIC_SCHEME_MC,
                     pic.PIC_SOLVER_M4 if so == "M4" else pic.PIC_SOLVER_YEE, int(ri)))
    reqs = engine.table1_requests(t_end, record_dt, precision=prec, only=sel, colocated=colocated)
    srv = engine.Server(budget_bytes=150e9, chunk=64)
    t0 = time.perf_counter()
    res = srv.serve(reqs)
    wall = time.perf_counter() - t0
    byid = {r.rid: r for r in res}
    runs = []
    for q in reqs:
        h = np.array(byid[q.rid].history)          # step, t, U_EM, K
        e0 = h[0, 3]
        ratio = h[:, 2] / e0
        t = h[:, 1]
        half = t >= t[-1] / 2
        slope = float(np.polyfit(t[half], np.log(np.maximum(ratio[half], 1e-300)), 1)[0])
        above = np.nonzero(ratio > 1e-3)[0]
        runs.append({"scheme": "WT4" if q.scheme == pic.PIC_SCHEME_WT else "MC4",
                     "solver": "M4" if q.solver == pic.PIC_SOLVER_M4 else "Yee",
                     "dt_over_dt_cfl": round(q.dt * math.sqrt(2.0), 4), "c_dt_over_dx": q.dt,
                     "steps": q.steps, "E_over_E0_max": float(ratio.max()),
                     "E_over_E0_end": float(ratio[-1]),
                     "E_over_E0_at": {str(int(x)): float(np.interp(x, t, ratio))
                                      for x in (10, 30, 100, 300, 1000) if x <= t[-1]},
                     "growth_rate_second_half": slope,
                     "t_first_above_1e-3": float(t[above[0]]) if len(above) else None,
                     "error_flags": byid[q.rid].diag.get("error_flags")})
        if history_path:
            q_tag = "%s_%s_%.4f" % (runs[-1]["scheme"], runs[-1]["solver"], runs[-1]["dt_over_dt_cfl"])
            np.savetxt("%s_%s.txt" % (history_path, q_tag), np.column_stack([t, ratio]),
                       header="t_omega_pe E_over_E0", fmt="%.6g")
    work = sum(q.particles * q.steps for q in reqs)
    return {"form": "table1", "t_end_omega_pe": t_end, "runs": runs, "wall_s": wall,
            "particle_steps_per_s": work / wall, "max_concurrent_runs": srv.max_active,
            "dtype": "f64" if precision == "fp64" else "f32 (FP64 fields)",
            "workload": "pair_256x128_l4_g1000_kT0.01_ppc64 (Table 1)",
            "start": "neutral (e+ at the e- positions)" if colocated else "independent positions"}


def form_3d(steps=10, warmup=3):
    """The 3D path (the served form's 3D requests): a 256x64x64 drifting pair plasma, 8 particles
    per cell (8,388,608 particles), quadratic WT, c dt = 0.4, gamma 20, in both forms; device-
    resident inputs, CUDA events around whole steps."""
    import torch
    import workloads
    import paper_1909_09613_gb300 as pic
    wl = workloads.pair_plasma((256, 64, 64), (1.0, 1.0, 1.0), 0.4, 2, 1, 20.0, 0.01, 8)
    caps = [wl.ncell * s.per_cell for s in wl.species]
    out = {"workload": "pair_256x64x64_l2_WT_g20_ppc8_cdt0.4", "particles": sum(caps)}
    for name, prec in (("fp32", pic.PIC_FP32_MIXED), ("fp64", pic.PIC_FP64)):
        r = pic.Run(wl.grid, wl.dx, wl.dt, 2, 1, precision=prec, capacity=caps)
        load_device(r, wl)
        r.step(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(r.stream)
        r.step(steps)
        e1.record(r.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"value": sum(caps) / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "tile": list(r.tile), "error_flags": r.diag()["error_flags"]}
        r.close()
    return out


def loader_form(reps=3):
    """The device loader (App. D) on the 2048x1024 grid, 64 per cell (134,217,728 particles) in
    the plain FP64 form: both species generated in HBM, Gaussian co-moving momenta (gamma 50,
    u_th 0.01) and Juttner-Synge momenta (theta 1, Sobol's method), each call timed from issue
    to return (generation, packing and the tile sort; the call synchronises)."""
    import torch
    import paper_1909_09613_gb300 as pic
    grid, ppc, gamma = (2048, 1024), 64, 50.0
    n = grid[0] * grid[1] * ppc // 2
    r = pic.Run(grid, (1.0, 1.0), 0.25, 3, 1, precision=pic.PIC_FP64, capacity=[n, n])
    w = 1e-3
    out = {"workload": "pair_2048x1024_ppc64_loader", "particles": 2 * n}
    for name, call in (("gaussian_u_th0.01",
                        lambda s, k: r.load_drifting_plasma(s, -1.0 + 2 * s, 1.0, w, ppc // 2,
                                                            gamma, 0.01, seed=k, pos_species=0)),
                       ("juttner_theta1",
                        lambda s, k: r.load_drifting_juttner(s, -1.0 + 2 * s, 1.0, w, ppc // 2,
                                                             gamma, 1.0, seed=k, pos_species=0))):
        best = None
        for k in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            call(0, 11 + k)
            call(1, 11 + k)
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        out[name] = {"particles_per_s": 2 * n / best, "ms": best * 1e3, "reps": reps,
                     "error_flags": r.diag()["error_flags"]}
    r.close()
    return out


def served_form(n_req=48, steps=500, budget=150e9, seed=None, alone_steps=100):
    """Config 5: a Poisson stream of NCI-scan requests, 90% drawn from the batched distribution
    and 10% 3D (128x32x32, 256x64x64 or 512x128x128 cells, 8 per cell, drift along x1), 500 steps
    each, admitted under a 150 GB budget and served by continuous batching (engine.Server), the
    arrival rate 0.8 x the measured service capacity of this mix.  Reports the latency
    (completion - arrival) p50/p99, every request's slowdown against its latency alone (the
    same form alone on the GPU: its set-up and load, its steps timed over alone_steps steps and
    scaled to its steps, and the final diagnostics read, the span the served latency covers; the
    slowdown against the steps alone is reported beside it), and the aggregate particle-steps/s."""
    import random
    import torch
    import workloads
    import paper_1909_09613_gb300 as pic
    from paper_1909_09613_gb300 import engine
    rng = random.Random(workloads.BASE_SEED if seed is None else seed)
    specs = workloads.served_requests(n_req, seed=workloads.BASE_SEED, steps=steps)
    reqs = [engine.Request(rid=i, grid=sp["grid"], dt=sp["dt"], l=sp["l"], gamma=sp["gamma"],
                           u_th=sp["u_th"], ppc=sp["ppc"], steps=sp["steps"],
                           seed=workloads.BASE_SEED) for i, sp in enumerate(specs)]
    tuner = engine.Autotuner()
    # every request alone, in its own form: the latency baseline (what a server with nothing
    # else to do takes: the run's set-up and load, its steps and the final diagnostics read;
    # the steps timed over alone_steps and scaled), and the 3D throughput
    alone, alone_steps_only, work3d, t3d = {}, {}, 0.0, 0.0
    for r in reqs:  # tune first: a request's set-up time must not include the autotuner's probes
        engine.request_tile(r, tuner)
    for r in reqs:
        torch.cuda.synchronize()
        ts = time.perf_counter()
        run = engine.make_run(r, tuner=tuner)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - ts
        run.step(2)
        torch.cuda.synchronize()
        n = min(r.steps, alone_steps)
        ta = time.perf_counter()
        run.step(n)
        torch.cuda.synchronize()
        t = time.perf_counter() - ta
        td = time.perf_counter()
        run.diag()
        t_diag = time.perf_counter() - td
        alone_steps_only[r.rid] = t * r.steps / n
        alone[r.rid] = t_setup + alone_steps_only[r.rid] + t_diag
        if r.dim == 3:
            work3d += r.particles * n
            t3d += t
        run.close()
    torch.cuda.empty_cache()
    # 2D service capacity: the batch of the 2D requests at once, steps timed
    probe = [engine.make_run(r, tuner=tuner) for r in reqs if r.dim == 2]
    b = pic.Batch(probe)
    b.step(2)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    b.step(10)
    torch.cuda.synchronize()
    cap2d = sum(p.counts[0] + p.counts[1] for p in probe) * 10 / (time.perf_counter() - t1)
    b.close()
    for p in probe:
        p.close()
    torch.cuda.empty_cache()
    cap3d = work3d / t3d if t3d > 0 else cap2d
    w2d = sum(r.particles * r.steps for r in reqs if r.dim == 2)
    w3d = sum(r.particles * r.steps for r in reqs if r.dim == 3)
    cap = (w2d + w3d) / (w2d / cap2d + w3d / cap3d)
    mean_work = (w2d + w3d) / len(reqs)
    lam = 0.8 * cap / mean_work
    t = 0.0
    for r in reqs:
        t += rng.expovariate(lam)
        r.arrival = t
    srv = engine.Server(budget_bytes=budget, chunk=10, tuner=tuner)
    t0 = time.perf_counter()
    res = srv.serve(reqs)
    makespan = time.perf_counter() - t0
    lat = [r.latency for r in res]
    slow = [r.latency / alone[r.rid] for r in res]
    slow_steps = [r.latency / alone_steps_only[r.rid] for r in res]
    lat2d = [r.latency for r in res if r.dim == 2]
    slow2d = [r.latency / alone[r.rid] for r in res if r.dim == 2]
    wait2d = [r.admitted - r.arrival for r in res if r.dim == 2]
    work = sum(r.particles * r.steps for r in res)
    # the plain FP64 single-run form on a sample of the 2D requests, alone
    alone64 = []
    for r in [q for q in reqs if q.dim == 2][:6]:
        run = engine.make_run(r, precision=pic.PIC_FP64)
        torch.cuda.synchronize()
        n = min(r.steps, alone_steps)
        ta = time.perf_counter()
        run.step(n)
        torch.cuda.synchronize()
        alone64.append((time.perf_counter() - ta) * r.steps / n)
        run.close()
    return {"value": work / makespan, "unit": UNIT, "requests": len(res),
            "p50_latency_s": engine.percentile(lat, 50), "p99_latency_s": engine.percentile(lat, 99),
            "p50_slowdown_vs_alone": engine.percentile(slow, 50),
            "p99_slowdown_vs_alone": engine.percentile(slow, 99),
            "p50_slowdown_vs_alone_steps_only": engine.percentile(slow_steps, 50),
            "p99_slowdown_vs_alone_steps_only": engine.percentile(slow_steps, 99),
            "p50_latency_2d_s": engine.percentile(lat2d, 50),
            "p50_slowdown_2d": engine.percentile(slow2d, 50),
            "p50_admission_wait_2d_s": engine.percentile(wait2d, 50),
            "p50_alone_latency_s": engine.percentile(list(alone.values()), 50),
            "p50_alone_steps_only_s": engine.percentile(list(alone_steps_only.values()), 50),
            "arrival_rate_per_s": lam, "arrival_window_s": reqs[-1].arrival,
            "service_capacity_particle_steps_per_s": cap,
            "capacity_2d_batched": cap2d, "capacity_3d_alone": cap3d,
            "makespan_s": makespan, "max_concurrent_runs": srv.max_active,
            "batch_builds": srv.batch_builds, "batch_set_changes": srv.set_changes,
            "batch_lane_runs": srv.lane_runs, "longest_host_block_s": srv.host_block_s,
            "hold_releases": srv.hold_releases,
            "batch_lanes": [{"chunks": st["chunks"], "steps": st["steps"],
                             "mean_runs_per_step": st["run_steps"] / max(st["steps"], 1),
                             "ms_per_step": st["gpu_ms"] / max(st["steps"], 1)}
                            for st in srv.lane_stats],
            "peak_admitted_bytes": srv.peak_bytes, "budget_bytes": budget,
            "steps_per_request": steps, "requests_3d": sum(1 for r in reqs if r.dim == 3),
            "largest_3d_grid": max((list(r.grid) for r in reqs if r.dim == 3), default=None,
                                   key=lambda g: g[0] * g[1] * g[2]),
            "alone_fp64_plain_latency_s_sample": alone64,
            "alone": "every request alone in its own form: set-up and load, its steps (timed "
                     "over %d and scaled) and the final diagnostics read; steps_only: the steps "
                     "alone" % alone_steps,
            "error_flags": sum(r.diag.get("error_flags", 0) for r in res)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=1, help="divide the grid extents (debug)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--t-end", type=float, default=300.0, help="table1 form: run length, 1/omega_pe")
    ap.add_argument("--history", default=None, help="table1 form: prefix of E/E0 history files")
    ap.add_argument("--t1-precision", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--t1-only", default=None, help="table1 form: e.g. WT4:Yee:0,MC4:M4:4")
    ap.add_argument("--t1-independent", action="store_true",
                    help="table1 form: species at independent positions (non-neutral start)")
    ap.add_argument("--form", default="both", choices=["both", "fp64", "fp32", "batched", "served",
                                                       "table1", "3d"],
                    help="fp32/batched/served/3d: time only that form (profiling runs)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--runs", type=int, default=256, help="batched form: number of runs")
    ap.add_argument("--max-nx", type=int, default=512, help="batched form: largest grid x")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--no-loader", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=None,
                    help="reference arm: seconds of oracle work per step (default: about a "
                         "minute over all steps)")
    args = ap.parse_args()
    rank, world, local = _rank_env()

    import workloads

    if args.impl == "reference":
        if rank != 0:
            return
        rates, secs = [], []
        budget = (args.ref_budget if args.ref_budget is not None
                  else max(1.0, 30.0 / max(1, args.steps + args.warmup)))
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            cb = cpu_baseline(budget_s=budget, one_core=False)
            if i >= args.warmup:
                rates.append(cb["value"])
                secs.append(time.perf_counter() - t0)
        v = statistics.median(rates)
        # a step of this arm is one bounded sample of the workload (see cpu_baseline.sample)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * statistics.median(secs),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid_sample": "256x128 (same per-particle work)"},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                 "nproc": cb["nproc"], "sample": cb["sample"]},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    dist_on = world > 1
    if dist_on:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group(backend="nccl")
    else:
        torch.cuda.set_device(0)
    import paper_1909_09613_gb300 as pic
    from paper_1909_09613_gb300 import _build
    _build.build()
    pic.load_library()

    if args.form == "table1":
        out = table1_form(args.t_end, history_path=args.history, precision=args.t1_precision,
                          only=args.t1_only, colocated=not args.t1_independent)
        if rank == 0:
            print(json.dumps(out))
        return
    wl = workloads.config_large(scheme=1, seed=workloads.BASE_SEED + rank, scale=args.scale)
    if args.form in ("batched", "served"):
        out = (batched_form(args.steps, args.warmup, args.runs, args.max_nx,
                            baselines=args.runs == 256 and args.max_nx == 512)
               if args.form == "batched" else served_form())
        if rank == 0:
            print(json.dumps({"form": args.form, **out}))
        return
    if args.form == "3d":
        out = form_3d(args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"form": "3d", **out}))
        return
    if args.form == "fp32":
        r32 = time_form(wl, pic.PIC_FP32_MIXED, args.steps, args.warmup, dist_on, clocks=False)
        r32.pop("run").close()
        if rank == 0:
            print(json.dumps({"form": "fp32", "ms_per_step": r32["ms"] / args.steps,
                              "gpp_ms": r32["gpp_ms"] / max(r32["gpp_launches"], 1),
                              "particles": r32["n"]}))
        return
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    digest = kernel_digest()
    res = time_form(wl, pic.PIC_FP64, args.steps, args.warmup, dist_on)
    run64 = res.pop("run")
    value = replica_rate(res["n"], world, args.steps, res["ms"])
    gpp_avg_s = res["gpp_ms"] / max(res["gpp_launches"], 1) * 1e-3
    peaks, peak_kind = _peaks()
    pb, gb = BYTES["fp64"]
    alg_bytes = res["n"] * pb + res["ncell"] * gb
    c64 = profile_counts("gpp2d_fp64")
    traffic64 = c64.get("dram_bytes_per_launch")
    fp64_peak = None
    try:
        fp64_peak = pic.pic_probe_fma_peak(0)
    except Exception:
        pass
    hbm_view = {"achieved_gbs": alg_bytes / gpp_avg_s / 1e9,
                "frac_of_measured_hbm": alg_bytes / gpp_avg_s / 1e9 / peaks["hbm_gbs"],
                "weight_cache_bytes_per_particle": WEIGHT_CACHE_BYTES_FP64_L3,
                "traffic_over_algorithmic": (traffic64 / alg_bytes) if traffic64 else None,
                "note": "the DRAM traffic includes the read and write of the cached B-spline "
                        "weights (128 B per particle-step), bytes spent to save FP64 "
                        "instructions in a form bound by its FP64 pipe"}
    flops = c64.get("fp64_flops_per_particle")
    if flops and fp64_peak:
        ach = res["n"] * flops / gpp_avg_s / 1e12
        roofline = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": ach / fp64_peak, "traffic": traffic64,
                    "peak_source": "measured FP64 FMA rate (pic_probe_fma_peak, all SMs)",
                    "flops_per_particle": flops,
                    "fp64_instr_frac": (res["n"] * c64.get("fp64_instr_per_particle", 0.0) / gpp_avg_s)
                                       / (fp64_peak * 1e12 / 2.0),
                    "hbm_view": hbm_view}
    else:
        ach = alg_bytes / gpp_avg_s / 1e9
        roofline = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": traffic64,
                    "peak_source": "%s hbm_gbs" % peak_kind,
                    "note": "no FP64 instruction count recorded for these kernel sources"}
    roofline["kernel"] = "k_gpp2d<3,4> (double): fused gather+push+move+deposit"
    roofline["kernel_ms"] = gpp_avg_s * 1e3
    roofline["algorithmic_bytes"] = alg_bytes
    roofline["counts_digest"] = digest
    roofline["counts_from_profile"] = bool(c64)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded, generated in HBM by the device loader)",
            "config": {"workload": WORKLOAD, "grid": list(wl.grid[:2]), "particles": res["n"],
                       "form": "plain FP64 single run", "spline_order": wl.l, "scheme": "WT",
                       "c_dt_over_dx": wl.dt, "sort_interval": res["sort_interval"],
                       "tile": list(res["tile"]),
                       "l2": "no flush: inputs larger than L2 (%.1f GB particle store)" % (res["n"] * 40 / 1e9),
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline,
            "gpu_launches": res["launches"],
            "clocks": res["clocks"],
            "sms": sms,
            "fp64_fma_peak_tflops": fp64_peak,
            "gpp_particle_steps_per_s": res["n"] / gpp_avg_s,
            "charge_conservation": res["charge_conservation"],
            # per step: the particle kernel (gather + push + deposit) and the rest (Yee, the
            # tile sort amortised over its interval, clearing the current)
            "split_ms_per_step": {"gather_push_deposit": gpp_avg_s * 1e3,
                                  "yee_sort_other": res["ms"] / args.steps - gpp_avg_s * 1e3}}
    if not args.no_e2e:
        try:
            line["e2e"] = e2e_form(run64, wl, args.steps)
        except Exception as ex:  # report, do not hide
            line["e2e"] = {"error": str(ex)}
    run64.close()
    del run64
    torch.cuda.empty_cache()

    if not args.no_fp32 and args.form == "both":
        r32 = time_form(wl, pic.PIC_FP32_MIXED, args.steps, args.warmup, dist_on)
        run32 = r32.pop("run")
        g32 = r32["gpp_ms"] / max(r32["gpp_launches"], 1) * 1e-3
        pb, gb = BYTES["fp32"]
        ab = r32["n"] * pb + r32["ncell"] * gb
        ach = ab / g32 / 1e9
        c32 = profile_counts("gpp2d_fp32")
        line["precision_form"] = {
            "value": replica_rate(r32["n"], world, args.steps, r32["ms"]), "unit": UNIT,
            "ms_per_step": r32["ms"] / args.steps, "dtype": "f32 (FP64 fields)",
            "gpp_particle_steps_per_s": r32["n"] / g32,
            "split_ms_per_step": {"gather_push_deposit": g32 * 1e3,
                                  "yee_sort_other": r32["ms"] / args.steps - g32 * 1e3},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"],
                         "traffic": c32.get("dram_bytes_per_launch"),
                         "kernel": "k_gpp2d<3,4> (float)", "kernel_ms": g32 * 1e3,
                         "algorithmic_bytes": ab, "peak_source": "%s hbm_gbs" % peak_kind,
                         "bytes_per_unit": {"particle": pb, "cell": gb},
                         "kernel_grid_only_frac": (r32["n"] * pb + r32["ncell"] * KERNEL_GRID_BYTES["fp32"])
                                                  / g32 / 1e9 / peaks["hbm_gbs"],
                         "counts_digest": digest, "counts_from_profile": bool(c32)},
            "charge_conservation": r32["charge_conservation"],
            "gpu_launches": r32["launches"], "clocks": r32["clocks"]}
        wip = c32.get("warp_instr_per_particle")
        if wip:
            mhz = (r32["clocks"] or {}).get("sm_mhz") or 2070.0
            issue_peak = sms * SCHEDULERS_PER_SM * mhz * 1e6
            issued = r32["n"] * wip / g32
            line["precision_form"]["roofline"]["issue_view"] = {
                "warp_instr_per_particle": wip,
                "achieved_warp_instr_per_s": issued, "peak_warp_instr_per_s": issue_peak,
                "frac": issued / issue_peak, "sm_mhz": mhz}
        if not args.no_e2e:
            try:
                line["precision_form"]["e2e"] = e2e_form(run32, wl, args.steps)
            except Exception as ex:  # report, do not hide
                line["precision_form"]["e2e"] = {"error": str(ex)}
        run32.close()
        del run32
        torch.cuda.empty_cache()
        try:
            line["fp32_fma_peak_tflops"] = pic.pic_probe_fma_peak(1)
        except Exception:
            pass

    if args.form == "both" and not args.no_batched:
        line["batched_form"] = batched_form(max(args.steps, 10), args.warmup)
    if args.form == "both" and not args.no_served:
        line["served_form"] = served_form()
    if args.form == "both" and not args.no_3d:
        line["form_3d"] = form_3d()
    if args.form == "both" and not args.no_loader and args.scale == 1:
        line["loader"] = loader_form()

    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if dist_on:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
