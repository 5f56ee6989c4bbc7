"""Batched form (pic_batch_*): many uneven 2D FP32 runs in one persistent particle kernel per
step, replayed from a CUDA graph.  Every run must evolve as it does alone (pic_step) and, for
one step, as the FP64 oracle does within the FP32 tolerance."""
import numpy as np
import pytest

import oracle
import plasma
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402

FP32_TOL = 2e-6

# (grid, cdt, l, ppc, gamma, seed): uneven sizes, both spline orders, narrow and wide T
RUNS = [((64, 32), 0.35, 2, 4, 10.0, 1), ((96, 48), 0.6, 3, 8, 30.0, 2), ((40, 24), 0.12, 2, 16, 80.0, 3),
        ((128, 64), 0.25, 3, 6, 15.0, 4), ((33, 21), 0.5, 3, 4, 50.0, 5)]


def rel(a, b):
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a)))


def make(spec, solver=pic.PIC_SOLVER_YEE):
    grid, cdt, l, ppc, gamma, seed = spec
    wl = plasma.pair_plasma(grid, (1.0, 1.0), cdt, l, 1, gamma, 0.01, ppc, seed=seed)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=pic.PIC_FP32_MIXED, capacity=caps,
                  solver=solver)
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, s.u)
    rng = np.random.default_rng(seed)
    f = [0.02 * rng.standard_normal((1, grid[1], grid[0])) for _ in range(6)]
    for c in range(6):
        run.set_field(c, f[c])
    return wl, run, f


def test_batch_matches_runs_alone():
    nsteps = 12  # crosses the sort interval of every run
    alone, batched = [], []
    for spec in RUNS:
        _, r, _ = make(spec)
        r.step(nsteps)
        alone.append(r)
    for spec in RUNS:
        _, r, _ = make(spec)
        batched.append(r)
    b = pic.Batch(batched)
    b.step(nsteps)
    b.sync()
    for ra, rb in zip(alone, batched):
        for c in range(9):
            assert rel(rb.field(c), ra.field(c)) < 1e-4, c
        da, db = ra.diag(), rb.diag()
        assert db["error_flags"] == 0
        assert abs(db["kinetic_energy"] - da["kinetic_energy"]) < 1e-5 * da["kinetic_energy"]
        for s in range(2):
            xa, ua, ca = ra.particles(s)
            xb, ub, cb = rb.particles(s)
            assert np.array_equal(np.sort(ca), np.sort(cb)) or rel(np.sort(xb, axis=1), np.sort(xa, axis=1)) < 1e-5
    b.close()
    for r in alone + batched:
        r.close()


def test_batch_mixed_solvers_match_runs_alone():
    """Runs with the M4 modified-Faraday stencil (App. C) and with Yee in one batch: the
    batched Yee launches take each run's stencil from its descriptor, so every run evolves as
    it does alone, and the M4 runs differ from the same runs under Yee."""
    specs = RUNS[:4]
    solvers = [pic.PIC_SOLVER_M4, pic.PIC_SOLVER_YEE, pic.PIC_SOLVER_M4, pic.PIC_SOLVER_YEE]
    alone = [make(sp, so)[1] for sp, so in zip(specs, solvers)]
    for r in alone:
        r.step(12)
    batched = [make(sp, so)[1] for sp, so in zip(specs, solvers)]
    b = pic.Batch(batched)
    b.step(12)
    b.sync()
    yee0 = make(specs[0])[1]
    yee0.step(12)
    for ra, rb in zip(alone, batched):
        for c in range(9):
            assert rel(rb.field(c), ra.field(c)) < 1e-4, c
        assert rb.diag()["error_flags"] == 0
    assert rel(batched[0].field(5), yee0.field(5)) > 1e-3   # the stencil really differs
    b.close()
    for r in alone + batched + [yee0]:
        r.close()


def test_batch_one_step_matches_oracle():
    runs, orcs = [], []
    for spec in RUNS[:3]:
        wl, r, f = make(spec)
        o = oracle.Sim(wl.grid[:2], wl.dx[:2], wl.dt, wl.l, wl.scheme)
        for i, s in enumerate(wl.species):
            x, u, _ = r.particles(i)
            o.add_species(s.q, s.m, s.w, x, u)
        for c in range(6):
            o.set_field(c, f[c])
        runs.append(r)
        orcs.append(o)
    b = pic.Batch(runs)
    b.step(1)
    b.sync()
    for r, o in zip(runs, orcs):
        o.step(1)
        for c in range(9):
            assert rel(r.field(c), o.field(c)) < FP32_TOL, c
        for s in range(2):
            _, ug, _ = r.particles(s)
            _, uo = o.particles(s)
            assert rel(ug, uo) < FP32_TOL
    b.close()
    for r in runs:
        r.close()


def test_batch_graph_replay_and_timing():
    runs = [make(spec)[1] for spec in RUNS]
    b = pic.Batch(runs)
    items, launches = b.info()
    # one work item per tile, the heavier tiles of this small set split into up to 8 items
    tiles = sum(r.ntiles for r in runs)
    assert tiles < items <= 8 * tiles
    b.step(3)
    ms = b.time_gpp()
    assert ms > 0.0
    b.sync()
    for r in runs:
        assert r.diag()["error_flags"] == 0
    b.close()


def test_batch_full_scale_sampled_particles():
    """The batched configuration at its benchmark size (256 uneven runs, 184,721,408 particles,
    one persistent kernel per step): after 3 batched steps, one more; sampled particles of 12
    runs (no sort due in that step) checked one by one against the oracle push from the run's
    fields, and on every run the charge is unchanged and D.E - rho conserved."""
    import workloads
    from paper_1909_09613_gb300 import engine
    specs = workloads.batched_runs(256)
    reqs = [engine.Request(rid=i, grid=sp["grid"], dt=sp["dt"], l=sp["l"], gamma=sp["gamma"],
                           u_th=sp["u_th"], ppc=sp["ppc"], steps=sp["steps"],
                           seed=workloads.BASE_SEED) for i, sp in enumerate(specs)]
    runs = [engine.make_run(r) for r in reqs]
    assert sum(r.counts[0] + r.counts[1] for r in runs) == 184721408
    b = pic.Batch(runs)
    b.step(3)
    b.sync()
    d0 = [r.diag() for r in runs]
    rng = np.random.default_rng(44)
    # runs whose 4th step does not sort (their particle order is unchanged by it)
    cand = [i for i, r in enumerate(runs) if r.sort_interval >= 5]
    pick = sorted(rng.choice(cand, 12, replace=False).tolist())
    snap = {}
    for i in pick:
        r, q = runs[i], reqs[i]
        orc = oracle.Sim(r.grid[:2], (1.0, 1.0), q.dt, q.l, q.scheme)
        for c in range(6):
            orc.set_field(c, r.field(c))
        parts = []
        for s in range(2):
            x, u, _ = r.particles(s)
            idx = rng.choice(x.shape[1], 40, replace=False)
            parts.append((idx, x[:, idx].copy(), u[:, idx].copy()))
        snap[i] = (orc, parts)
    b.step(1)
    b.sync()
    for i in pick:
        r = runs[i]
        orc, parts = snap[i]
        L = np.array([r.grid[0], r.grid[1]], dtype=float)
        for s, (q, m) in enumerate(((-1.0, 1.0), (1.0, 1.0))):
            idx, xb, ub = parts[s]
            x, u, _ = r.particles(s)
            xg, ug = x[:, idx], u[:, idx]
            umax = np.max(np.abs(ug))
            for k in range(len(idx)):
                xo, uo = orc.push_particle(q, m, xb[:, k], ub[:, k])
                assert np.max(np.abs(ug[:, k] - uo)) <= FP32_TOL * umax, (i, s, k)
                dxy = xg[:, k] - xo
                dxy -= L * np.round(dxy / L)
                assert np.max(np.abs(dxy)) <= FP32_TOL * L.max(), (i, s, k)
        orc.close()
    for r, q, a in zip(runs, reqs, d0):
        d = r.diag()
        assert d["error_flags"] == 0
        assert d["total_charge"] == a["total_charge"]
        # charge density of one species: w ppc/2 / V_c = omega_p^2 gamma (omega_p = 1/16)
        rho_scale = q.gamma / 256.0
        assert abs(d["max_gauss_residual"] - a["max_gauss_residual"]) <= 1e-4 * rho_scale
    b.close()
    for r in runs:
        r.close()


def test_batch_tiles_keep_two_ctas_per_sm():
    """A batch runs at the largest shared-memory stage of its runs.  For batchable requests whose
    tuned tile would exceed what two CTAs per SM leave, the engine picks a fallback tile that
    fits (pic_smem_info on the device), and the fitted tile is unchanged when it already fits."""
    from paper_1909_09613_gb300 import engine
    two = None
    for l, dt, ppc in ((3, 0.7, 32), (2, 0.6, 8), (3, 0.25, 16)):
        req = engine.Request(rid=0, grid=(512, 256, 1), l=l, dt=dt, gamma=20.0, u_th=0.01,
                             ppc=ppc, steps=1)
        for tile in ((64, 16, 1), (32, 32, 1), (64, 8, 1)):
            t, si = engine.fit_batch_tile(req, tile, 4)
            opt = pic.pic_options()
            opt.precision = pic.PIC_FP32_MIXED
            opt.n_species = 2
            opt.capacity[0] = opt.capacity[1] = 512 * 256 * ppc // 2
            opt.tile[0], opt.tile[1], opt.tile[2] = t
            opt.sort_interval = si
            ctx = pic.pic_create(req.grid, (1.0, 1.0, 1.0), dt, l, req.scheme, opt)
            try:
                own, batched, two = pic.pic_smem_info(ctx)
            finally:
                pic.pic_destroy(ctx)
            assert two > 100 * 1024          # a device is present
            assert batched <= two, (l, dt, tile, t, batched, two)
            if t == tile:
                assert si == 4


def test_batch_set_runs_keeps_the_graph_and_matches_alone():
    """Runs join and leave a batch between steps (pic_batch_set_runs): the batch keeps its
    captured graph (its launches walk device tables of any set within its capacities), and
    every run evolves exactly as it does alone, through sorts, over the steps it spent in the
    batch and out of it."""
    specs = RUNS[:4]
    alone = [make(sp)[1] for sp in specs]
    mixed = [make(sp)[1] for sp in specs]
    for r in alone:
        r.step(20)
    cap = pic.pic_batch_capacity()
    cap.runs = 8
    cap.cells = 4 * sum(r.ncell for r in mixed)
    cap.tiles = 4 * sum(r.ntiles for r in mixed)
    cap.stage_bytes = max(pic.pic_smem_info(r.ctx)[1] for r in mixed)
    b = pic.Batch(mixed[:2], capacity=cap)
    b.step(5)                              # runs 0, 1: 5 steps (graph captured)
    assert b.set_runs(mixed[1:4])          # run 0 leaves, 2 and 3 join
    mixed[0].step(15)                      # run 0 goes on alone
    b.step(7)                              # runs 1, 2, 3: 7 steps
    assert b.set_runs([mixed[3], mixed[0]])  # 1 and 2 leave, 0 comes back
    mixed[1].step(8)
    mixed[2].step(13)
    b.step(8)                              # runs 3, 0: 8 steps
    assert b.set_runs([])
    mixed[3].step(5)                       # run 3: 7 + 8 + 5 = 20 steps
    for r in mixed:
        r.sync()
    for i in (1, 2):
        assert mixed[i].diag()["step"] == 20
    for i in (1, 2):  # identical step sequences: equal to the alone runs at FP32 round-off growth
        for c in range(9):
            assert rel(mixed[i].field(c), alone[i].field(c)) < 1e-4, (i, c)
    assert mixed[0].diag()["step"] == 28 and mixed[3].diag()["step"] == 20
    alone[0].step(8)
    for i in (0, 3):
        for c in range(9):
            assert rel(mixed[i].field(c), alone[i].field(c)) < 1e-4, (i, c)
        assert mixed[i].diag()["error_flags"] == 0
    # a set beyond the capacities is refused and the batch keeps its runs; a run may not be
    # in a set twice
    big = [make(sp)[1] for sp in RUNS + RUNS]
    assert not b.set_runs(big)
    with pytest.raises(pic.PicError) as e:
        b.set_runs([big[0], big[0]])
    assert e.value.status == pic.PIC_EINVAL
    b.close()
    for r in alone + mixed + big:
        r.close()
