"""Served form (engine.Server): requests arrive over time, are admitted under a device-memory
budget, share one of two batches (2D, by size) or run on their own streams (3D) concurrently,
and each result must equal the same request run alone, within the FP32 multi-step tolerance
(the order of the floating-point atomics differs between the two, so results agree to
round-off growth, not bit for bit)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402
from paper_1909_09613_gb300 import engine  # noqa: E402

MULTI_STEP_TOL = 1e-4


def rel(a, b):
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a)))


def _requests():
    specs = [((64, 32, 1), 0.35, 2, 8, 10.0, 24, 0.00), ((96, 48, 1), 0.6, 3, 4, 40.0, 18, 0.00),
             ((48, 32, 1), 0.15, 3, 16, 20.0, 30, 0.05), ((24, 16, 16), 0.4, 2, 8, 5.0, 12, 0.05),
             ((128, 64, 1), 0.25, 2, 4, 70.0, 20, 0.10), ((40, 40, 1), 0.5, 3, 8, 15.0, 16, 0.15)]
    reqs = [engine.Request(rid=i, grid=g, dt=dt, l=l, gamma=gm, u_th=0.01, ppc=ppc, steps=st,
                           arrival=arr, seed=100 + i)
            for i, (g, dt, l, ppc, gm, st, arr) in enumerate(specs)]
    # requests the batch does not take (quartic; the plain FP64 form) step on their own streams;
    # one batched request uses the M4 solver; two record their field-energy history
    n = len(reqs)
    reqs.append(engine.Request(rid=n, grid=(64, 32, 1), dt=0.3, l=4, gamma=20.0, u_th=0.01, ppc=8,
                               steps=20, arrival=0.02, seed=200, record_every=5))
    reqs.append(engine.Request(rid=n + 1, grid=(48, 24, 1), dt=0.35, l=3, gamma=30.0, u_th=0.01,
                               ppc=8, steps=15, arrival=0.05, seed=201,
                               precision=pic.PIC_FP64, record_every=3))
    reqs.append(engine.Request(rid=n + 2, grid=(64, 32, 1), dt=0.4, l=2, gamma=25.0, u_th=0.01,
                               ppc=8, steps=18, arrival=0.0, seed=202, solver=pic.PIC_SOLVER_M4))
    # a batched request that records its history: its state is read between batched sorts
    reqs.append(engine.Request(rid=n + 3, grid=(80, 40, 1), dt=0.3, l=3, gamma=20.0, u_th=0.01,
                               ppc=16, steps=24, arrival=0.01, seed=203, record_every=4))
    return reqs


def test_served_results_equal_alone():
    reqs = _requests()
    # budget for roughly three resident runs: admission has to wait for memory
    sizes = sorted(engine.footprint_estimate(r) for r in reqs)
    budget = sum(sizes[-3:])
    # the size split puts batchable requests in both batch lanes (small and larger runs)
    srv = engine.Server(budget_bytes=budget, chunk=5, keep_runs=True, small_particles=20000)
    res = srv.serve(reqs)
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    assert srv.max_active >= 2          # work of several requests overlapped
    assert min(srv.lane_runs) >= 2      # both batches served runs
    assert srv.peak_bytes <= budget
    for r in res:
        assert r.latency >= 0.0 and r.diag["error_flags"] == 0
        q = reqs[r.rid]
        if q.record_every:
            assert [h[0] for h in r.history] == list(range(0, q.steps + 1, q.record_every))
            assert all(h[3] > 0.0 for h in r.history)
    by_id = {r.rid: r for r in res}
    for req in reqs:
        alone = engine.make_run(req)
        if req.record_every:
            # the history of the served run equals the same run's alone at the same steps
            hist = by_id[req.rid].history
            for k in range(len(hist)):
                if k:
                    alone.step(req.record_every)
                d = alone.diag()
                assert hist[k][0] == d["step"]
                assert abs(hist[k][2] - d["field_energy"]) <= 1e-3 * max(d["field_energy"], 1e-30), (req.rid, k)
                assert abs(hist[k][3] - d["kinetic_energy"]) <= 1e-5 * d["kinetic_energy"], (req.rid, k)
        else:
            alone.step(req.steps)
        mixed = srv.finished_runs[req.rid]
        for c in range(9):
            assert rel(mixed.field(c), alone.field(c)) < MULTI_STEP_TOL, (req.rid, c)
        da, dm = alone.diag(), mixed.diag()
        assert abs(dm["kinetic_energy"] - da["kinetic_energy"]) < 1e-5 * da["kinetic_energy"]
        assert dm["step"] == da["step"] == req.steps
        alone.close()
        mixed.close()


def test_autotuner_picks_a_valid_configuration():
    tuner = engine.Autotuner(probe_grid=(64, 32))
    tile, si = tuner.choose(2, 8, 0.35)
    assert tile in [(t[0], t[1], 1) for t in engine.Autotuner.TILES]
    assert si >= 1
    assert len(tuner.log) >= 2
