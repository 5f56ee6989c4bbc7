"""Parity at the benchmark's full size (2048x1024 grid, 64 particles per cell = 134,217,728
particles, cubic WT, c dt = 0.25), in the launch configuration bench.py times: sampled
particles are checked one by one against the oracle, and properties that hold at any size
(Gauss's law, charge) are checked on the whole grid."""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402

NSAMPLE = 1500


@pytest.mark.parametrize("prec,tol", [(pic.PIC_FP64, 1e-12), (pic.PIC_FP32_MIXED, 2e-6)],
                         ids=["fp64", "fp32"])
def test_full_size_sampled_particles_and_gauss(prec, tol):
    wl = workloads.config_large(scheme=1, device="cuda")
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps)
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, s.u)
    del wl.species[0].x, wl.species[0].u  # free the device inputs early
    run.step(3)                      # non-trivial fields, no sort due yet (interval 9)
    d0 = run.diag()
    orc = oracle.Sim(wl.grid[:2], wl.dx[:2], wl.dt, wl.l, wl.scheme)
    for c in range(6):
        orc.set_field(c, run.field(c))
    rng = np.random.default_rng(2026)
    before = []
    for s in range(2):
        x, u, _ = run.particles(s)
        idx = rng.choice(x.shape[1], NSAMPLE, replace=False)
        before.append((idx, x[:, idx].copy(), u[:, idx].copy()))
        del x, u
    run.step(1)
    d1 = run.diag()
    qm = [(-1.0, 1.0), (1.0, 1.0)]
    L = np.array([wl.grid[0] * wl.dx[0], wl.grid[1] * wl.dx[1]])
    for s in range(2):
        idx, xb, ub = before[s]
        x, u, _ = run.particles(s)
        xg, ug = x[:, idx], u[:, idx]
        del x, u
        umax = np.max(np.abs(ug))
        for k in range(NSAMPLE):
            xo, uo = orc.push_particle(qm[s][0], qm[s][1], xb[:, k], ub[:, k])
            assert np.max(np.abs(ug[:, k] - uo)) <= tol * umax, (s, k)
            dxy = xg[:, k] - xo
            dxy -= L * np.round(dxy / L)
            assert np.max(np.abs(dxy)) <= tol * L.max(), (s, k)
    # at any size: charge is unchanged and D.E - rho is conserved by the charge-conserving
    # deposit (to round-off of the precision form)
    assert d1["total_charge"] == d0["total_charge"]
    rho_scale = abs(wl.species[0].q * wl.species[0].w) * 32
    gauss_tol = 1e-9 if prec == pic.PIC_FP64 else 1e-4
    assert abs(d1["max_gauss_residual"] - d0["max_gauss_residual"]) <= gauss_tol * rho_scale
    assert d1["error_flags"] == 0
    run.close()
