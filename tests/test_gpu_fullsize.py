"""Parity at the benchmark's full size (2048x1024 grid, 64 particles per cell = 134,217,728
particles, cubic WT, c dt = 0.25), in the launch configuration bench.py times.

The device loader generates the plasma in HBM; smooth fields made on the host are set.  The
oracle draws the particles of sampled cells itself (oracle.load_drifting at the same stream
counters, plus the neighbouring cells an FP32 carry can move a particle in from), so nothing it
is given comes from the GPU: every sampled cell's segment of the GPU's stable tile order must
hold exactly those particles in input order, and after one step each must equal the oracle's
push of it.  Whole-grid properties -- charge, the discrete continuity residual and the drift of
D.E - rho -- are checked by pic_diag at this size."""
import math

import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import host_packed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402

NCELLS = 48


def smooth_fields_2d(nx, ny, amp, seed):
    rng = np.random.default_rng(seed)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for _ in range(6):
        f = np.zeros((1, ny, nx))
        for _ in range(4):
            mx, my = rng.integers(0, 6, 2)
            f[0] += rng.uniform(-1, 1) * np.cos(2 * math.pi * (mx * ii / nx + my * jj / ny)
                                                + rng.uniform(0, 2 * math.pi))
        out.append(amp * f)
    return out


def oracle_cell(wl, s, prec, c):
    """(input indices, x, u, packed cells) of species s's particles whose packed cell is c, in
    input order, drawn by the oracle: the particles of c and of the three cells from which an
    FP32 carry along x, y or both can bring one in."""
    nx, ny = wl.grid[0], wl.grid[1]
    i, j = c % nx, c // nx
    per = wl.species[s].per_cell
    src = sorted({((i - di) % nx) + ((j - dj) % ny) * nx for di in (0, 1) for dj in (0, 1)})
    idx, xs, us, cs = [], [], [], []
    for cc in src:
        x, u, f = oracle.load_drifting(wl.grid, wl.dx, per, wl.gamma, wl.u_th, wl.theta, wl.seed,
                                       wl.run, s, wl.species[s].pos_species, first=cc * per,
                                       count=per)
        assert f == 0
        cells, xp, up = host_packed(x, u, wl.grid, wl.dx, 2, prec)
        keep = cells == c
        idx.append(cc * per + np.nonzero(keep)[0])
        xs.append(xp[:, keep])
        us.append(up[:, keep])
        cs.append(cells[keep])
    idx = np.concatenate(idx)
    o = np.argsort(idx)
    return idx[o], np.concatenate(xs, axis=1)[:, o], np.concatenate(us, axis=1)[:, o]


@pytest.mark.parametrize("prec,tol", [(pic.PIC_FP64, 1e-12), (pic.PIC_FP32_MIXED, 2e-6)],
                         ids=["fp64", "fp32"])
def test_full_size_sampled_cells_and_conservation(prec, tol):
    wl = workloads.config_large(scheme=1)
    nx, ny = wl.grid[0], wl.grid[1]
    caps = [wl.ncell * s.per_cell for s in wl.species]
    assert sum(caps) == 134217728
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps)
    for i, s in enumerate(wl.species):
        run.load_drifting_plasma(i, s.q, s.m, s.w, s.per_cell, wl.gamma, wl.u_th, seed=wl.seed,
                                 run=wl.run, pos_species=s.pos_species)
    fields = smooth_fields_2d(nx, ny, 0.02, seed=2026)
    orc = oracle.Sim(wl.grid[:2], wl.dx[:2], wl.dt, wl.l, wl.scheme)
    for c, f in enumerate(fields):
        run.set_field(c, f)
        orc.set_field(c, f)
    d0 = run.diag()
    rng = np.random.default_rng(2026)
    cells = np.sort(rng.choice(wl.ncell, NCELLS, replace=False))
    want, where = [], []
    for s in range(2):
        _, _, cg = run.particles(s)
        mask = np.isin(cg, cells)
        pos = np.nonzero(mask)[0]
        cgs = cg[pos]
        del cg
        w_s, p_s = [], []
        for c in cells:
            idx, x, u = oracle_cell(wl, s, prec, int(c))
            p = pos[cgs == c]              # the cell's positions in the stable order
            assert len(p) == len(idx), (s, c)
            w_s.append((idx, x, u))
            p_s.append(p)
        want.append(w_s)
        where.append(p_s)
    # the loaded state of every sampled cell, position by position
    for s in range(2):
        xg, ug, _ = run.particles(s)
        for (idx, x, u), p in zip(want[s], where[s]):
            assert np.array_equal(xg[:, p], x)
            utol = 4e-16 if prec == pic.PIC_FP64 else 1.2e-7
            assert np.max(np.abs(ug[:, p] - u)) <= utol * max(1.0, np.max(np.abs(u)))
        del xg, ug
    run.step(1)                                # no sort is due (interval 9)
    d1 = run.diag()
    L = np.array([nx * wl.dx[0], ny * wl.dx[1]])
    for s in range(2):
        q, m = wl.species[s].q, wl.species[s].m
        xg, ug, _ = run.particles(s)
        for (idx, x, u), p in zip(want[s], where[s]):
            xa, ua = xg[:, p], ug[:, p]
            umax = max(np.max(np.abs(ua)), 1.0)
            for k in range(len(idx)):
                xo, uo = orc.push_particle(q, m, x[:, k], u[:, k])
                assert np.max(np.abs(ua[:, k] - uo)) <= tol * umax, (s, k)
                d = xa[:, k] - xo
                d -= L * np.round(d / L)
                assert np.max(np.abs(d)) <= tol * L.max(), (s, k)
        del xg, ug
    # whole grid: charge unchanged; the Esirkepov deposit keeps the discrete continuity
    # equation (to the round-off of the form) and so D.E - rho
    assert d1["total_charge"] == d0["total_charge"]
    rho_scale = abs(wl.species[0].q * wl.species[0].w) * 32
    ctol = 1e-12 if prec == pic.PIC_FP64 else 2e-5
    assert d1["max_continuity_residual"] <= ctol * rho_scale / wl.dt
    gtol = 1e-11 if prec == pic.PIC_FP64 else 1e-4
    assert d1["max_gauss_residual_drift"] <= gtol * rho_scale
    assert d1["error_flags"] == 0
    run.close()


def smooth_fields_3d(nx, ny, nz, amp, seed):
    rng = np.random.default_rng(seed)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for _ in range(6):
        f = np.zeros((nz, ny, nx))
        for _ in range(3):
            mx, my, mz = rng.integers(0, 5, 3)
            f += rng.uniform(-1, 1) * np.cos(2 * math.pi * (mx * ii / nx + my * jj / ny
                                                            + mz * kk / nz)
                                             + rng.uniform(0, 2 * math.pi))
        out.append(amp * f)
    return out


def oracle_cell_3d(wl, s, c):
    """(input indices, x, u) of species s's particles whose packed FP32 cell is c, in input
    order, drawn by the oracle: the particles of c and of the seven cells from which an FP32
    carry along any set of axes can bring one in."""
    nx, ny, nz = wl.grid
    i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
    per = wl.species[s].per_cell
    src = sorted({((i - di) % nx) + ((j - dj) % ny) * nx + ((k - dk) % nz) * nx * ny
                  for di in (0, 1) for dj in (0, 1) for dk in (0, 1)})
    idx, xs, us = [], [], []
    for cc in src:
        x, u, f = oracle.load_drifting(wl.grid, wl.dx, per, wl.gamma, wl.u_th, wl.theta, wl.seed,
                                       wl.run, s, wl.species[s].pos_species, first=cc * per,
                                       count=per)
        assert f == 0
        cells, xp, up = host_packed(x, u, wl.grid, wl.dx, 3, pic.PIC_FP32_MIXED)
        keep = cells == c
        idx.append(cc * per + np.nonzero(keep)[0])
        xs.append(xp[:, keep])
        us.append(up[:, keep])
    idx = np.concatenate(idx)
    o = np.argsort(idx)
    return idx[o], np.concatenate(xs, axis=1)[:, o], np.concatenate(us, axis=1)[:, o]


def test_full_size_3d_sampled_cells_and_conservation():
    """The largest 3D request of the served workload (512x128x128, 8 per cell = 67,108,864
    particles, quadratic WT, c dt = 0.4, drift along x1) in the FP32 form: its tile stage in
    shared memory and its FP32 current.  Sampled cells hold exactly the oracle's particles in
    input order; after one step each equals the oracle's push of it; the continuity residual
    and the Gauss drift bound the whole grid."""
    wl = workloads.pair_plasma((512, 128, 128), (1.0, 1.0, 1.0), 0.4, 2, 1, 20.0, 0.01, 8)
    nx, ny, nz = wl.grid
    caps = [wl.ncell * s.per_cell for s in wl.species]
    assert sum(caps) == 67108864
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=pic.PIC_FP32_MIXED,
                  capacity=caps)
    for i, s in enumerate(wl.species):
        run.load_drifting_plasma(i, s.q, s.m, s.w, s.per_cell, wl.gamma, wl.u_th, seed=wl.seed,
                                 run=wl.run, pos_species=s.pos_species)
    fields = smooth_fields_3d(nx, ny, nz, 0.02, seed=2027)
    orc = oracle.Sim(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme)
    for c, f in enumerate(fields):
        run.set_field(c, f)
        orc.set_field(c, f)
    d0 = run.diag()
    rng = np.random.default_rng(2027)
    cells = np.sort(rng.choice(wl.ncell, NCELLS, replace=False))
    want, where = [], []
    for s in range(2):
        xg, ug, cg = run.particles(s)
        mask = np.isin(cg, cells)
        pos = np.nonzero(mask)[0]
        cgs = cg[pos]
        w_s, p_s = [], []
        for c in cells:
            idx, x, u = oracle_cell_3d(wl, s, int(c))
            p = pos[cgs == c]              # the cell's positions in the stable order
            assert len(p) == len(idx), (s, c)
            assert np.array_equal(xg[:, p], x)
            assert np.max(np.abs(ug[:, p] - u)) <= 1.2e-7 * max(1.0, np.max(np.abs(u)))
            w_s.append((idx, x, u))
            p_s.append(p)
        want.append(w_s)
        where.append(p_s)
        del xg, ug, cg
    run.step(1)                                # no sort is due yet
    d1 = run.diag()
    L = np.array([nx * wl.dx[0], ny * wl.dx[1], nz * wl.dx[2]])
    for s in range(2):
        q, m = wl.species[s].q, wl.species[s].m
        xg, ug, _ = run.particles(s)
        for (idx, x, u), p in zip(want[s], where[s]):
            xa, ua = xg[:, p], ug[:, p]
            umax = max(np.max(np.abs(ua)), 1.0)
            for k in range(len(idx)):
                xo, uo = orc.push_particle(q, m, x[:, k], u[:, k])
                assert np.max(np.abs(ua[:, k] - uo)) <= 2e-6 * umax, (s, k)
                d = xa[:, k] - xo
                d -= L * np.round(d / L)
                assert np.max(np.abs(d)) <= 2e-6 * L.max(), (s, k)
        del xg, ug
    assert d1["total_charge"] == d0["total_charge"]
    rho_scale = abs(wl.species[0].q * wl.species[0].w) * 4
    assert d1["max_continuity_residual"] <= 2e-5 * rho_scale / wl.dt
    assert d1["max_gauss_residual_drift"] <= 1e-4 * rho_scale
    assert d1["error_flags"] == 0
    run.close()
