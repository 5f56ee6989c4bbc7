"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle, element by element.

Tolerances (relative, per array: max |a - b| / max |b|):
  FP64 form: 1e-12 after one step from the same state;
  FP32 form: 2e-6 after one step from the same state (the FP32 round-off of a gather of
  O(10-25) products plus one Boris rotation stays well inside it);
Integer results (cell indices, the tile order) are compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle
import plasma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402

FP64_TOL = 1e-12
FP32_TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_09613_gb300 import _build
    _build.build()
    oracle.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    if den == 0.0:
        return float(np.max(np.abs(a)))
    return float(np.max(np.abs(a - b)) / den)


def smooth_fields(shape, amp, seed):
    """Seeded smooth random fields: a few low Fourier modes per component."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = []
    for _ in range(6):
        f = np.zeros(shape)
        for _ in range(4):
            mx, my, mz = rng.integers(0, 4, 3)
            ph = rng.uniform(0, 2 * math.pi)
            f += rng.uniform(-1, 1) * np.cos(2 * math.pi * (mx * ii / nx + my * jj / ny
                                                           + (mz * kk / nz if nz > 1 else 0)) + ph)
        out.append(amp * f)
    return out


def host_packed(x, u, grid, dx, dim, prec):
    """The particle state a load stores, computed on the host from the input arrays: the cell
    of every particle and, for the FP32 form, the positions and momenta rounded as stored (an
    in-cell offset that rounds to 1.0 in FP32 carries into the next cell, decided in FP32 as
    the packing kernel does).  Returns (cells, x, u) in physical FP64 units."""
    x = np.array(x, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    cells = np.zeros(x.shape[1], dtype=np.int64)
    stride = 1
    for a in range(dim):
        xi = x[a] / dx[a]
        n = float(grid[a])
        xi = np.where(xi >= n, xi - n, xi)
        xi = np.where(xi < 0.0, xi + n, xi)
        c = np.floor(xi)
        if prec == pic.PIC_FP32_MIXED:
            off = (xi - c).astype(np.float32)
            carry = off >= np.float32(1.0)
            off = np.where(carry, np.float32(0.0), off)
            c = c + carry
            c = np.where(c >= n, c - n, c)
            x[a] = (c + off.astype(np.float64)) * dx[a]
        cells += c.astype(np.int64) * stride
        stride *= grid[a]
    if prec == pic.PIC_FP32_MIXED:
        u = u.astype(np.float32).astype(np.float64)
    return cells, x, u


def make_pair(wl, prec, fields=None, tile=None, sort_interval=0, solver=0, deterministic=False):
    """Same initial state on the GPU (libpic) and in the oracle, both from the input arrays:
    the GPU loads them (packing and tile-sorting), the oracle takes them in input order as the
    load stores them (the FP32 rounding done on the host).  run.orc_perm[s] is the oracle's
    stable tile order of species s (oracle.tile_sort of the packed cells): the GPU particle at
    sorted position k is the oracle's particle orc_perm[s][k]."""
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps,
                  tile=tile, sort_interval=sort_interval, solver=solver,
                  deterministic=deterministic)
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, s.u)
    dim = wl.dim
    orc = oracle.Sim(wl.grid[:dim], wl.dx[:dim], wl.dt, wl.l, wl.scheme, solver=solver)
    run.orc_perm = []
    for i, s in enumerate(wl.species):
        cells, x, u = host_packed(s.x, s.u, wl.grid, wl.dx, dim, prec)
        orc.add_species(s.q, s.m, s.w, x, u)
        perm, _ = oracle.tile_sort(wl.grid, run.tile, cells,
                                   oracle.SLOT_MAJOR if run.slot_major else oracle.CELL_MAJOR)
        run.orc_perm.append(perm)
    if fields is not None:
        for c, f in enumerate(fields):
            run.set_field(c, f)
            orc.set_field(c, f)
    return run, orc


def compare_state(run, orc, nsp, tol, what=""):
    """Fields element by element; particles position by position, the GPU's sorted position k
    against the oracle's particle run.orc_perm[s][k] (one step after make_pair: no re-sort)."""
    errs = {}
    for c in range(9):
        errs["F%d" % c] = rel(run.field(c), orc.field(c))
    for s in range(nsp):
        xg, ug, _ = run.particles(s)
        xo, uo = orc.particles(s)
        perm = run.orc_perm[s]
        xo, uo = xo[:, perm], uo[:, perm]
        errs["u%d" % s] = rel(ug, uo)
        L = np.array([orc.grid[a] * orc.dx[a] for a in range(orc.dim)]).reshape(-1, 1)
        d = xg - xo
        d = d - L * np.round(d / L)
        errs["x%d" % s] = float(np.max(np.abs(d)) / np.max(L)) if d.size else 0.0
    bad = {k: v for k, v in errs.items() if v > tol}
    assert not bad, (what, bad, errs)
    return errs


CASES_2D = [
    # (grid, dx, cdt, l, scheme, gamma, u_th, ppc)
    ((64, 32), (1.0, 1.0), 0.35, 2, 1, 20.0, 0.0, 4),
    ((64, 32), (1.0, 1.0), 0.35, 2, 0, 20.0, 0.0, 4),
    ((40, 24), (1.0, 1.0), 0.25, 3, 1, 5.0, 0.05, 6),
    ((40, 24), (1.0, 1.0), 0.25, 3, 0, 5.0, 0.05, 6),
    ((37, 21), (0.9, 1.1), 0.3, 1, 1, 3.0, 0.1, 4),
    ((48, 20), (1.0, 1.0), 0.6, 3, 1, 10.0, 0.05, 4),
    ((48, 20), (1.0, 1.0), 0.3, 4, 1, 10.0, 0.05, 4),
    ((33, 18), (1.0, 1.0), 0.5, 2, 1, 2.0, 0.2, 4),
]


@pytest.mark.parametrize("case", CASES_2D, ids=lambda c: "g%dx%d_l%d_s%d_dt%.2f" % (c[0] + (c[3], c[4], c[2])))
@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
def test_one_step_2d(case, prec):
    grid, dx, cdt, l, scheme, gamma, uth, ppc = case
    wl = plasma.pair_plasma(grid, dx, cdt, l, scheme, gamma, uth, ppc, omega_p=0.2, seed=11)
    f = smooth_fields((1, grid[1], grid[0]), 0.05, seed=5)
    run, orc = make_pair(wl, prec, f)
    run.step(1)
    orc.step(1)
    compare_state(run, orc, 2, FP64_TOL if prec == pic.PIC_FP64 else FP32_TOL, case)
    run.close()


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", [((12, 10, 8), 0.3, 2, 1), ((12, 10, 8), 0.3, 2, 0),
                                  ((10, 9, 7), 0.25, 3, 1), ((9, 8, 8), 0.5, 1, 1),
                                  # grids narrower than a deposit window: the padded FP32
                                  # current folds several periodic images onto one node
                                  ((4, 3, 5), 0.3, 2, 1), ((5, 4, 3), 0.25, 3, 1)],
                         ids=lambda c: "g%dx%dx%d_l%d_s%d" % (c[0] + (c[2], c[3])))
def test_one_step_3d(case, prec):
    grid, cdt, l, scheme = case
    wl = plasma.pair_plasma(grid, (1.0, 1.0, 1.0), cdt, l, scheme, 4.0, 0.1, 4, omega_p=0.2,
                               seed=3)
    f = smooth_fields((grid[2], grid[1], grid[0]), 0.05, seed=9)
    run, orc = make_pair(wl, prec, f)
    run.step(1)
    orc.step(1)
    compare_state(run, orc, 2, FP64_TOL if prec == pic.PIC_FP64 else FP32_TOL, case)
    run.close()


def random_position_plasma(grid, l, per, gamma, u_th, seed, cdt=0.25):
    """Pair plasma with positions uniform over the whole grid (Poisson cell counts, so the
    warps of the cell-major order straddle cells and tile rows), momenta from the oracle's
    App. D loader, plasma frequency of 16 cells per skin depth."""
    wl = plasma.pair_plasma(grid, (1.0, 1.0), cdt, l, 1, gamma, u_th, 2 * per, seed=seed)
    rng = np.random.default_rng(seed)
    for s in wl.species:
        n = s.x.shape[1]
        s.x = rng.uniform(0, 1, (2, n)) * np.array(grid, dtype=float)[:, None]
    return wl


TIMED_CASES = {
    # the large configuration on a 256x128 section: 32 per species in every cell, so every warp
    # of the cell-major order holds the 32 particles of one cell
    "config2_section_l3_ppc64": lambda: plasma.config_large(scale=8),
    # Poisson cell counts on a ragged grid (200 = 3 x 64 + 8): warps straddle cells and rows
    "l3_16_per_species_ragged": lambda: random_position_plasma((200, 72), 3, 16, 50.0, 0.01, 7),
    "l3_8_per_species": lambda: random_position_plasma((128, 64), 3, 8, 50.0, 0.01, 8),
    "l4_12_per_species": lambda: random_position_plasma((150, 40), 4, 12, 50.0, 0.01, 9),
}


@pytest.mark.parametrize("name", list(TIMED_CASES))
def test_one_step_timed_configuration_fp32(name):
    """The precision form in the configuration the benchmark times (FP32, cubic or quartic WT,
    c dt = 0.25, gamma 50, u_th = 0.01, cell-major warp-summed deposit, default 64x8 tiles):
    one step from the same state, J1..J3, E, B and every particle against the oracle at 2e-6."""
    wl = TIMED_CASES[name]()
    shape = (1, wl.grid[1], wl.grid[0])
    f = smooth_fields(shape, 0.02, seed=12)
    run, orc = make_pair(wl, pic.PIC_FP32_MIXED, f)
    assert run.slot_major == 0 and tuple(run.tile) == (64, 8, 1)
    run.step(1)
    orc.step(1)
    compare_state(run, orc, 2, FP32_TOL, name)
    assert run.diag()["error_flags"] == 0
    run.close()


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", [((40, 24), (1.0, 1.0), 0.3), ((37, 21), (0.9, 1.1), 0.25),
                                  ((12, 10, 8), (1.0, 1.0, 1.0), 0.3)],
                         ids=["2d", "2d_aniso", "3d"])
def test_one_step_m4_solver(case, prec):
    """The M4 Faraday stencil (App. C) on the GPU against the oracle, one step from the same
    state, and a few more steps (fields only) in FP64."""
    grid, dx, cdt = case
    wl = plasma.pair_plasma(grid, dx, cdt, 3, 1, 4.0, 0.05, 4, omega_p=0.2, seed=13)
    shape = (grid[2] if len(grid) == 3 else 1, grid[1], grid[0])
    f = smooth_fields(shape, 0.05, seed=8)
    run, orc = make_pair(wl, prec, f, solver=pic.PIC_SOLVER_M4)
    run.step(1)
    orc.step(1)
    compare_state(run, orc, 2, FP64_TOL if prec == pic.PIC_FP64 else FP32_TOL, case)
    if prec == pic.PIC_FP64:
        run.step(4)
        orc.step(4)
        for c in range(6):
            assert rel(run.field(c), orc.field(c)) < 1e-11, c
    run.close()


def test_multi_step_across_sorts_fp64():
    """20 steps at c dt = 0.35 (sort every 6 steps): fields and diagnostics stay at round-off
    from the oracle."""
    wl = plasma.config_small(scheme=1)
    wl2 = plasma.pair_plasma(wl.grid, wl.dx, wl.dt, wl.l, 1, 20.0, 0.01, 4,
                                omega_p=wl.omega_p)
    run, orc = make_pair(wl2, pic.PIC_FP64)
    assert run.sort_interval < 20
    run.step(20)
    orc.step(20)
    for c in range(9):
        assert rel(run.field(c), orc.field(c)) < 1e-10, c
    dg, do = run.diag(), orc.diag()
    assert abs(dg["field_energy"] - do["field_energy"]) <= 1e-9 * do["field_energy"]
    assert abs(dg["kinetic_energy"] - do["kinetic_energy"]) <= 1e-12 * do["kinetic_energy"]
    # particles: compare as sets (the GPU re-sorted them), matched by sorted positions
    for s in range(2):
        xg, ug, _ = run.particles(s)
        xo, uo = orc.particles(s)
        kg = np.lexsort(xg[::-1])
        ko = np.lexsort(xo[::-1])
        assert np.max(np.abs(xg[:, kg] - xo[:, ko])) < 1e-9
        assert rel(ug[:, kg], uo[:, ko]) < 1e-10
    run.close()


@pytest.mark.parametrize("l", [2, 3, 4])
def test_weight_cache_follows_sorts_and_reloads_fp64(l):
    """The FP64 form keeps each particle's B-spline weights at its stored position for the next
    step's Esirkepov deposit (l <= 3).  Every re-ordering must invalidate them: 16 steps with the
    automatic sort every 4 steps, an explicit sort after step 5 and a reload of one species
    (re-packed and re-sorted) after step 9, against the oracle."""
    wl = plasma.pair_plasma((40, 24), (1.0, 1.0), 0.3, l, pic.PIC_SCHEME_WT, 5.0, 0.05, 6)
    run, orc = make_pair(wl, pic.PIC_FP64, sort_interval=4)
    run.step(5)
    orc.step(5)
    run.sort()
    run.step(4)
    orc.step(4)
    s1 = wl.species[1]
    x, u, _ = run.particles(1)
    run.load(1, s1.q, s1.m, s1.w, x, u)
    run.step(7)
    orc.step(7)
    for c in range(9):
        assert rel(run.field(c), orc.field(c)) < 1e-10, c
    for s in range(2):
        xg, ug, _ = run.particles(s)
        xo, uo = orc.particles(s)
        kg = np.lexsort(xg[::-1])
        ko = np.lexsort(xo[::-1])
        assert np.max(np.abs(xg[:, kg] - xo[:, ko])) < 1e-9
        assert rel(ug[:, kg], uo[:, ko]) < 1e-10
    assert run.diag()["error_flags"] == 0
    run.close()


TAG_SCALE = 2.0 ** -12  # (i + 1) * TAG_SCALE is exact in FP32 for i + 1 < 2^24


def tagged_momenta(u):
    """u with u_z replaced by a tag that identifies particle i exactly in both forms."""
    u = np.array(u, dtype=np.float64)
    u[2] = (np.arange(u.shape[1]) + 1) * TAG_SCALE
    return u


def read_tags(uz):
    t = np.rint(np.asarray(uz) / TAG_SCALE).astype(np.int64) - 1
    assert np.array_equal((t + 1) * TAG_SCALE, uz)
    return t


def packed_cells(x, grid, dx, dim, prec):
    """Linear cell of every particle as the load computes it (FP32 form: an offset that rounds
    to 1.0 in FP32 carries into the next cell, decided in FP32 as the packing kernel does)."""
    cells = np.zeros(x.shape[1], dtype=np.int64)
    stride = 1
    for a in range(dim):
        xi = x[a] / dx[a]
        c = np.floor(xi)
        if prec == pic.PIC_FP32_MIXED:
            off = (xi - c).astype(np.float32)
            c = c.astype(np.int64) + (off >= np.float32(1.0))
            c = np.where(c >= grid[a], c - grid[a], c)
        cells += c.astype(np.int64) * stride
        stride *= grid[a]
    return cells


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("ppc", [6, 16], ids=["ppc6", "ppc16"])
@pytest.mark.parametrize("grid,tile", [((64, 32, 1), None), ((37, 21, 1), (8, 4, 1)),
                                       ((12, 10, 8), None), ((5, 3, 1), None)])
def test_tile_sort_bit_exact(prec, ppc, grid, tile):
    """The sort is stable and reproducible: the permutation a load applies equals the oracle's
    (tile, cell, input index) order -- or (tile, rank in cell, cell) for the slot-major order --
    bit for bit, and so do the cell at every position and the tile offsets."""
    g = tuple(grid)
    dim = 3 if g[2] > 1 else 2
    wl = plasma.pair_plasma(g if dim == 3 else g[:2], (1.0,) * dim, 0.3, 2, 1, 3.0, 0.1, ppc,
                               omega_p=0.2, seed=21)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps, tile=tile)
    if prec == pic.PIC_FP32_MIXED:
        assert run.slot_major == (0 if ppc // 2 >= 6 else 1)
    us = [tagged_momenta(s.u) for s in wl.species]
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, us[i])
    for i, s in enumerate(wl.species):
        x0 = s.x
        cells_in = packed_cells(x0, wl.grid, wl.dx, wl.dim, prec)
        perm, ts = oracle.tile_sort(wl.grid, run.tile, cells_in,
                                    oracle.SLOT_MAJOR if run.slot_major else oracle.CELL_MAJOR)
        xg, ug, cg = run.particles(i)
        assert np.array_equal(read_tags(ug[2]), perm)
        assert np.array_equal(cg, cells_in[perm])
        assert np.array_equal(run.tile_offsets(i), ts)
        if prec == pic.PIC_FP64:  # the packed FP64 position is x / dx exactly
            assert np.array_equal(xg, x0[:, perm])
            assert np.array_equal(ug[:2], us[i][:2, perm])
    run.close()


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("ppc", [4, 20], ids=["ppc4", "ppc20"])
def test_tile_sort_stable_after_steps(prec, ppc):
    """A re-sort after particles moved keeps the previous order inside every cell: neutral
    particles (q = 0: no force, no current) drift for three steps, then pic_sort must apply the
    oracle's stable order of the cells they reached, permutation included, on a ragged grid."""
    grid, dt = (45, 27), 0.3
    wl = plasma.pair_plasma(grid, (1.0, 1.0), dt, 3, 1, 3.0, 0.3, ppc, omega_p=0.2, seed=4)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps,
                  tile=(16, 8, 1), sort_interval=4)
    for i, s in enumerate(wl.species):
        run.load(i, 0.0, 1.0, s.w, s.x, tagged_momenta(s.u))
    run.step(3)
    before = [run.particles(i) for i in range(2)]
    run.sort()
    for i in range(2):
        xb, ub, cb = before[i]
        perm, ts = oracle.tile_sort(wl.grid, run.tile, cb,
                                    oracle.SLOT_MAJOR if run.slot_major else oracle.CELL_MAJOR)
        xa, ua, ca = run.particles(i)
        assert np.array_equal(read_tags(ua[2]), read_tags(ub[2])[perm])
        assert np.array_equal(ca, cb[perm])
        assert np.array_equal(xa, xb[:, perm])
        assert np.array_equal(run.tile_offsets(i), ts)
    assert run.diag()["error_flags"] == 0
    run.close()


def test_tile_sort_one_crowded_cell():
    """Degenerate occupancy: every particle of a species in one cell (the rank stage scans the
    whole cell), the other species spread; the order is still the oracle's, bit for bit."""
    grid = (24, 16)
    n = 3000
    rng = np.random.default_rng(8)
    x0 = np.vstack([5.0 + rng.uniform(0, 1, n), 7.0 + rng.uniform(0, 1, n)])
    x1 = rng.uniform(0, 1, (2, n)) * np.array(grid, dtype=float)[:, None]
    u = tagged_momenta(rng.normal(0, 0.1, (3, n)))
    for prec in (pic.PIC_FP64, pic.PIC_FP32_MIXED):
        run = pic.Run(grid, (1.0, 1.0), 0.3, 2, 1, precision=prec, capacity=(n, n))
        run.load(0, -1.0, 1.0, 0.1, x0, u)
        run.load(1, 1.0, 1.0, 0.1, x1, u)
        for i, x in enumerate((x0, x1)):
            cells = packed_cells(x, (24, 16), (1.0, 1.0), 2, prec)
            perm, ts = oracle.tile_sort((24, 16), run.tile, cells,
                                        oracle.SLOT_MAJOR if run.slot_major else oracle.CELL_MAJOR)
            _, ug, cg = run.particles(i)
            assert np.array_equal(read_tags(ug[2]), perm)
            assert np.array_equal(run.tile_offsets(i), ts)
        run.close()


def test_gauss_law_conserved_gpu_fp64():
    wl = plasma.pair_plasma((48, 24), (1.0, 1.0), 0.3, 3, 1, 5.0, 0.05, 8, omega_p=0.3)
    run, orc = make_pair(wl, pic.PIC_FP64)
    d0 = run.diag()
    run.step(60)
    d1 = run.diag()
    rho_scale = abs(wl.species[0].q * wl.species[0].w) * 8
    # D.E - rho is conserved; its max over nodes starts at the noise level and stays there
    assert abs(d1["max_gauss_residual"] - d0["max_gauss_residual"]) < 1e-11 * rho_scale
    assert d1["error_flags"] == 0
    run.close()


def test_empty_and_single_particle():
    grid = (16, 8)
    run = pic.Run(grid, (1.0, 1.0), 0.3, 2, 1, capacity=(0, 1))
    run.load(0, -1.0, 1.0, 1.0, np.zeros((2, 0)), np.zeros((3, 0)))
    x = np.array([[5.3], [2.7]])
    u = np.array([[0.5], [0.2], [-0.1]])
    run.load(1, 1.0, 1.0, 0.7, x, u)
    orc = oracle.Sim(grid, (1.0, 1.0), 0.3, 2, 1)
    orc.add_species(-1.0, 1.0, 1.0, np.zeros((2, 0)), np.zeros((3, 0)))
    orc.add_species(1.0, 1.0, 0.7, x, u)
    for _ in range(12):
        run.step(1)
        orc.step(1)
    for c in range(9):
        assert rel(run.field(c), orc.field(c)) < 1e-11, c
    xg, ug, _ = run.particles(1)
    xo, uo = orc.particles(1)
    assert np.max(np.abs(xg - xo)) < 1e-12 and rel(ug, uo) < 1e-11
    run.close()


@pytest.mark.parametrize("l", [1, 2, 3, 4])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("grid", [(8, 8), (6, 6, 6)])
def test_tiny_runs_ten_steps(grid, scheme, l):
    """Brute-force-sized whole runs: 1-4 particles per species on an 8x8 (or 6x6x6) periodic grid
    whose staged region wraps onto itself, 10 full steps of the FP64 form against the oracle."""
    rng = np.random.default_rng(1000 + 10 * l + scheme + len(grid))
    dim = len(grid)
    dt = 0.35 if dim == 2 else 0.3
    run = pic.Run(grid, (1.0,) * dim, dt, l, scheme, capacity=(4, 3))
    orc = oracle.Sim(grid, (1.0,) * dim, dt, l, scheme)
    for sp, (q, n) in enumerate(((-1.0, 4), (1.0, 3))):
        x = rng.uniform(0, 1, (dim, n)) * np.array(grid, dtype=float)[:, None]
        u = rng.normal(0, 1.5, (3, n))
        run.load(sp, q, 1.0, 0.5, x, u)
        orc.add_species(q, 1.0, 0.5, x, u)
    for _ in range(10):
        run.step(1)
        orc.step(1)
    for c in range(9):
        assert rel(run.field(c), orc.field(c)) < 1e-11, c
    for sp in range(2):
        xg, ug, _ = run.particles(sp)
        xo, uo = orc.particles(sp)
        # both are in the store order of their own sort: compare as sets
        kg, ko = np.lexsort(xg[::-1]), np.lexsort(xo[::-1])
        assert np.max(np.abs(xg[:, kg] - xo[:, ko])) < 1e-12
        assert rel(ug[:, kg], uo[:, ko]) < 1e-11
    assert run.diag()["error_flags"] == 0
    run.close()


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
def test_nonfinite_particle_is_reported(prec):
    """A particle whose momentum is not finite (made on the host) spreads NaN through its
    current into the fields; the kernels keep every index in range, pic_diag reports it in
    error_flags and the next syncing call returns PIC_ENAN."""
    grid = (16, 8)
    run = pic.Run(grid, (1.0, 1.0), 0.3, 2, 1, precision=prec, capacity=(8, 1))
    rng = np.random.default_rng(5)
    run.load(0, -1.0, 1.0, 0.5, rng.uniform(0, 8, (2, 8)), rng.normal(0, 1, (3, 8)))
    run.load(1, 1.0, 1.0, 0.5, np.array([[3.5], [2.5]]), np.array([[np.nan], [0.0], [0.0]]))
    run.step(3)
    d = run.diag()
    assert d["status"] == pic.PIC_ENAN
    assert d["error_flags"] & 2
    with pytest.raises(pic.PicError) as e:
        run.sync()
    assert e.value.status == pic.PIC_ENAN
    run.close()


def test_diagnostics_match_oracle_and_keep_total_energy():
    """pic_diag on the Langmuir oscillation of the oracle's energy pin (quiet neutral pair
    plasma, dx = 0.5): field energy, kinetic energy, charge and the Gauss residual follow the
    oracle's (FP64 form; 1e-9 over the 440 steps: round-off grows about linearly in this
    non-chaotic oscillation, 2e-12 after 40 steps), and in both forms the total energy stays
    within 5% of the energy the oscillation exchanges."""
    import test_oracle_pins as pins
    grid, dx, dt = (32, 2), (0.5, 0.5), 0.1
    x, ue, up, w = pins._langmuir(grid, dx, dt, 0.2, 0.01)
    orc = oracle.Sim(grid, dx, dt, 2, 0)
    orc.add_species(-1.0, 1.0, w, x, ue)
    orc.add_species(1.0, 1.0, w, x, up)
    runs = {}
    for prec in (pic.PIC_FP64, pic.PIC_FP32_MIXED):
        r = pic.Run(grid, dx, dt, 2, 0, precision=prec, capacity=(x.shape[1], x.shape[1]))
        r.load(0, -1.0, 1.0, w, x, ue)
        r.load(1, 1.0, 1.0, w, x, up)
        runs[prec] = (r, [], [])
    for it in range(110):
        orc.step(4)
        do = orc.diag()
        for prec, (r, ke, fe) in runs.items():
            r.step(4)
            d = r.diag()
            assert d["error_flags"] == 0
            ke.append(d["kinetic_energy"])
            fe.append(d["field_energy"])
            if prec == pic.PIC_FP64 and it % 10 == 9:
                for key in ("field_energy", "kinetic_energy", "total_charge"):
                    assert abs(d[key] - do[key]) <= 1e-9 * max(abs(do[key]), 1e-300), key
                assert abs(d["max_gauss_residual"] - do["max_gauss_residual"]) <= 1e-9 * abs(w) / 0.25
    for prec, (r, ke, fe) in runs.items():
        ke, fe = np.array(ke), np.array(fe)
        total = ke + fe
        assert np.max(np.abs(total - total[0])) < 0.05 * (ke.max() - ke.min()), prec
        r.close()
    orc.close()


def test_wt_equals_mc_at_half_step_gpu():
    """c dt = dx/2: the WT tables reduce to W_l, so WT and MC steps agree (Sec. 2)."""
    outs = []
    for scheme in (0, 1):
        wl = plasma.pair_plasma((32, 16), (1.0, 1.0), 0.5, 3, scheme, 4.0, 0.05, 4, omega_p=0.4)
        f = smooth_fields((1, 16, 32), 0.05, seed=1)
        run, orc = make_pair(wl, pic.PIC_FP64, f)
        run.step(3)
        outs.append([run.field(c) for c in range(6)])
        run.close()
    for a, b in zip(*outs):
        assert rel(a, b) < 1e-13


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("grid", [(48, 24), (12, 10, 8)], ids=["2d", "3d"])
def test_load_from_pinned_host_arrays_matches_pageable(prec, grid):
    """pic_load_particles reads page-locked host arrays in place (no staging copies) and
    pageable ones through the staging buffer: both must store the same particles, bit for bit,
    in the same tile order."""
    dim = len(grid)
    wl = plasma.pair_plasma(grid, (1.0,) * dim, 0.3, 2, 1, 5.0, 0.1, 12, omega_p=0.2, seed=33)
    caps = [int(s.x.shape[1]) for s in wl.species]
    runs = []
    for pinned in (False, True):
        r = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps)
        for i, s in enumerate(wl.species):
            x = np.ascontiguousarray(s.x, dtype=np.float64)
            u = np.ascontiguousarray(s.u, dtype=np.float64)
            if pinned:
                x, u = torch.from_numpy(x).pin_memory(), torch.from_numpy(u).pin_memory()
                assert x.is_pinned()
            r.load(i, s.q, s.m, s.w, x, u)
        runs.append(r)
    for i in range(len(wl.species)):
        a, b = runs[0].particles(i), runs[1].particles(i)
        for va, vb in zip(a, b):
            assert np.array_equal(va, vb)
    for r in runs:
        r.close()
