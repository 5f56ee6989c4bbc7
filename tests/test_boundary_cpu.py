"""CPU checks of the C-ABI boundary: the library loads, exports every declared symbol, and its
host-side logic (argument validation, footprint, interpolation tables) is right.  No device
work is issued here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1909_09613_gb300 as pic
from paper_1909_09613_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return pic.load_library()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pic_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(pic.exported_names()) | {"pic_strerror"}


def test_binding_constants_match_the_header():
    txt = open(os.path.join(ROOT, "include", "pic.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    found = {}
    for name, val in re.findall(r"#define\s+(PIC_[A-Z0-9_]+)\s+([-0-9.]+)\s*$", txt, flags=re.M):
        found[name] = float(val)
    for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", txt, flags=re.S):
        for name, val in re.findall(r"(PIC_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            found[name] = float(val)
    assert len(found) > 20
    for name, val in found.items():
        assert getattr(pic, name) == val, name


def test_juttner_loader_rejects_cold_theta(lib):
    """Sobol's method needs theta >= 0.3 for its bounded attempts; the check precedes any use
    of the context, so it is exercised here without a device."""
    f = lib.pic_load_drifting_juttner
    for theta in (0.0, 0.29, float("nan"), -1.0):
        assert f(None, 0, -1.0, 1.0, 1.0, 1, 10.0, theta, 1, 0, 0) == pic.PIC_EINVAL
    assert f(None, 0, -1.0, 1.0, 1.0, 1, 10.0, 0.5, 1, 0, 0) == pic.PIC_EINVAL  # no context


def test_strerror(lib):
    assert pic.pic_strerror(0) == "ok"
    assert "Courant" in pic.pic_strerror(pic.PIC_ECFL)


def _opt(cap=(100, 100), prec=pic.PIC_FP64):
    o = pic.pic_options()
    o.n_species = len(cap)
    for i, c in enumerate(cap):
        o.capacity[i] = c
    o.precision = prec
    return o


def test_create_validates_courant_and_order(lib):
    with pytest.raises(pic.PicError) as e:
        pic.pic_create((64, 32, 1), (1.0, 1.0, 1.0), 0.71, 2, pic.PIC_SCHEME_WT, _opt())
    assert e.value.status == pic.PIC_ECFL
    with pytest.raises(pic.PicError) as e:
        pic.pic_create((64, 32, 1), (1.0, 1.0, 1.0), 0.3, 5, pic.PIC_SCHEME_WT, _opt())
    assert e.value.status == pic.PIC_EINVAL
    with pytest.raises(pic.PicError) as e:
        pic.pic_create((16, 16, 16), (1.0, 1.0, 1.0), 0.58, 2, pic.PIC_SCHEME_WT, _opt())
    assert e.value.status == pic.PIC_ECFL


def test_size_limits(lib):
    """The largest accepted sizes and the first refused ones: 2^30 cells (int32 cell indices and
    tile keys), 2^31 - 1 particles per species (int32 slot and key scratch of the sort), 1024
    cells per tile.  Creation and the footprint query only: nothing is allocated."""
    big = 2 ** 31 - 1
    ctx = pic.pic_create((1 << 15, 1 << 15, 1), (1.0, 1.0, 1.0), 0.25, 3, pic.PIC_SCHEME_WT,
                         _opt((big, 1), pic.PIC_FP32_MIXED))
    try:
        b = pic.pic_footprint(ctx)
        assert b >= 2 * big * 24 + (1 << 30) * 9 * 8   # two FP32 stores + the FP64 grid
    finally:
        pic.pic_destroy(ctx)
    for grid, cap, tile in ((((1 << 15) + 1, 1 << 15, 1), (16, 16), None),
                            ((64, 32, 1), (2 ** 31, 1), None),
                            ((64, 32, 1), (16, 16), (64, 32, 1))):
        o = _opt(cap)
        if tile:
            for a in range(3):
                o.tile[a] = tile[a]
        with pytest.raises(pic.PicError) as e:
            pic.pic_create(grid, (1.0, 1.0, 1.0), 0.25, 3, pic.PIC_SCHEME_WT, o)
        assert e.value.status == pic.PIC_EINVAL, (grid, cap, tile)


def test_smem_info(lib):
    """Shared memory per CTA of the particle kernels (host query): the batched kernel's stage
    carries no T tables of its own but a copy of the run descriptor; the FP64 form has no
    batched items; a larger tile needs more; without a device the two-per-SM limit is 0."""
    sizes = {}
    for tile in ((16, 8), (64, 8)):
        o = _opt((1 << 20, 1 << 20), pic.PIC_FP32_MIXED)
        o.tile[0], o.tile[1], o.tile[2] = tile[0], tile[1], 1
        ctx = pic.pic_create((512, 256, 1), (1.0, 1.0, 1.0), 0.4, 3, pic.PIC_SCHEME_WT, o)
        try:
            sizes[tile] = pic.pic_smem_info(ctx)
        finally:
            pic.pic_destroy(ctx)
    own, batched, two = sizes[(64, 8)]
    assert own > 64 * 1024 and batched > 0 and abs(batched - own) < 8 * 1024
    assert sizes[(16, 8)][0] < own and sizes[(16, 8)][1] < batched
    ctx = pic.pic_create((512, 256, 1), (1.0, 1.0, 1.0), 0.4, 3, pic.PIC_SCHEME_WT, _opt())
    try:
        assert pic.pic_smem_info(ctx)[1] == 0
    finally:
        pic.pic_destroy(ctx)


def test_create_m4_courant_limit(lib):
    """Courant limit with the M4 stencil (App. C): on these grids the worst wavenumber is a
    corner of the Brillouin zone and the limit coincides with Yee's (1/sqrt(2) for dx = dy,
    1/sqrt(1 + 1/4) for dy = 2 dx)."""
    for grid, dx, ok, bad in (((64, 32, 1), (1.0, 1.0, 1.0), 0.70, 0.71),
                              ((64, 32, 1), (1.0, 2.0, 1.0), 0.89, 0.90)):
        o = _opt()
        o.solver = pic.PIC_SOLVER_M4
        ctx = pic.pic_create(grid, dx, ok, 2, pic.PIC_SCHEME_WT, o)
        pic.pic_destroy(ctx)
        with pytest.raises(pic.PicError) as e:
            pic.pic_create(grid, dx, bad, 2, pic.PIC_SCHEME_WT, o)
        assert e.value.status == pic.PIC_ECFL


@pytest.mark.parametrize("grid,prec", [((2048, 1024, 1), pic.PIC_FP64), ((2048, 1024, 1), pic.PIC_FP32_MIXED),
                                       ((64, 32, 1), pic.PIC_FP64), ((128, 32, 32), pic.PIC_FP32_MIXED)])
def test_footprint_is_about_two_stores_plus_fields(lib, grid, prec):
    n = grid[0] * grid[1] * grid[2] * 32
    ctx = pic.pic_create(grid, (1.0, 1.0, 1.0), 0.25, 3, pic.PIC_SCHEME_WT, _opt((n, n), prec))
    try:
        b = pic.pic_footprint(ctx)
        dim = 3 if grid[2] > 1 else 2
        per = (4 + 4 * dim + 12) if prec else (8 * dim + 24)
        ncell = grid[0] * grid[1] * grid[2]
        # FP64 2D (l <= 3) keeps the B-spline weights of the stored positions: 2 (l + 1) doubles
        cache = 2 * (3 + 1) * 8 if (prec == pic.PIC_FP64 and dim == 2) else 0
        low = 2 * 2 * n * per + 2 * n * cache + 9 * 8 * ncell
        staging = min(n, 1 << 22) * (dim + 4) * 8
        assert low <= b <= 1.3 * low + 64 * ncell + staging + (1 << 22)
        tile, ntiles, si, sm = pic.pic_tile_info(ctx)
        assert si >= 1 and ntiles >= 1
    finally:
        pic.pic_destroy(ctx)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
@pytest.mark.parametrize("dtt", [0.1, 0.25, 0.35, 0.5, 0.6, 0.7])
def test_axis_weight_tables_match_oracle_T(lib, l, dtt):
    """The kernels' per-particle T_l weights (Taylor tables) equal the oracle's T_l."""
    rng = np.random.default_rng(l * 100 + int(dtt * 100))
    for delta in np.concatenate([rng.uniform(0, 1, 40), [0.0, 0.5, 1 - 1e-12]]):
        base, w = pic.pic_axis_weights(l, pic.PIC_SCHEME_WT, dtt, delta)
        for k in range(-4, 6):
            node = base + k
            expect = oracle.T(l, dtt, delta - node)
            got = w[k] if 0 <= k < len(w) else 0.0
            assert abs(got - expect) < 1e-14, (delta, node, got, expect)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_axis_weight_tables_mc_are_bsplines(lib, l):
    rng = np.random.default_rng(7 + l)
    for delta in rng.uniform(0, 1, 50):
        base, w = pic.pic_axis_weights(l, pic.PIC_SCHEME_MC, 0.3, delta)
        for k in range(-4, 6):
            got = w[k] if 0 <= k < len(w) else 0.0
            assert abs(got - oracle.W(l, delta - (base + k))) < 1e-14


def _golden(name):
    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            out[line[0]] = [float(v) for v in line[1:]]
    return out


def test_table1_requests_follow_table_1():
    """The Table 1 scan against the printed parameters (tests/golden/table1_parameters.txt):
    2 schemes x 2 solvers x 5 time steps, dt / dt_CFL as printed (dt_CFL = dx / (sqrt 2 c)),
    c dt = dx / 2 exactly for the last one, the printed cells, particles per cell, drift gamma
    and temperature (Gaussian co-moving spread sqrt(kT/mc^2)), a skin depth of 16 cells (the
    printed domain over the printed cells), quartic, samples aligned with the end of the run."""
    import math
    from paper_1909_09613_gb300 import engine
    g = _golden("table1_parameters.txt")
    reqs = engine.table1_requests(50.0, 1.0)
    assert len(reqs) == 20
    ratios = sorted({round(r.dt * math.sqrt(2.0), 12) for r in reqs})
    assert ratios == [round(v, 12) for v in g["dt_over_dt_cfl"]]
    assert any(r.dt == 0.5 for r in reqs)
    cells = tuple(int(v) for v in g["cells"])
    de_cells = cells[0] / g["domain_skin_depths"][0]
    assert de_cells == cells[1] / g["domain_skin_depths"][1] == 16.0
    assert int(g["particles_per_cell"][0]) == 2 * int(g["particles_per_cell_per_species"][0])
    for r in reqs:
        assert r.grid == cells + (1,) and r.ppc == int(g["particles_per_cell"][0]) and r.l == 4
        assert r.gamma == g["drift_lorentz_factor"][0]
        assert abs(r.u_th - math.sqrt(g["temperature_kT_over_mc2"][0])) < 1e-15
        assert r.steps % r.record_every == 0
        assert r.steps * r.dt / 16.0 >= 50.0           # t in 1/omega_pe, 16 cells per d_e
        assert abs(r.record_every * r.dt / 16.0 - 1.0) < 0.6
        assert not r.batchable                          # quartic runs step on their own
    only = {(pic.PIC_SCHEME_WT, pic.PIC_SOLVER_M4, 0)}
    sub = engine.table1_requests(50.0, 1.0, only=only)
    assert len(sub) == 1 and sub[0].solver == pic.PIC_SOLVER_M4
    assert abs(sub[0].dt - 0.1 / math.sqrt(2.0)) < 1e-15


def test_neutral_start_colocates_species():
    """colocated=True: the positrons take the electrons' positions (rho = 0 at the start),
    momenta independent; the default keeps independent positions.  The engine's request
    normalisation (the weight of a 16-cells-per-skin-depth plasma) equals the workload's."""
    import workloads
    from paper_1909_09613_gb300 import engine
    a = workloads.pair_plasma((8, 4), (1.0, 1.0), 0.3, 2, 1, 50.0, 0.1, 4, colocated=True)
    b = workloads.pair_plasma((8, 4), (1.0, 1.0), 0.3, 2, 1, 50.0, 0.1, 4)
    assert [s.pos_species for s in a.species] == [0, 0]
    assert [s.pos_species for s in b.species] == [0, 1]
    for wl, grid in ((b, (8, 4, 1)), (workloads.pair_plasma((6, 5, 4), (1.0,) * 3, 0.3, 2, 1, 20.0,
                                                              0.01, 8), (6, 5, 4))):
        req = engine.Request(rid=0, grid=grid, dt=0.3, l=2, gamma=wl.gamma, u_th=wl.u_th,
                             ppc=wl.ppc, steps=1)
        for i, s in enumerate(wl.species):
            assert engine.species_constants(req, i) == (s.q, s.m, s.w, s.per_cell, s.pos_species)


def test_fit_batch_tile_without_device_keeps_the_tuned_tile(lib):
    """Without a device the two-per-SM limit is unknown (0): the tuned tile stands."""
    from paper_1909_09613_gb300 import engine
    req = engine.Request(rid=0, grid=(512, 256, 1), l=3, dt=0.7, gamma=20.0, u_th=0.01, ppc=32,
                         steps=1)
    assert engine.fit_batch_tile(req, (64, 16, 1), 4) == ((64, 16, 1), 4)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host, no GPU) prints one JSON line
    with the fields of the bench contract."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1", "--ref-budget", "0.3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def _c_layout(struct, fields):
    """offsetof of `fields` and sizeof of `struct` as the C compiler lays out include/pic.h."""
    import subprocess
    import tempfile
    body = "".join('printf("%%zu ", offsetof(%s, %s));' % (struct, f) for f in fields)
    src = ('#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\nint main(void){%s'
           'printf("%%zu\\n", sizeof(%s));return 0;}\n' % (body, struct))
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        return [int(v) for v in subprocess.check_output([exe]).split()]


@pytest.mark.parametrize("cls,struct", [(pic.pic_options, "pic_options"), (pic.pic_diag_t, "pic_diag_t"),
                                        (pic.pic_batch_capacity, "pic_batch_capacity")])
def test_struct_layouts_match_the_header(cls, struct):
    """The ctypes mirrors of the option and diagnostics structs have the C header's field
    offsets and size (a field added on one side only would shift every later one)."""
    names = [f[0] for f in cls._fields_]
    want = _c_layout(struct, names)
    got = [getattr(cls, n).offset for n in names] + [ctypes.sizeof(cls)]
    assert got == want


def test_create_validates_deterministic_flag(lib):
    o = _opt((1000, 1000), pic.PIC_FP32_MIXED)
    o.deterministic = 2
    with pytest.raises(pic.PicError) as e:
        pic.pic_create((256, 128, 1), (1.0, 1.0, 1.0), 0.25, 3, pic.PIC_SCHEME_WT, o)
    assert e.value.status == pic.PIC_EINVAL
    # a deterministic FP32 run keeps 64-bit words in its shared current tile: 32 x 8 tiles
    for det, tile in ((0, (64, 8, 1)), (1, (32, 8, 1))):
        o.deterministic = det
        ctx = pic.pic_create((256, 128, 1), (1.0, 1.0, 1.0), 0.25, 3, pic.PIC_SCHEME_WT, o)
        try:
            assert pic.pic_tile_info(ctx)[0] == tile
            own, _, _ = pic.pic_smem_info(ctx)
            assert own > 0
        finally:
            pic.pic_destroy(ctx)


@pytest.mark.parametrize("dtt", [0.1, 0.25, 0.4, 0.5, 0.6])
def test_default_sort_interval_keeps_particles_in_the_halo(lib, dtt):
    """The default sort interval K bounds the drift since the last sort, (K - 1) c dt/dx, by
    the staged halo: 2 cells in 2D, 1 cell in the 3D FP32 form (whose tile stage holds one
    cell of drift), and K = 8 for the 3D FP64 form (fields through L1).  The FP32 3D stage
    must fit in shared memory."""
    cases = [((128, 64, 1), pic.PIC_FP64, 2), ((128, 64, 1), pic.PIC_FP32_MIXED, 2),
             ((64, 16, 16), pic.PIC_FP32_MIXED, 1), ((64, 16, 16), pic.PIC_FP64, None)]
    for grid, prec, drift in cases:
        if grid[2] > 1 and dtt * np.sqrt(3.0) >= 1.0:
            continue  # beyond the 3D Courant limit
        n = grid[0] * grid[1] * grid[2] * 4
        ctx = pic.pic_create(grid, (1.0, 1.0, 1.0), dtt, 2, pic.PIC_SCHEME_WT, _opt((n, n), prec))
        try:
            _, _, si, _ = pic.pic_tile_info(ctx)
            if drift is None:
                assert si == 8
            else:
                assert si == int(np.floor(drift / dtt)) + 1
                assert (si - 1) * dtt <= drift + 1e-12
            if grid[2] > 1 and prec == pic.PIC_FP32_MIXED:
                own = pic.pic_smem_info(ctx)[0]
                assert 0 < own <= 75 * 1024  # three 128-thread blocks per SM
        finally:
            pic.pic_destroy(ctx)


@pytest.mark.parametrize("l,per_species,cell_major", [(3, 4, True), (3, 3, False), (2, 4, False),
                                                       (2, 6, True), (4, 5, False), (1, 4, True)])
def test_tile_order_threshold_depends_on_spline_order(lib, l, per_species, cell_major):
    """FP32 runs use the cell-major tile order from 4 particles of a species per cell for odd l
    (the lanes of one cell row share their y window) and from 6 for even l; the FP64 form always
    uses the slot-major order."""
    grid = (128, 64, 1)
    n = grid[0] * grid[1] * per_species
    for prec in (pic.PIC_FP32_MIXED, pic.PIC_FP64):
        ctx = pic.pic_create(grid, (1.0, 1.0, 1.0), 0.3, l, pic.PIC_SCHEME_WT, _opt((n, n), prec))
        try:
            slot_major = pic.pic_tile_info(ctx)[3]
            want = 0 if (cell_major and prec == pic.PIC_FP32_MIXED) else 1
            assert slot_major == want, (l, per_species, prec)
        finally:
            pic.pic_destroy(ctx)


@pytest.mark.parametrize("l,per_species,cell_major", [(2, 4, True), (2, 3, False), (3, 4, True)])
def test_tile_order_threshold_3d(lib, l, per_species, cell_major):
    """3D FP32 runs (current by L2 reductions, no warp frame) use the cell-major order from 4
    particles of a species per cell for every spline order."""
    grid = (32, 16, 16)
    n = grid[0] * grid[1] * grid[2] * per_species
    ctx = pic.pic_create(grid, (1.0, 1.0, 1.0), 0.3, l, pic.PIC_SCHEME_WT,
                         _opt((n, n), pic.PIC_FP32_MIXED))
    try:
        assert pic.pic_tile_info(ctx)[3] == (0 if cell_major else 1)
    finally:
        pic.pic_destroy(ctx)
