"""Charge-conservation diagnostics of pic_diag and the deterministic mode of pic_step.

* max_continuity_residual = max |(rho^{n+1} - rho^n)/dt + D.J^{n+1/2}| (the discrete continuity
  equation of the Esirkepov deposit, Sec. 1; App. B) and max_gauss_residual_drift = max |G - G_0|
  with G = D.E - rho (App. B, Eq. gauss) are recomputed on the host from the read-back state --
  the oracle's rho of the read-back particles, the read-back E and J -- and must agree with the
  device's values to FP64 round-off of those sums; both stay at the round-off of the form.
* pic_options.deterministic: two runs from the same state give bit-identical fields and
  particles after steps that cross tile sorts, and one step agrees with the oracle at the
  tolerance of the form.
"""
import numpy as np
import pytest

import oracle
import plasma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402
from test_gpu_parity import FP32_TOL, FP64_TOL, compare_state, make_pair, smooth_fields  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1909_09613_gb300 import _build
    _build.build()
    oracle.build()


def host_rho(run, wl):
    """rho of the run's current particles by the oracle (Sec. 2, Eq. shape-real)."""
    dim = wl.dim
    orc = oracle.Sim(wl.grid[:dim], wl.dx[:dim], wl.dt, wl.l, wl.scheme)
    for i, s in enumerate(wl.species):
        x, u, _ = run.particles(i)
        orc.add_species(s.q, s.m, s.w, x, u)
    r = orc.rho()
    orc.close()
    return r


def div_back(fx, fy, fz, dx, dim):
    """Backward-difference divergence at integer nodes of a Yee-staggered vector (E or J)."""
    d = (fx - np.roll(fx, 1, axis=2)) / dx[0] + (fy - np.roll(fy, 1, axis=1)) / dx[1]
    if dim == 3:
        d = d + (fz - np.roll(fz, 1, axis=0)) / dx[2]
    return d


CASES = [((40, 24), 0.3, 3, 16), ((37, 21), 0.45, 2, 4), ((12, 10, 8), 0.3, 2, 4)]


@pytest.mark.parametrize("prec", [pic.PIC_FP64, pic.PIC_FP32_MIXED], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=["2d_l3_ppc16", "2d_l2_ppc4", "3d_l2"])
def test_continuity_and_gauss_drift_match_host(case, prec):
    grid, cdt, l, ppc = case
    dim = len(grid)
    wl = plasma.pair_plasma(grid, (1.0,) * dim, cdt, l, 1, 5.0, 0.1, ppc, omega_p=0.3, seed=31)
    shape = (grid[2] if dim == 3 else 1, grid[1], grid[0])
    f = smooth_fields(shape, 0.05, seed=17)
    run, orc = make_pair(wl, prec, f)
    orc.close()
    dx = wl.dx
    d0 = run.diag()
    assert np.isnan(d0["max_continuity_residual"])  # no earlier pic_diag
    assert d0["max_gauss_residual_drift"] == 0.0     # no step since the load
    rho0 = host_rho(run, wl)
    E0 = [run.field(c) for c in range(3)]
    g0 = div_back(E0[0], E0[1], E0[2], dx, dim) - rho0
    rho_scale = np.max(np.abs(rho0))
    run.step(1)
    d1 = run.diag()
    rho1 = host_rho(run, wl)
    J = [run.field(6 + a) for a in range(3)]
    cont = np.max(np.abs((rho1 - rho0) / wl.dt + div_back(J[0], J[1], J[2], dx, dim)))
    scale = rho_scale / wl.dt
    assert abs(d1["max_continuity_residual"] - cont) <= 1e-10 * scale
    # Esirkepov: continuity at FP64 round-off; FP32 form: at the FP32 round-off of the current
    assert d1["max_continuity_residual"] <= (1e-12 if prec == pic.PIC_FP64 else 2e-5) * scale
    run.step(2)  # two steps since the last pic_diag: no continuity residual
    d3 = run.diag()
    assert np.isnan(d3["max_continuity_residual"])
    rho3 = host_rho(run, wl)
    E3 = [run.field(c) for c in range(3)]
    g3 = div_back(E3[0], E3[1], E3[2], dx, dim) - rho3
    drift = np.max(np.abs(g3 - g0))
    assert abs(d3["max_gauss_residual_drift"] - drift) <= 1e-10 * rho_scale
    assert d3["max_gauss_residual_drift"] <= (1e-11 if prec == pic.PIC_FP64 else 1e-4) * rho_scale
    assert abs(d3["max_gauss_residual"] - np.max(np.abs(g3))) <= 1e-10 * rho_scale
    # a field set moves the reference to the next step
    run.set_field(0, E3[0])
    assert run.diag()["max_gauss_residual_drift"] == 0.0
    run.close()


DET_CASES = [
    # (grid, cdt, l, ppc, prec)
    ((48, 24), 0.3, 3, 16, pic.PIC_FP32_MIXED),   # cell-major warp sums
    ((40, 24), 0.45, 2, 4, pic.PIC_FP32_MIXED),   # slot-major per-lane atomics
    ((40, 24), 0.3, 3, 8, pic.PIC_FP64),
    ((12, 10, 8), 0.3, 2, 6, pic.PIC_FP32_MIXED),
    ((12, 10, 8), 0.3, 2, 6, pic.PIC_FP64),
]


def _det_run(case, f, seed=41):
    """A deterministic run of the case from the oracle-drawn plasma, fields f set."""
    grid, cdt, l, ppc, prec = case
    dim = len(grid)
    wl = plasma.pair_plasma(grid, (1.0,) * dim, cdt, l, 1, 8.0, 0.1, ppc, omega_p=0.3, seed=seed)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps,
                  deterministic=True)
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, s.u)
    for c, a in enumerate(f):
        run.set_field(c, a)
    return wl, run


@pytest.mark.parametrize("case", DET_CASES, ids=["fp32_cell", "fp32_slot", "fp64", "3d_fp32", "3d_fp64"])
def test_deterministic_runs_are_bit_identical(case):
    grid = case[0]
    dim = len(grid)
    shape = (grid[2] if dim == 3 else 1, grid[1], grid[0])
    f = smooth_fields(shape, 0.05, seed=23)
    runs = [_det_run(case, f)[1] for _ in range(2)]
    if case[4] == pic.PIC_FP32_MIXED and dim == 2:
        # cell-major from 4 particles of a species per cell for odd l, from 6 for even l
        assert runs[0].slot_major == (0 if case[3] // 2 >= (4 if case[2] % 2 else 6) else 1)
    for r in runs:
        assert r.sort_interval < 12
        r.step(12)
    for c in range(9):
        assert np.array_equal(runs[0].field(c), runs[1].field(c)), c
    for s in range(2):
        a, b = runs[0].particles(s), runs[1].particles(s)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), s
    assert runs[0].diag()["error_flags"] == 0
    for r in runs:
        r.close()


@pytest.mark.parametrize("case", DET_CASES, ids=["fp32_cell", "fp32_slot", "fp64", "3d_fp32", "3d_fp64"])
def test_deterministic_step_matches_oracle(case):
    grid, cdt, l, ppc, prec = case
    dim = len(grid)
    shape = (grid[2] if dim == 3 else 1, grid[1], grid[0])
    f = smooth_fields(shape, 0.05, seed=29)
    wl = plasma.pair_plasma(grid, (1.0,) * dim, cdt, l, 1, 8.0, 0.1, ppc, omega_p=0.3, seed=43)
    run, orc = make_pair(wl, prec, f, deterministic=True)
    run.step(1)
    orc.step(1)
    compare_state(run, orc, 2, FP64_TOL if prec == pic.PIC_FP64 else FP32_TOL, case)
    run.close()


def test_batch_refuses_deterministic_runs():
    wl = plasma.pair_plasma((32, 16), (1.0, 1.0), 0.3, 2, 1, 5.0, 0.1, 16, omega_p=0.3)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=pic.PIC_FP32_MIXED,
                  capacity=caps, deterministic=True)
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, s.u)
    with pytest.raises(pic.PicError) as e:
        pic.Batch([run])
    assert e.value.status == pic.PIC_EINVAL
    run.close()
