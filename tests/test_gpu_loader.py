"""The drifting-plasma loaders on the device (pic_load_drifting_plasma and, for Juttner-Synge
momenta by Sobol's method, pic_load_drifting_juttner; App. D) against the FP64 oracle's loader
(oracle.load_drifting).  Both implement the one counter-based generator (SplitMix64) from its
published definition, so the cells, the positions, the stable tile order, the accepted Sobol
attempts and the flip decisions must agree exactly, and the momenta to the last bits of
log/cos/sin (the FP32 form: to one rounding of the stored FP32 value)."""
import math

import numpy as np
import pytest

import oracle
import workloads
from test_gpu_parity import host_packed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402

CASES = [((48, 20), 2, pic.PIC_FP64, 50.0, 0.01, 6),
         ((48, 20), 3, pic.PIC_FP32_MIXED, 1000.0, 0.1, 16),
         ((33, 17), 4, pic.PIC_FP32_MIXED, 20.0, 0.0, 4),
         ((12, 8, 6), 2, pic.PIC_FP64, 10.0, 0.05, 4)]


def _device_run(wl, prec):
    caps = [wl.ncell * s.per_cell for s in wl.species]
    r = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=prec, capacity=caps)
    for i, s in enumerate(wl.species):
        if wl.theta > 0.0:
            r.load_drifting_juttner(i, s.q, s.m, s.w, s.per_cell, wl.gamma, wl.theta,
                                    seed=wl.seed, run=wl.run, pos_species=s.pos_species)
        else:
            r.load_drifting_plasma(i, s.q, s.m, s.w, s.per_cell, wl.gamma, wl.u_th,
                                   seed=wl.seed, run=wl.run, pos_species=s.pos_species)
    return r


def _check_against_oracle(r, wl, prec):
    """Every particle of the device load against the oracle's draw of the same counters, in
    the oracle's stable tile order."""
    for i, s in enumerate(wl.species):
        x, u, failed = oracle.load_drifting(wl.grid, wl.dx, s.per_cell, wl.gamma, wl.u_th,
                                            wl.theta, wl.seed, wl.run, i, s.pos_species)
        assert failed == 0
        cells, xp, up = host_packed(x, u, wl.grid, wl.dx, wl.dim, prec)
        perm, ts = oracle.tile_sort(wl.grid, r.tile, cells,
                                    oracle.SLOT_MAJOR if r.slot_major else oracle.CELL_MAJOR)
        xg, ug, cg = r.particles(i)
        assert np.array_equal(cg, cells[perm])               # cells and the stable order: exact
        assert np.array_equal(r.tile_offsets(i), ts)
        assert np.array_equal(xg, xp[:, perm])              # positions: exact
        # momenta: log/cos/sin may differ in the last bit between the two math libraries; the
        # FP32 store may round such a difference either way
        tol = 4e-16 if prec == pic.PIC_FP64 else 1.2e-7
        assert np.max(np.abs(ug - up[:, perm])) <= tol * max(1.0, np.max(np.abs(up)))
    return r


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("colocated", [False, True])
def test_device_loader_matches_oracle(case, colocated):
    grid, l, prec, gamma, u_th, ppc = case
    wl = workloads.pair_plasma(grid, (1.0,) * len(grid), 0.3, l, pic.PIC_SCHEME_WT, gamma, u_th,
                               ppc, seed=77, run=3, colocated=colocated)
    r = _device_run(wl, prec)
    _check_against_oracle(r, wl, prec)
    r.step(2)
    assert r.diag()["error_flags"] == 0
    r.close()


def test_device_loader_moments_and_cold_beam():
    """Large sample: <u_x> of the loaded drifting Maxwellian against the App. D value
    gamma (<u'_x flipped> + beta <E'>) evaluated from the co-moving distribution by quadrature,
    <u_y> = <u_z> = 0; the cold beam is exactly u = (sqrt(gamma^2 - 1), 0, 0)."""
    grid, ppc, gamma, u_th = (256, 128), 64, 5.0, 0.3
    r = pic.Run(grid, (1.0, 1.0), 0.3, 2, pic.PIC_SCHEME_WT, precision=pic.PIC_FP64,
                capacity=[grid[0] * grid[1] * ppc // 2] * 2)
    r.load_drifting_plasma(0, -1.0, 1.0, 1e-3, ppc // 2, gamma, u_th, seed=5)
    _, u, _ = r.particles(0)
    n = u.shape[1]
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    # App. D: the loaded density in u'_x is proportional to (1 + beta v'_x) f(u'); its mean
    # boosted u_x = gamma <(u'_x + beta E') (1 + beta v'_x)> / <1 + beta v'_x> = gamma <...>
    # since <v'_x> = 0.  Evaluate the 3D Gaussian expectation by Gauss-Hermite quadrature.
    xg, wg = np.polynomial.hermite_e.hermegauss(40)
    wg = wg / wg.sum()
    ux_, uy_, uz_ = np.meshgrid(u_th * xg, u_th * xg, u_th * xg, indexing="ij")
    ww = wg[:, None, None] * wg[None, :, None] * wg[None, None, :]
    ep = np.sqrt(1.0 + ux_ ** 2 + uy_ ** 2 + uz_ ** 2)
    expect = gamma * np.sum(ww * (ux_ + beta * ep) * (1.0 + beta * ux_ / ep))
    sd = gamma * u_th * 2.0
    assert abs(u[0].mean() - expect) < 5.0 * sd / math.sqrt(n)
    assert abs(u[1].mean()) < 5.0 * u_th / math.sqrt(n)
    assert abs(u[2].mean()) < 5.0 * u_th / math.sqrt(n)
    r.load_drifting_plasma(1, 1.0, 1.0, 1e-3, ppc // 2, gamma, 0.0, seed=5)
    _, u1, _ = r.particles(1)
    assert np.all(u1[0] == math.sqrt(gamma * gamma - 1.0)) and np.all(u1[1:] == 0.0)
    # argument checks
    with pytest.raises(pic.PicError):
        r.load_drifting_plasma(0, -1.0, 1.0, 1e-3, ppc, gamma, u_th, seed=5)   # over capacity
    with pytest.raises(pic.PicError):
        r.load_drifting_plasma(0, -1.0, 1.0, 1e-3, 2, 0.5, u_th, seed=5)       # gamma < 1
    r.close()


JCASES = [((48, 20), 2, pic.PIC_FP64, 50.0, 0.3, 6),
          ((33, 17), 3, pic.PIC_FP32_MIXED, 1000.0, 1.0, 4),
          ((12, 8, 6), 2, pic.PIC_FP64, 1.0, 4.0, 4)]


@pytest.mark.parametrize("case", JCASES)
def test_device_juttner_loader_matches_oracle(case):
    grid, l, prec, gamma, theta, ppc = case
    wl = workloads.pair_plasma(grid, (1.0,) * len(grid), 0.3, l, pic.PIC_SCHEME_WT, gamma, 0.0,
                               ppc, seed=77, run=3, theta=theta)
    a = _device_run(wl, prec)
    _check_against_oracle(a, wl, prec)
    # at gamma = 1 (no boost, no flip) the loaded |u| is the Sobol speed itself: mean gamma of
    # the Juttner-Synge distribution is 3 theta + K1(1/theta) / K2(1/theta)
    if gamma == 1.0:
        from scipy.special import kve
        u = np.concatenate([a.particles(s)[1] for s in range(2)], axis=1)
        g = np.sqrt(1.0 + np.sum(u * u, axis=0))
        expect = 3.0 * theta + kve(1, 1.0 / theta) / kve(2, 1.0 / theta)
        assert abs(g.mean() - expect) < 5.0 * g.std() / math.sqrt(g.size)
    a.step(2)
    assert a.diag()["error_flags"] == 0
    with pytest.raises(pic.PicError):   # below the temperature the bounded sampler supports
        a.load_drifting_juttner(0, -1.0, 1.0, 1e-3, 1, gamma, 0.2, seed=5)
    a.close()


def test_engine_requests_load_on_the_device():
    """The served and batched forms generate every request's plasma with the device loader:
    a request's run holds the oracle's draw of the same streams."""
    from paper_1909_09613_gb300 import engine
    req = engine.Request(rid=5, grid=(40, 24, 1), dt=0.3, l=3, gamma=30.0, u_th=0.01, ppc=16,
                         steps=1, seed=99)
    r = engine.make_run(req)
    wl = workloads.pair_plasma((40, 24), (1.0, 1.0), 0.3, 3, 1, 30.0, 0.01, 16, seed=99, run=5)
    for i, s in enumerate(wl.species):
        assert engine.species_constants(req, i) == (s.q, s.m, s.w, s.per_cell, s.pos_species)
    _check_against_oracle(r, wl, req.precision)
    r.close()
