"""The drifting-plasma loaders on the device (pic_load_drifting_plasma and, for Juttner-Synge
momenta by Sobol's method, pic_load_drifting_juttner; App. D) against the same distribution
drawn by the seeded input generator and loaded from arrays: the two implement the one
counter-based generator (SplitMix64) from its published definition, so cells, offsets, the
accepted Sobol attempts and the flip decisions must agree exactly, and the momenta to the last
bits of log/cos/sin."""
import math

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402

CASES = [((48, 20), 2, pic.PIC_FP64, 50.0, 0.01, 6),
         ((48, 20), 3, pic.PIC_FP32_MIXED, 1000.0, 0.1, 8),
         ((33, 17), 4, pic.PIC_FP32_MIXED, 20.0, 0.0, 4),
         ((12, 8, 6), 2, pic.PIC_FP64, 10.0, 0.05, 4)]


def _pair(run_loader, grid, l, prec, gamma, u_th, ppc, colocated, theta=None):
    dx = (1.0,) * len(grid)
    wl = workloads.pair_plasma(grid, dx, 0.3, l, pic.PIC_SCHEME_WT, gamma, u_th, ppc,
                               device="cuda", seed=77, run=3, colocated=colocated, theta=theta)
    caps = [int(s.x.shape[1]) for s in wl.species]
    r = pic.Run(wl.grid, wl.dx, wl.dt, l, pic.PIC_SCHEME_WT, precision=prec, capacity=caps)
    for i, s in enumerate(wl.species):
        if run_loader and theta is not None:
            r.load_drifting_juttner(i, s.q, s.m, s.w, ppc // 2, gamma, theta, seed=77, run=3,
                                    pos_species=0 if colocated else i)
        elif run_loader:
            r.load_drifting_plasma(i, s.q, s.m, s.w, ppc // 2, gamma, u_th, seed=77, run=3,
                                   pos_species=0 if colocated else i)
        else:
            r.load(i, s.q, s.m, s.w, s.x, s.u)
    return r


def _same_particles(a, b, prec):
    for s in range(2):
        xa, ua, ca = a.particles(s)
        xb, ub, cb = b.particles(s)
        assert np.array_equal(ca, cb)          # cells and the tile order: exact
        # the order of the particles of one cell is not unique: compare per-cell sets
        ka = np.lexsort(np.vstack([xa, ca[None, :]])[::-1])
        kb = np.lexsort(np.vstack([xb, cb[None, :]])[::-1])
        xa, ua, xb, ub = xa[:, ka], ua[:, ka], xb[:, kb], ub[:, kb]
        assert np.array_equal(xa, xb)          # positions: exact
        # one rounding of the stored form (an FP32 store may round a last-bit difference of
        # log/cos either way)
        tol = 4e-16 if prec == pic.PIC_FP64 else 1.2e-7
        assert np.max(np.abs(ua - ub)) <= tol * max(1.0, np.max(np.abs(ub)))


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("colocated", [False, True])
def test_device_loader_matches_generator(case, colocated):
    grid, l, prec, gamma, u_th, ppc = case
    a = _pair(True, grid, l, prec, gamma, u_th, ppc, colocated)
    b = _pair(False, grid, l, prec, gamma, u_th, ppc, colocated)
    _same_particles(a, b, prec)
    a.step(3)
    b.step(3)
    # same particle sets; the summation order of the current (order within a cell) is not
    # unique, so the fields agree to the rounding of the form's current accumulation.  (With
    # the neutral start the net fields are the small difference of the species' currents, and
    # comparing them measures that cancellation, not the loader.)
    if not colocated:
        ftol = 1e-12 if prec == pic.PIC_FP64 else 2e-6
        for c in range(9):
            fa, fb = a.field(c), b.field(c)
            den = max(np.max(np.abs(fb)), 1e-300)
            assert np.max(np.abs(fa - fb)) / den < ftol
    assert a.diag()["error_flags"] == 0
    a.close()
    b.close()


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
def test_device_juttner_loader_matches_generator(case):
    grid, l, prec, gamma, theta, ppc = case
    a = _pair(True, grid, l, prec, gamma, 0.0, ppc, False, theta)
    b = _pair(False, grid, l, prec, gamma, 0.0, ppc, False, theta)
    _same_particles(a, b, prec)
    # at gamma = 1 (no boost, no flip) the loaded |u| is the Sobol speed itself: mean gamma of
    # the Juttner-Synge distribution is 3 theta + K1(1/theta) / K2(1/theta)
    if gamma == 1.0:
        from scipy.special import kve
        u = np.concatenate([a.particles(s)[1] for s in range(2)], axis=1)
        g = np.sqrt(1.0 + np.sum(u * u, axis=0))
        expect = 3.0 * theta + kve(1, 1.0 / theta) / kve(2, 1.0 / theta)
        assert abs(g.mean() - expect) < 5.0 * g.std() / math.sqrt(g.size)
    a.step(3)
    b.step(3)
    ftol = 1e-12 if prec == pic.PIC_FP64 else 2e-6
    for c in range(9):
        fa, fb = a.field(c), b.field(c)
        den = max(np.max(np.abs(fb)), 1e-300)
        assert np.max(np.abs(fa - fb)) / den < ftol
    assert a.diag()["error_flags"] == 0
    with pytest.raises(pic.PicError):   # below the temperature the bounded sampler supports
        a.load_drifting_juttner(0, -1.0, 1.0, 1e-3, 1, gamma, 0.2, seed=5)
    a.close()
    b.close()
