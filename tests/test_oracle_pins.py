"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Every test here checks the oracle against something other than itself: a closed form printed
in the paper, a textbook identity, a brute-force sum, a Fourier transform computed
numerically, a conservation law, or an analytic trajectory.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import MC, WT, Sim

RNG = np.random.default_rng(1909096130)


# ------------------------------------------------------------------------------------------
# W_l: B-splines (Sec. 2, Eq. shape-real)
# ------------------------------------------------------------------------------------------

def _w_closed(l, x):
    """Textbook closed forms of the centred B-splines of order 1..4."""
    a = abs(x)
    if l == 1:
        return max(0.0, 1.0 - a)
    if l == 2:
        if a <= 0.5:
            return 0.75 - a * a
        return 0.5 * (1.5 - a) ** 2 if a < 1.5 else 0.0
    if l == 3:
        if a <= 1.0:
            return 2.0 / 3.0 - a * a + 0.5 * a ** 3
        return (2.0 - a) ** 3 / 6.0 if a < 2.0 else 0.0
    if l == 4:
        if a <= 0.5:
            return 115.0 / 192.0 - 5.0 * a * a / 8.0 + a ** 4 / 4.0
        if a <= 1.5:
            return (55.0 + 20.0 * a - 120.0 * a * a + 80.0 * a ** 3 - 16.0 * a ** 4) / 96.0
        return (2.5 - a) ** 4 / 24.0 if a < 2.5 else 0.0
    raise ValueError(l)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_W_closed_form(l):
    xs = np.concatenate([RNG.uniform(-3.0, 3.0, 400), np.arange(-3.0, 3.01, 0.5)])
    for x in xs:
        assert abs(oracle.W(l, x) - _w_closed(l, x)) < 1e-15


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_W_partition_of_unity_and_unit_integral(l):
    for x in RNG.uniform(0.0, 1.0, 50):
        s = sum(oracle.W(l, x - n) for n in range(-4, 6))
        assert abs(s - 1.0) < 1e-14
    # integral by the composite Simpson rule on knot-aligned panels (exact for cubics)
    h = 1.0 / 64
    xs = np.arange(-3.0, 3.0 + h / 2, h)
    ys = np.array([oracle.W(l, x) for x in xs])
    simpson = h / 3.0 * (ys[0] + ys[-1] + 4 * ys[1:-1:2].sum() + 2 * ys[2:-1:2].sum())
    assert abs(simpson - 1.0) < 1e-9


# ------------------------------------------------------------------------------------------
# T_l: the WT interpolation functions (Sec. 2, Eq. tau_l and the four printed closed forms)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("l", [1, 2, 3, 4])
@pytest.mark.parametrize("dtt", [0.05, 0.25, 0.35, 0.5])
def test_T_definition_matches_printed_closed_forms(l, dtt):
    xs = np.concatenate([RNG.uniform(-3.2, 3.2, 300), np.arange(-3.0, 3.01, 0.25)])
    for x in xs:
        a = oracle.T(l, dtt, x)
        b = oracle.T_paper(l, dtt, x)
        assert abs(a - b) < 2e-14, (l, dtt, x, a, b)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_T_at_half_step_equals_W(l):
    """c dt = dx/2 gives tau_l = s_l, so T_l = W_l and WT recovers MC (Sec. 2)."""
    for x in RNG.uniform(-3.0, 3.0, 200):
        assert abs(oracle.T(l, 0.5, x) - oracle.W(l, x)) < 1e-14
        assert abs(oracle.T_paper(l, 0.5, x) - oracle.W(l, x)) < 1e-14


@pytest.mark.parametrize("l", [1, 2, 3, 4])
@pytest.mark.parametrize("dtt", [0.1, 0.35, 0.6, 0.7])
def test_T_partition_of_unity(l, dtt):
    for x in RNG.uniform(0.0, 1.0, 30):
        s = sum(oracle.T(l, dtt, x - n) for n in range(-5, 7))
        assert abs(s - 1.0) < 1e-14


@pytest.mark.parametrize("l", [2, 3, 4])
def test_T_small_step_limit_is_lower_order_spline(l):
    """sinc(k c dt) -> 1 as dt -> 0, so T_l -> W_{l-1}."""
    for x in RNG.uniform(-2.5, 2.5, 100):
        assert abs(oracle.T(l, 1e-7, x) - oracle.W(l - 1, x)) < 1e-6


def _ft_even(f, support, k, panels=2048):
    """integral f(x) cos(k x) dx by Gauss-Legendre on many panels (f is even)."""
    gx, gw = np.polynomial.legendre.leggauss(8)
    edges = np.linspace(-support, support, panels + 1)
    tot = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        c, h = 0.5 * (a + b), 0.5 * (b - a)
        xs = c + h * gx
        tot += h * sum(w * f(x) * math.cos(k * x) for w, x in zip(gw, xs))
    return tot


@pytest.mark.parametrize("l,dtt", [(2, 0.25), (3, 0.35), (3, 0.6), (4, 0.1)])
def test_T_fourier_transform_is_tau(l, dtt):
    """F(T_l) = sinc^l(k dx/2) sinc(k c dt) (Sec. 2, Eq. tau_l), in cell units."""
    sup = 0.5 * l + dtt + 0.01
    for k in (0.7, 1.9, 3.0):
        num = _ft_even(lambda x: oracle.T(l, dtt, x), sup, k, panels=256)
        tau = (math.sin(k / 2) / (k / 2)) ** l * (math.sin(k * dtt) / (k * dtt))
        assert abs(num - tau) < 1e-7, (k, num, tau)


# ------------------------------------------------------------------------------------------
# Field gather (Eq. interpolation-EB-real-org and Eq. interpolation-EB-real-mod)
# ------------------------------------------------------------------------------------------

def _random_sim(grid, scheme, dtt, l, rng):
    s = oracle.Sim(grid, (1.0,) * len(grid), dtt, l, scheme)
    for c in range(6):
        s.set_field(c, rng.standard_normal(s.shape))
    return s


@pytest.mark.parametrize("scheme,dtt,l", [(MC, 0.3, 2), (WT, 0.3, 2), (WT, 0.25, 3),
                                          (WT, 0.6, 3), (WT, 0.1, 4), (WT, 0.45, 1)])
def test_gather_window_equals_brute_force_2d(scheme, dtt, l):
    s = _random_sim((8, 8), scheme, dtt, l, RNG)
    for _ in range(6):
        p = RNG.uniform(0.0, 8.0, 2)
        a, b = s.gather(p), s.gather_brute(p)
        assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("scheme,dtt,l", [(MC, 0.3, 2), (WT, 0.3, 2), (WT, 0.55, 3)])
def test_gather_window_equals_brute_force_3d(scheme, dtt, l):
    s = _random_sim((6, 6, 6), scheme, dtt, l, RNG)
    for _ in range(3):
        p = RNG.uniform(0.0, 6.0, 3)
        a, b = s.gather(p), s.gather_brute(p)
        assert np.max(np.abs(a - b)) < 1e-13


def _fourier_symbols(l, dtt, k, scheme):
    """Per-axis transforms: s_l for W (Eq. s_l), tau_l for T (Eq. tau_l), nu = 0."""
    def s_(kk):
        return 1.0 if kk == 0 else (math.sin(kk / 2) / (kk / 2)) ** (l + 1)

    def t_(kk):
        if scheme == MC:
            return s_(kk)
        if kk == 0:
            return 1.0
        return (math.sin(kk / 2) / (kk / 2)) ** l * math.sin(kk * dtt) / (kk * dtt)
    return s_, t_


@pytest.mark.parametrize("scheme,dtt,l", [(WT, 0.25, 2), (WT, 0.2, 3), (MC, 0.2, 3)])
def test_gather_fourier_symbol_matches_interpolation_tensor(scheme, dtt, l):
    """Cell average of g(x) e^{-ik.x} for a field e^{ik.x_g} on the component's own nodes
    equals the nu = 0 interpolation tensor of Eq. shapeEB (WT) / Eq. shapeEB-org (MC):
    E1 ~ s1 t2, E2 ~ t1 s2, E3 ~ t1 t2, B1 ~ t1 s2, B2 ~ s1 t2, B3 ~ s1 s2 in 2D.
    This pins which axis carries T for every component."""
    n = 16
    m1, m2 = 3, 2
    k1, k2 = 2 * math.pi * m1 / n, 2 * math.pi * m2 / n
    s_, t_ = _fourier_symbols(l, dtt, None, scheme)
    stag = {0: (1, 0), 1: (0, 1), 2: (0, 0), 3: (0, 1), 4: (1, 0), 5: (1, 1)}
    expect = {}
    for c, (a1, a2) in stag.items():
        expect[c] = (s_(k1) if a1 else t_(k1)) * (s_(k2) if a2 else t_(k2))
    sims = []
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for part in (np.cos, np.sin):
        s = oracle.Sim((n, n), (1.0, 1.0), dtt, l, scheme)
        for c, (a1, a2) in stag.items():
            ph = k1 * (ii + 0.5 * a1) + k2 * (jj + 0.5 * a2)
            s.set_field(c, part(ph)[None])
        sims.append(s)
    M = 40  # midpoint rule over one cell; error is from the spline kinks only
    acc = np.zeros(6, dtype=complex)
    for a in range(M):
        for b in range(M):
            p = np.array([5.0 + (a + 0.5) / M, 7.0 + (b + 0.5) / M])
            g = sims[0].gather(p) + 1j * sims[1].gather(p)
            acc += g * np.exp(-1j * (k1 * p[0] + k2 * p[1]))
    acc /= M * M
    for c in range(6):
        assert abs(acc[c].imag) < 2e-4
        assert abs(acc[c].real - expect[c]) < 2e-4, (c, acc[c], expect[c])


def test_wt_swapped_axes_would_be_detected():
    """The symbols of s and tau differ enough at the test wavenumbers to tell the axes apart."""
    l, dtt = 3, 0.2
    s_, t_ = _fourier_symbols(l, dtt, None, WT)
    k = 2 * math.pi * 3 / 16
    assert abs(s_(k) - t_(k)) > 1e-2


def test_self_force_vanishes_with_transverse_T():
    """App. B: a charge with B-spline form factor, a field whose Green's function is odd along
    the force axis (periodic centred-difference gradient of the periodic Poisson solution,
    co-located with rho along that axis), W along the force axis and T along the transverse
    axis gives zero self-force for any dt; T along the force axis does not."""
    n = 16
    for l, dtt in ((1, 0.3), (2, 0.7), (3, 0.3), (4, 0.45)):
        pos = np.array([5.3, 7.77])
        s = oracle.Sim((n, n), (1.0, 1.0), dtt, l, WT)
        s.add_species(1.0, 1.0, 1.0, pos.reshape(2, 1), np.zeros((3, 1)))
        rho = s.rho()[0]
        rho = rho - rho.mean()
        kk = 2 * np.pi * np.fft.fftfreq(n)
        lam = (2 - 2 * np.cos(kk))[None, :] + (2 - 2 * np.cos(kk))[:, None]
        lam[0, 0] = 1.0
        ph = np.fft.fft2(rho) / lam
        ph[0, 0] = 0.0
        phi = np.real(np.fft.ifft2(ph))
        e1 = -(np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1)) / 2.0
        f_ok = f_bad = 0.0
        for j in range(n):
            for i in range(n):
                for mi in (-1, 0, 1):
                    for mj in (-1, 0, 1):
                        xi, yj = pos[0] - i - mi * n, pos[1] - j - mj * n
                        f_ok += oracle.W(l, xi) * oracle.T(l, dtt, yj) * e1[j, i]
                        f_bad += oracle.T(l, dtt, xi) * oracle.W(l, yj) * e1[j, i]
        scale = np.abs(e1).max()
        assert abs(f_ok) < 1e-14 * scale * 100
        assert abs(f_bad) > 1e-4 * scale


# ------------------------------------------------------------------------------------------
# Boris push
# ------------------------------------------------------------------------------------------

def test_boris_gyration_angle_and_energy():
    qmdt, bz = -0.37, 1.3
    u = np.array([3.0, 0.0, 0.4])
    g = math.sqrt(1 + (u ** 2).sum())
    theta = 2 * math.atan(abs(qmdt) * bz / (2 * g))
    out = oracle.boris(qmdt, [0, 0, 0], [0, 0, bz], u)
    assert abs(np.linalg.norm(out) - np.linalg.norm(u)) < 1e-14
    assert abs(out[2] - u[2]) < 1e-15
    ang = math.atan2(out[1], out[0]) - math.atan2(u[1], u[0])
    # negative charge in +B_z rotates counter-clockwise
    assert abs(ang - theta) < 1e-14


def test_boris_exb_drift():
    """Slow particle in crossed E = E_y, B = B_z, |E| << |B|: mean velocity E x B / B^2."""
    ey, bz, dt = 1e-3, 1.0, 0.05
    u = np.zeros(3)
    vs = []
    for _ in range(40000):
        u = oracle.boris(dt, [0, ey, 0], [0, 0, bz], u)
        g = math.sqrt(1 + (u ** 2).sum())
        vs.append(u / g)
    vmean = np.mean(vs, axis=0)
    assert abs(vmean[0] - ey / bz) < 2e-3 * ey / bz
    assert abs(vmean[1]) < 2e-3 * ey / bz


def test_boris_rotation_is_second_order():
    """Pure B: the Boris rotation per step is 2 atan(q B dt / (2 m gamma)) (tan half-angle
    form), so over a fixed time T the phase error against the exact (q B / (m gamma)) T
    shrinks 4x when dt halves (second order), and |u| is kept exactly."""
    qm, bz, T = -1.0, 2.0, 3.0
    u0 = np.array([0.8, 0.0, 0.3])
    g = math.sqrt(1 + (u0 ** 2).sum())
    exact = abs(qm) * bz / g * T
    errs = []
    for n in (40, 80, 160):
        dt = T / n
        u = u0.copy()
        ang = 0.0
        for _ in range(n):
            un = oracle.boris(qm * dt, [0, 0, 0], [0, 0, bz], u)
            d = math.atan2(un[1], un[0]) - math.atan2(u[1], u[0])
            ang += (d + math.pi) % (2 * math.pi) - math.pi
            u = un
        assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-13
        errs.append(abs(abs(ang) - exact))
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


# ------------------------------------------------------------------------------------------
# Esirkepov deposit
# ------------------------------------------------------------------------------------------

def _div(j1, j2, j3, dx):
    d = (j1 - np.roll(j1, 1, axis=2)) / dx[0] + (j2 - np.roll(j2, 1, axis=1)) / dx[1]
    if j1.shape[0] > 1:
        d = d + (j3 - np.roll(j3, 1, axis=0)) / dx[2]
    return d


@pytest.mark.parametrize("grid,l", [((12, 10), 1), ((12, 10), 2), ((12, 10), 3), ((12, 10), 4),
                                    ((8, 7, 9), 2), ((8, 7, 9), 3)])
def test_esirkepov_discrete_continuity(grid, l):
    dim = len(grid)
    dx = (0.7, 1.3, 0.9)[:dim]
    dt = 0.3
    for _ in range(4):
        xo = RNG.uniform(0, 1, dim) * np.array(grid) * np.array(dx)
        step = RNG.uniform(-0.95, 0.95, dim) * np.array(dx)
        xn = xo + step
        L = np.array(grid) * np.array(dx)
        xn_w = np.where(xn >= L, xn - L, np.where(xn < 0, xn + L, xn))
        qw = -0.8
        s = oracle.Sim(grid, dx, dt, l, WT)
        s.add_species(-1.0, 1.0, 0.8, xo.reshape(dim, 1), np.zeros((3, 1)))
        r0 = s.rho()
        s.set_particles(0, xn_w.reshape(dim, 1), np.zeros((3, 1)))
        r1 = s.rho()
        s.deposit(qw, xo, xn, np.array([0.1, -0.2, 0.3]))
        j1, j2, j3 = s.field(6), s.field(7), s.field(8)
        res = (r1 - r0) / dt + _div(j1, j2, j3, list(dx) + [1.0])
        vc = np.prod(dx)
        assert np.max(np.abs(res)) < 1e-13 * abs(qw) / (vc * dt)


def test_esirkepov_motion_along_x_only():
    grid, dx, dt, l = (12, 10), (1.0, 1.0), 0.4, 3
    xo = np.array([5.3, 4.6])
    xn = np.array([5.9, 4.6])
    s = oracle.Sim(grid, dx, dt, l, WT)
    s.deposit(2.0, xo, xn, np.zeros(3))
    j1, j2 = s.field(6)[0], s.field(7)[0]
    assert np.max(np.abs(j2)) == 0.0
    # 1-D: J1(i+1/2, j) = -(q w dx / (Vc dt)) S0y_j sum_{i' <= i} (S1x - S0x)_{i'}
    expect = np.zeros_like(j1)
    for jn in range(10):
        sy = oracle.W(l, xo[1] - jn)
        acc = 0.0
        for i in range(12):
            acc += oracle.W(l, xn[0] - i) - oracle.W(l, xo[0] - i)
            expect[jn, i] = -2.0 * 1.0 / (1.0 * dt) * sy * acc
    assert np.max(np.abs(j1 - expect)) < 1e-14


def test_esirkepov_static_particle_out_of_plane_current():
    grid, dx, dt, l = (10, 10), (1.0, 1.0), 0.4, 2
    x = np.array([4.2, 6.7])
    s = oracle.Sim(grid, dx, dt, l, WT)
    vz = 0.6
    s.deposit(1.5, x, x, np.array([0.0, 0.0, vz]))
    j1, j2, j3 = s.field(6)[0], s.field(7)[0], s.field(8)[0]
    assert np.max(np.abs(j1)) == 0.0 and np.max(np.abs(j2)) == 0.0
    expect = np.array([[1.5 * vz * oracle.W(l, x[0] - i) * oracle.W(l, x[1] - j)
                        for i in range(10)] for j in range(10)])
    assert np.max(np.abs(j3 - expect)) < 1e-15


# ------------------------------------------------------------------------------------------
# Yee solver (App. C, A_i = 1) and Gauss's law (App. B, Eq. gauss)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("grid,dx,cdt,comp,m", [((32, 16), (1.0, 1.0), 0.5, 2, (3, 2, 0)),
                                                 ((24, 20), (0.8, 1.1), 0.4, 2, (3, 2, 0)),
                                                 ((12, 10, 8), (1.0, 0.9, 1.2), 0.45, 0, (0, 2, 1)),
                                                 ((12, 10, 8), (1.0, 1.0, 1.0), 0.5, 2, (3, 1, 0))])
def test_yee_vacuum_dispersion(grid, dx, cdt, comp, m):
    """Transverse standing mode of E_comp (k . e_comp = 0, B = 0 at t = 0): E^n = cos(n w dt) E^0
    with sin^2(w dt/2)/(c dt)^2 = sum_i sin^2(k_i dx_i/2)/dx_i^2 (App. C with A_i = 1)."""
    s = oracle.Sim(grid, dx, cdt, 2, MC)
    sh = s.shape
    kk, jj, ii = np.meshgrid(np.arange(sh[0]), np.arange(sh[1]), np.arange(sh[2]), indexing="ij")
    dim = len(grid)
    k = [2 * math.pi * m[a] / (grid[a] * dx[a]) for a in range(dim)]
    node = [ii + 0.0, jj + 0.0, kk + 0.0]
    node[comp] = node[comp] + 0.5
    ph = sum(k[a] * node[a] * dx[a] for a in range(dim))
    e0 = np.sin(ph + 0.3)
    s.set_field(comp, e0)
    sw2 = sum(math.sin(k[a] * dx[a] / 2) ** 2 / dx[a] ** 2 for a in range(dim))
    w = 2.0 / cdt * math.asin(cdt * math.sqrt(sw2))
    nsteps = 60
    for _ in range(nsteps):
        s.yee_b(0.5 * cdt)
        s.yee_e()
        s.yee_b(0.5 * cdt)
    e = s.field(comp)
    assert np.max(np.abs(e - math.cos(nsteps * w * cdt) * e0)) < 1e-12


@pytest.mark.parametrize("solver", [oracle.YEE, oracle.M4])
def test_vacuum_field_energy_stays_bounded(solver):
    """No particles, random initial E and B: the leapfrog conserves a discrete energy, so the
    field energy 1/2 sum (E^2 + B^2) V_c only oscillates -- no growth over 3000 steps at
    c dt = 0.6 dx (below the Courant limit of App. C for both stencils)."""
    grid = (24, 20)
    s = oracle.Sim(grid, (1.0, 1.0), 0.6, 2, MC, solver=solver)
    rng = np.random.default_rng(11)
    for c in range(6):
        s.set_field(c, rng.standard_normal((1, grid[1], grid[0])))
    u = []
    for _ in range(30):
        s.step(100)
        u.append(s.diag()["field_energy"])
    u = np.array(u)
    assert u.max() < 1.2 * u[0] and u.min() > 0.8 * u[0]
    # no trend: the last third averages like the first
    assert abs(u[20:].mean() / u[:10].mean() - 1.0) < 0.05


def _m4_A(k, dx, cdt):
    """A_i of Eq. Maxwell-A with the M4 coefficients of App. C."""
    dim = len(k)
    out = []
    for i in range(dim):
        a = 1.0
        for j in range(dim):
            if j == i:
                delta = ((cdt / dx[i]) ** 2 - 1.0) / 12.0
                a -= 2 * delta * (1 - math.cos(k[i] * dx[i]))
            else:
                beta = (cdt / dx[j]) ** 2 / 12.0
                a -= 2 * beta * (1 - math.cos(k[j] * dx[j]))
        out.append(a)
    return out


@pytest.mark.parametrize("grid,dx,cdt,comp,m", [((32, 16), (1.0, 1.0), 0.5, 2, (3, 2, 0)),
                                                 ((24, 20), (0.8, 1.1), 0.4, 2, (3, 2, 0)),
                                                 ((12, 10, 8), (1.0, 0.9, 1.2), 0.45, 0, (0, 2, 1))])
def test_m4_vacuum_dispersion(grid, dx, cdt, comp, m):
    """M4 solver: a transverse standing mode follows sin^2(w dt/2)/(c dt)^2 = sum s_i^2 A_i
    with A_i of Eq. Maxwell-A and the M4 beta, delta of App. C."""
    s = oracle.Sim(grid, dx, cdt, 2, MC, solver=oracle.M4)
    sh = s.shape
    kk, jj, ii = np.meshgrid(np.arange(sh[0]), np.arange(sh[1]), np.arange(sh[2]), indexing="ij")
    dim = len(grid)
    k = [2 * math.pi * m[a] / (grid[a] * dx[a]) for a in range(dim)]
    node = [ii + 0.0, jj + 0.0, kk + 0.0]
    node[comp] = node[comp] + 0.5
    ph = sum(k[a] * node[a] * dx[a] for a in range(dim))
    e0 = np.sin(ph + 0.3)
    s.set_field(comp, e0)
    A = _m4_A(k, dx, cdt)
    sw2 = sum(math.sin(k[a] * dx[a] / 2) ** 2 / dx[a] ** 2 * A[a] for a in range(dim))
    w = 2.0 / cdt * math.asin(cdt * math.sqrt(sw2))
    for _ in range(60):
        s.yee_b(0.5 * cdt)
        s.yee_e()
        s.yee_b(0.5 * cdt)
    assert np.max(np.abs(s.field(comp) - math.cos(60 * w * cdt) * e0)) < 1e-12


def _measured_phase_error(solver, m, n=512, cdt=0.5, steps=40):
    """w/(c k) - 1 measured from a simulated x-directed E3 standing wave."""
    s = oracle.Sim((n, 2), (1.0, 1.0), cdt, 2, MC, solver=solver)
    k = 2 * math.pi * m / n
    ii = np.arange(n)[None, None, :] + 0 * np.arange(2)[None, :, None]
    e0 = np.sin(k * ii + 0.2)
    s.set_field(2, e0)
    for _ in range(steps):
        s.yee_b(0.5 * cdt)
        s.yee_e()
        s.yee_b(0.5 * cdt)
    ratio = np.sum(s.field(2) * e0) / np.sum(e0 * e0)
    w = math.acos(ratio) / (steps * cdt)
    return w / k - 1.0


def test_m4_phase_error_is_fourth_order():
    """App. C: the M4 choice cancels the O((k dx)^2) phase-velocity error: halving k divides
    the error by ~16 (Yee: ~4)."""
    e_m4 = [_measured_phase_error(oracle.M4, m) for m in (8, 4)]
    e_yee = [_measured_phase_error(oracle.YEE, m) for m in (8, 4)]
    assert 12 < e_m4[0] / e_m4[1] < 20
    assert 3.5 < e_yee[0] / e_yee[1] < 4.5
    assert abs(e_m4[0]) < 0.05 * abs(e_yee[0])


@pytest.mark.parametrize("solver", [oracle.YEE, oracle.M4])
def test_gauss_law_conserved_over_run(solver):
    """The charge-conserving deposit keeps D.E - rho unchanged (App. B, Eq. gauss); the M4
    solver modifies only Faraday's stencil, so this still holds (Sec. 3)."""
    import plasma
    wl = plasma.pair_plasma((16, 8), (1.0, 1.0), 0.3, 3, WT, 5.0, 0.05, 4, omega_p=0.3)
    s = oracle.Sim(wl.grid[:2], wl.dx[:2], wl.dt, wl.l, WT, solver=solver)
    for sp in wl.species:
        s.add_species(sp.q, sp.m, sp.w, sp.x, sp.u)
    r0 = s.gauss_residual()
    s.step(200)
    r1 = s.gauss_residual()
    scale = np.abs(s.rho()).max()
    assert np.max(np.abs(r1 - r0)) < 1e-11 * scale
    assert s.diag()["field_energy"] > 0.0


def test_wt_equals_mc_at_half_step_full_run():
    """c dt = dx/2 with equal dx: the WT step is the MC step (Sec. 2)."""
    import plasma
    outs = []
    for scheme in (MC, WT):
        wl = plasma.pair_plasma((16, 8), (1.0, 1.0), 0.5, 3, scheme, 4.0, 0.05, 4, omega_p=0.4)
        s = oracle.Sim(wl.grid[:2], wl.dx[:2], wl.dt, wl.l, scheme)
        for sp in wl.species:
            s.add_species(sp.q, sp.m, sp.w, sp.x, sp.u)
        s.step(8)
        outs.append((s.field(0), s.field(5), s.particles(0)[1]))
    for a, b in zip(*outs):
        assert np.max(np.abs(a - b)) <= 1e-13 * max(np.max(np.abs(b)), 1e-300)


# ------------------------------------------------------------------------------------------
# Tile sort order
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("order", [oracle.CELL_MAJOR, oracle.SLOT_MAJOR])
@pytest.mark.parametrize("grid,tile", [((10, 7), (4, 3)), ((8, 8), (8, 8)), ((6, 5, 4), (4, 2, 3))])
def test_tile_sort_order_brute_force(grid, tile, order):
    g3 = list(grid) + [1] * (3 - len(grid))
    t3 = list(tile) + [1] * (3 - len(tile))
    ncell = int(np.prod(g3))
    cells = RNG.integers(0, ncell, 300)
    perm, ts = oracle.tile_sort(grid, tile, cells, order)
    assert sorted(perm.tolist()) == list(range(len(cells)))

    def coords(c):
        return c % g3[0], (c // g3[0]) % g3[1], c // (g3[0] * g3[1])
    ntx = [(g3[a] + t3[a] - 1) // t3[a] for a in range(3)]
    seen = {}
    slot = []
    for c in cells:
        slot.append(seen.get(c, 0))
        seen[c] = seen.get(c, 0) + 1
    prev = None
    for p, src in enumerate(perm):
        i, j, k = coords(cells[src])
        tid = ((k // t3[2]) * ntx[1] + j // t3[1]) * ntx[0] + i // t3[0]
        assert ts[tid] <= p < ts[tid + 1]
        local = ((k % t3[2]) * t3[1] + j % t3[1]) * t3[0] + i % t3[0]
        key = (tid, local, slot[src]) if order == oracle.CELL_MAJOR else (tid, slot[src], local)
        if prev is not None:
            assert key > prev
        prev = key
    # slots follow input order inside a cell
    for c in set(cells.tolist()):
        idx = [p for p in perm if cells[p] == c]
        assert [slot[p] for p in idx] == sorted(slot[p] for p in idx)


# ------------------------------------------------------------------------------------------
# Loader (App. D): the flip reproduces the volume-transform weight
# ------------------------------------------------------------------------------------------

def test_loader_drift_moment():
    """<u_x> = gamma beta (<E'> + <u'_x^2 / E'>) for a drifting Maxwellian loaded with the
    App. D flip; without the volume-transform weight it would be gamma beta <E'>."""
    gamma, uth = 2.0, 0.1
    _, u, failed = oracle.load_drifting((64, 64), (1.0, 1.0), 256, gamma, uth, seed=3)
    assert failed == 0
    ux = u[0]
    beta = math.sqrt(1 - 1 / gamma ** 2)
    # co-moving moments by radial quadrature of the isotropic Gaussian
    r = np.linspace(0, 12 * uth, 200001)
    pdf = 4 * np.pi * r ** 2 * np.exp(-r ** 2 / (2 * uth ** 2)) / (2 * np.pi * uth ** 2) ** 1.5
    ep = np.sqrt(1 + r ** 2)
    m_e = np.trapezoid(pdf * ep, r)
    m_u2e = np.trapezoid(pdf * r ** 2 / (3 * ep), r)
    expect = gamma * beta * (m_e + m_u2e)
    no_flip = gamma * beta * m_e
    err = ux.std() / math.sqrt(len(ux))
    assert abs(ux.mean() - expect) < 5 * err
    assert abs(no_flip - expect) > 20 * err
    # the transverse components are the co-moving Gaussian itself (untouched by the boost)
    assert abs(u[1].std() / uth - 1.0) < 0.01 and abs(u[2].mean()) < 5 * uth / math.sqrt(len(ux))


def test_loader_positions_cold_beam_and_colocation():
    """Particle p sits in cell p / per_cell (x fastest) at an offset in [0, 1); u_th = 0 gives the
    cold beam u = (sqrt(gamma^2 - 1), 0, 0) exactly; a species loaded on another's positions
    (pos_species) shares them exactly while its momenta are its own; a sub-range of particles
    equals the same slice of a whole load (counter-based streams)."""
    grid, per, gamma = (12, 5), 3, 7.0
    x, u, _ = oracle.load_drifting(grid, (0.5, 2.0), per, gamma, 0.0, seed=9, species=1)
    p = np.arange(grid[0] * grid[1] * per)
    cell = p // per
    ci = np.vstack([cell % grid[0], cell // grid[0]]).astype(np.float64)
    off = x / np.array([[0.5], [2.0]]) - ci
    assert np.all(off >= 0.0) and np.all(off < 1.0)
    assert np.all(u[0] == math.sqrt(gamma * gamma - 1.0)) and np.all(u[1:] == 0.0)
    xa, ua, _ = oracle.load_drifting(grid, (1.0, 1.0), per, gamma, 0.05, seed=9, species=0)
    xb, ub, _ = oracle.load_drifting(grid, (1.0, 1.0), per, gamma, 0.05, seed=9, species=1,
                                     pos_species=0)
    xc, _, _ = oracle.load_drifting(grid, (1.0, 1.0), per, gamma, 0.05, seed=9, species=1)
    assert np.array_equal(xa, xb) and not np.array_equal(xa, xc)
    assert not np.array_equal(ua, ub)
    xs, us, _ = oracle.load_drifting(grid, (1.0, 1.0), per, gamma, 0.05, seed=9, species=0,
                                     first=17, count=40)
    assert np.array_equal(xs, xa[:, 17:57]) and np.array_equal(us, ua[:, 17:57])


# ------------------------------------------------------------------------------------------
# App. A: the lowest-order NCI growth rate of Eq. NCI-Xu2013 vanishes for WT at any dt
# ------------------------------------------------------------------------------------------

def _nci_factor(scheme, k1, nu1, k2, l, dx, cdt):
    """S_B3 xi_0 - S_E2 [k]_B1 on the beam resonance omega' = c k1' (App. A), 2D (k3 = 0, the
    x3 factors are 1), with the interpolation tensors of Eq. shapeEB (WT) / shapeEB-org (MC)
    and tau_l of Eq. tau_l, for aliasing order nu1 along x1 (nu2 = 0)."""
    def sinc(x):
        return 1.0 if x == 0 else math.sin(x) / x
    k1p = k1 + nu1 * 2 * math.pi / dx
    s1 = sinc(k1p * dx / 2) ** (l + 1)
    s2 = sinc(k2 * dx / 2) ** (l + 1)
    tau1 = sinc(k1p * dx / 2) ** l * sinc(k1p * cdt)
    eta1 = (-1) ** nu1
    wdt2 = k1p * cdt / 2                       # omega' dt / 2 on the resonance
    if scheme == WT:
        s_b3 = math.cos(wdt2) * s1 * s2 * eta1  # s_{l,1} s_{l,2} tau_{l,3}(=1) eta1 eta2
        s_e2 = tau1 * s2
    else:
        s_b3 = math.cos(wdt2) * s1 * s2 * eta1
        s_e2 = s1 * s2
    xi0 = math.sin(k1p * cdt / 2) / (cdt / 2)  # dt = cdt with c = 1
    kb1 = math.sin(k1 * dx / 2) / (dx / 2)
    return s_b3 * xi0 - s_e2 * kb1


@pytest.mark.parametrize("l", [2, 3, 4])
def test_wt_removes_lowest_order_nci_any_dt(l):
    rng = np.random.default_rng(l)
    for cdt in (0.1, 0.25, 0.35, 0.6):
        for _ in range(20):
            k1 = rng.uniform(-math.pi, math.pi)
            k2 = rng.uniform(-math.pi, math.pi)
            for nu1 in (-2, -1, 0, 1, 2):
                assert abs(_nci_factor(WT, k1, nu1, k2, l, 1.0, cdt)) < 1e-12
    # MC cancels it only at c dt = dx/2
    k1, k2 = 1.1, 0.7
    assert abs(_nci_factor(MC, k1, 1, k2, l, 1.0, 0.5)) < 1e-12
    assert abs(_nci_factor(MC, k1, 1, k2, l, 1.0, 0.35)) > 1e-4


# ------------------------------------------------------------------------------------------
# Diagnostics: the energy normalisations agree with the equations of motion (App. E units)
# ------------------------------------------------------------------------------------------

def _langmuir(grid, dx, dt, wp, delta):
    """Neutral cold pair plasma on a quiet lattice (4 x 4 per cell and species); the electrons
    carry a velocity perturbation u_x = delta sin(k x) of the longest mode along x."""
    per = 16
    vc = dx[0] * dx[1]
    w = wp * wp * vc / per
    sub = (np.arange(4) + 0.5) / 4.0
    cx, cy, ox, oy = np.meshgrid(np.arange(grid[0]), np.arange(grid[1]), sub, sub, indexing="ij")
    x = np.vstack([((cx + ox) * dx[0]).ravel(), ((cy + oy) * dx[1]).ravel()])
    k = 2.0 * math.pi / (grid[0] * dx[0])
    ue = np.zeros((3, x.shape[1]))
    ue[0] = delta * np.sin(k * x[0])
    return x, ue, np.zeros_like(ue), w


def test_energy_exchange_keeps_total_energy():
    """A Langmuir oscillation moves energy between the particles, sum w m (gamma - 1), and the
    field, 1/2 sum (E^2 + B^2) V_c; with both normalised as the equations of motion imply, their
    sum stays constant to the leapfrog's phase offset (kinetic energy at t^(n-1/2), fields at
    t^n: O(omega dt) of the exchanged amount).  dx != 1 so that a missing cell volume shows."""
    grid, dx = (32, 2), (0.5, 0.5)
    wp, dt = 0.2, 0.1                      # omega_p dt = 0.02 per species
    x, ue, up, w = _langmuir(grid, dx, dt, wp, 0.01)
    s = oracle.Sim(grid, dx, dt, 2, MC)
    s.add_species(-1.0, 1.0, w, x, ue)
    s.add_species(1.0, 1.0, w, x, up)
    ke, fe = [], []
    for _ in range(220):                  # about two periods of sqrt(2) omega_p
        s.step(2)
        d = s.diag()
        ke.append(d["kinetic_energy"])
        fe.append(d["field_energy"])
    ke, fe = np.array(ke), np.array(fe)
    total = ke + fe
    swing = ke.max() - ke.min()
    assert fe.max() > 0.5 * ke.max()       # the energy does go into the field and back
    assert np.max(np.abs(total - total[0])) < 0.05 * swing
    s.close()


def test_langmuir_frequency_is_pair_plasma_frequency():
    """The same cold Langmuir mode oscillates at omega = sqrt(omega_pe^2 + omega_pp^2) =
    sqrt(2) omega_p (cold-fluid result, independent of k): the kinetic energy oscillates at twice
    that.  Measured from the zero crossings over about five periods; within 2% (the B-spline
    smoothing of the k dx = 0.2 mode and the leapfrog shift it by less than 1%).  A wrong charge,
    weight or cell-volume factor in the deposit or the gather moves it by sqrt of that factor."""
    grid, dx, dt, wp = (32, 2), (0.5, 0.5), 0.1, 0.2
    x, ue, up, w = _langmuir(grid, dx, dt, wp, 0.01)
    s = oracle.Sim(grid, dx, dt, 2, MC)
    s.add_species(-1.0, 1.0, w, x, ue)
    s.add_species(1.0, 1.0, w, x, up)
    ke = []
    for _ in range(560):
        s.step(2)
        ke.append(s.diag()["kinetic_energy"])
    s.close()
    ke = np.array(ke) - np.mean(ke)
    t = 2 * dt * (np.arange(len(ke)) + 1)
    idx = np.nonzero(np.diff(np.sign(ke)) != 0)[0]
    # linear interpolation of the crossings; consecutive crossings are half a period of ke apart
    tc = t[idx] - ke[idx] * (t[idx + 1] - t[idx]) / (ke[idx + 1] - ke[idx])
    half = np.mean(np.diff(tc))
    omega = 2 * math.pi / (2 * half) / 2      # ke oscillates at 2 omega
    assert abs(omega / (math.sqrt(2.0) * wp) - 1.0) < 0.02, omega


@pytest.mark.parametrize("scheme", [MC, WT])
@pytest.mark.parametrize("grid,dx", [((12, 10), (1.0, 0.8)), ((6, 7, 5), (1.0, 1.2, 0.9))])
def test_push_particle_in_uniform_fields(grid, dx, scheme):
    """Uniform E and B on every component's nodes: the interpolation weights sum to one (W_l and
    T_l alike), so the particle push sees exactly those fields -- the push equals the Boris
    rotation of the pinned routine followed by x += dt u/gamma, wrapped into the box."""
    dim = len(grid)
    dt, q, m = 0.3, -1.0, 1.0
    s = oracle.Sim(grid, dx, dt, 3, scheme)
    E = np.array([0.02, -0.05, 0.03])
    B = np.array([0.4, 0.1, -0.7])
    shape = (1,) + tuple(grid[::-1]) if dim == 2 else tuple(grid[::-1])
    for c in range(3):
        s.set_field(c, np.full(shape, E[c]))
        s.set_field(3 + c, np.full(shape, B[c]))
    rng = np.random.default_rng(9)
    L = np.array(grid, dtype=float) * np.array(dx)
    for _ in range(20):
        x = rng.uniform(0, 1, dim) * L
        u = rng.normal(0, 2, 3)
        xn, un = s.push_particle(q, m, x, u)
        ub = oracle.boris(q / m * dt, E, B, u)
        g = math.sqrt(1 + (ub ** 2).sum())
        xb = np.mod(x + dt * ub[:dim] / g, L)
        assert np.max(np.abs(un - ub)) < 1e-13 * max(1.0, np.max(np.abs(ub)))
        d = xn - xb
        d -= L * np.round(d / L)
        assert np.max(np.abs(d)) < 1e-12 * L.max()
    s.close()


@pytest.mark.parametrize("theta", [0.3, 1.0, 4.0])
def test_juttner_loader_matches_the_distribution(theta):
    """App. D, Eq. Maxwell-dist-relativistic, sampled with Sobol's method by the oracle: the
    co-moving |u| follows f(u) ~ u^2 exp(-sqrt(1 + u^2)/theta) (CDF at five sample quantiles
    against numerical integration), the mean Lorentz factor is the closed form
    3 theta + K1(1/theta)/K2(1/theta), and the directions are isotropic."""
    from scipy import integrate
    from scipy.special import kn
    n = 400000
    u = oracle.juttner_speeds(theta, n, seed=11)
    assert not np.isnan(u).any()
    g = np.sqrt(1.0 + u * u)
    expect = 3.0 * theta + kn(1, 1.0 / theta) / kn(2, 1.0 / theta)
    assert abs(g.mean() - expect) < 4.0 * g.std() / math.sqrt(n)
    f = lambda x: x * x * math.exp(-(math.sqrt(1.0 + x * x) - 1.0) / theta)
    z = integrate.quad(f, 0, np.inf, limit=200)[0]
    for q in (0.1, 0.25, 0.5, 0.75, 0.9):
        x = np.quantile(u, q)
        assert abs(integrate.quad(f, 0, x, limit=200)[0] / z - q) < 0.004
    # a full load at rest (gamma0 = 1: no boost, no flip): isotropic momenta whose magnitudes
    # are the sampler's speeds
    _, up, failed = oracle.load_drifting((32, 16), (1.0, 1.0), 32, 1.0, 0.0, theta=theta, seed=11)
    assert failed == 0
    m2 = (up ** 2).mean(axis=1)
    assert np.max(np.abs(m2 / m2.mean() - 1.0)) < 0.03
    sp = oracle.juttner_speeds(theta, up.shape[1], seed=11)
    assert np.max(np.abs(np.sqrt((up ** 2).sum(axis=0)) - sp)) <= 1e-12 * np.max(sp)


def test_juttner_attempt_bound():
    """The bounded Sobol loop: with a single attempt per particle the accepted fraction is the
    acceptance probability of one attempt, P(eta^2 - u^2 > 1), evaluated by quadrature from the
    method's own construction (below), and every particle left without an accepted attempt is
    marked rather than given a biased speed; the default bound leaves none at theta = 0.3."""
    from scipy import integrate
    theta, n = 0.3, 200000
    u = oracle.juttner_speeds(theta, n, seed=12, attempts=1)
    acc = np.isfinite(u)
    # one attempt proposes u ~ Gamma(3, theta) (density u^2 e^{-u/theta} / (2 theta^3)) and
    # accepts it with probability e^{-(sqrt(1+u^2) - u)/theta}; the accepted fraction is the
    # integral of their product
    f = lambda x: x * x * math.exp(-x / theta) / (2.0 * theta ** 3) \
        * math.exp(-(math.sqrt(1.0 + x * x) - x) / theta)
    p = integrate.quad(f, 0, np.inf, limit=200)[0]
    assert abs(acc.mean() - p) < 5.0 * math.sqrt(p * (1 - p) / n)
    assert np.all(u[acc] > 0.0)
    u = oracle.juttner_speeds(theta, n, seed=12)
    assert np.isfinite(u).all()


def test_threaded_particle_pass_equals_serial_pass():
    """The timing build's particle pass over host threads (private currents added at the end)
    gives the particles of the serial pass bit for bit and the same current up to the order of
    the final additions."""
    import plasma
    import workloads
    wl = plasma.fill(workloads.config_large(scale=16), count=20000)
    res = []
    for timing, threads in ((False, 1), (True, 4)):
        s = Sim(wl.grid[:2], wl.dx[:2], wl.dt, wl.l, wl.scheme, timing=timing)
        for sp in wl.species:
            s.add_species(sp.q, sp.m, sp.w, sp.x, sp.u)
        if timing:
            assert s.particle_pass_threads(0, 20000, threads) == threads
        else:
            s.particle_pass(0, 20000)
        res.append(([s.field(c) for c in (6, 7, 8)], [s.particles(i) for i in range(2)]))
        s.close()
    (ja, pa), (jb, pb) = res
    for a, b in zip(ja, jb):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))
    for (xa, ua), (xb, ub) in zip(pa, pb):
        assert np.array_equal(xa, xb) and np.array_equal(ua, ub)
