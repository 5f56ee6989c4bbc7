"""The NCI growth-rate evaluator (paper_1909_09613_gb300/nci.py, Eq. NCI-Xu2013) against what
Sec. 2 and App. A fix: the WT factor vanishes for every wavenumber, aliasing order, dt and
Faraday stencil; WT equals MC at c dt = dx/2, where the MC rate vanishes too; off that step MC
is unstable.  Also cross-checked against the independent factor of the App. A pin."""
import math

import numpy as np
import pytest

from paper_1909_09613_gb300 import nci

WP = 1.0 / 16.0


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_wt_factor_vanishes_everywhere(l):
    rng = np.random.default_rng(100 + l)
    k1 = rng.uniform(-math.pi, math.pi, 4000)
    k2 = rng.uniform(-math.pi, math.pi, 4000)
    for cdt in (0.05, 0.2, 0.35, 0.5, 0.65):
        for nu in (-2, -1, 0, 1, 2):
            f_wt = nci.lowest_order_factor(nci.WT, l, cdt, k1, k2, nu)
            f_mc = nci.lowest_order_factor(nci.MC, l, cdt, k1, k2, nu)
            assert np.max(np.abs(f_wt)) < 1e-14
            if cdt == 0.5:
                assert np.max(np.abs(f_mc)) < 1e-14
            elif nu != 0:
                assert np.max(np.abs(f_mc)) > 1e-6


def test_factor_matches_independent_app_a_pin():
    import test_oracle_pins as pins  # the App. A pin's own evaluation of the same factor
    rng = np.random.default_rng(7)
    for _ in range(50):
        k1, k2 = rng.uniform(-math.pi, math.pi, 2)
        for scheme in (nci.MC, nci.WT):
            for l in (2, 4):
                for nu in (-1, 1, 2):
                    cdt = float(rng.uniform(0.05, 0.7))
                    a = float(nci.lowest_order_factor(scheme, l, cdt, k1, k2, nu))
                    b = pins._nci_factor(scheme, k1, nu, k2, l, 1.0, cdt)
                    assert abs(a - b) <= 1e-13 * max(1.0, abs(b))


@pytest.mark.parametrize("solver", [nci.YEE, nci.M4])
def test_growth_rates_wt_zero_mc_depends_on_dt(solver):
    ratios = (0.1, 0.3, 0.5, 0.7)
    g_mc = [nci.max_growth_rate(nci.MC, solver, 4, r / math.sqrt(2.0), WP, n=96)[0] for r in ratios]
    g_wt = [nci.max_growth_rate(nci.WT, solver, 4, r / math.sqrt(2.0), WP, n=96)[0] for r in ratios]
    g_half = nci.max_growth_rate(nci.MC, solver, 4, 0.5, WP, n=96)[0]
    # WT: zero up to the cube root of round-off; MC: finite, vanishing at c dt = dx/2
    assert max(g_wt) < 1e-4 * min(g_mc)
    assert g_half < 1e-4 * min(g_mc)
    # MC weakens as dt approaches dx / (2 c) (the order the Table 1 runs show)
    assert g_mc[0] >= g_mc[1] >= g_mc[2] > g_mc[3] > 0.0
    # the M4 stencil enters only through [k]_E2: A_2 = 1 at k = 0
    a1, a2 = nci.faraday_factor(solver, 0.3, np.array([0.0]), np.array([0.0]))
    assert abs(a1[0] - 1.0) < 1e-15 and abs(a2[0] - 1.0) < 1e-15


def test_m4_factor_matches_app_c_dispersion():
    """A_i of the M4 coefficients makes the App. C dispersion relation fourth-order accurate:
    s_w^2 = sum s_i^2 A_i with omega = c |k| leaves an O(k^6) residual (dx = 1)."""
    cdt = 0.4
    errs = []
    for h in (0.2, 0.1):
        k1, k2 = h * 0.8, h * 0.6
        a1, a2 = nci.faraday_factor(nci.M4, cdt, k1, k2)
        s1, s2 = math.sin(k1 / 2) ** 2, math.sin(k2 / 2) ** 2
        lhs = math.sin(h * cdt / 2) ** 2 / cdt ** 2
        errs.append(abs(lhs - (s1 * a1 + s2 * a2)))
    assert errs[0] / errs[1] > 40.0  # ~2^6
