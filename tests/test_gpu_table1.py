"""The drifting pair-plasma NCI test of Table 1 (256x128 cells, 64 particles per cell,
gamma0 = 1000, kT = 0.01, quartic splines), served as NCI-scan requests that record E/E0 (field
energy over the initial kinetic energy, Sec. 4), run to t = 40 / omega_pe from a neutral start.

What Sec. 4 and App. A fix for this set-up:
  * MC4 with the Yee solver at dt = 0.3 dt_CFL is unstable (NCI), its field energy grows by orders
    of magnitude within tens of 1/omega_pe;
  * WT4 at the same dt suppresses it: E/E0 stays at the noise level;
  * at c dt = dx / 2 (dt = dt_CFL / sqrt 2) WT4 is MC4 (Eq. tau_l: T_l = W_l there).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1909_09613_gb300 as pic  # noqa: E402
from paper_1909_09613_gb300 import engine  # noqa: E402

MC, WT = pic.PIC_SCHEME_MC, pic.PIC_SCHEME_WT
YEE = pic.PIC_SOLVER_YEE


def _ratio(served):
    h = np.array(served.history)  # step, t, U_EM, K
    return h[:, 1], h[:, 2] / h[0, 3]


def test_table1_short_scan_wt_suppresses_nci():
    only = {(MC, YEE, 1), (WT, YEE, 1), (MC, YEE, 4), (WT, YEE, 4)}
    reqs = engine.table1_requests(40.0, 2.0, only=only)
    assert len(reqs) == 4
    res = {r.rid: r for r in engine.Server(chunk=64).serve(reqs)}
    out = {}
    for q in reqs:
        s = res[q.rid]
        assert s.diag["error_flags"] == 0
        assert s.history[-1][0] == q.steps
        out[(q.scheme, round(q.dt, 4))] = _ratio(s)
    t_mc, e_mc = out[(MC, 0.2121)]
    t_wt, e_wt = out[(WT, 0.2121)]
    print("E/E0 at t=40: MC4 %.3e WT4 %.3e" % (e_mc[-1], e_wt[-1]))
    assert e_mc[-1] > 1e-2            # NCI under MC4
    assert np.max(e_wt) < 1e-5        # suppressed under WT4
    assert e_mc[-1] > 1e3 * e_wt[-1]
    # dt = dt_CFL / sqrt 2: the two schemes coincide
    _, a = out[(MC, 0.5)]
    _, b = out[(WT, 0.5)]
    assert np.max(np.abs(a[1:] - b[1:]) / b[1:]) < 1e-3


def test_table1_fp32_matches_fp64_at_gamma_1000():
    """The precision form in the Table 1 regime (gamma0 = 1000, kT = 0.01, quartic): E/E0 of
    the FP32 form against the plain FP64 form over 40 / omega_pe on a 128x64 section (32 per
    cell), for the unstable MC4 run and the suppressed WT4 run (same seeded plasma)."""
    only = {(MC, YEE, 1), (WT, YEE, 1)}
    out = {}
    for prec in (pic.PIC_FP64, pic.PIC_FP32_MIXED):
        reqs = engine.table1_requests(40.0, 2.0, only=only, grid=(128, 64, 1), ppc=32,
                                      precision=prec)
        for s, q in zip(sorted(engine.Server(chunk=64).serve(reqs), key=lambda r: r.rid), reqs):
            out[(prec, q.scheme)] = _ratio(s)[1]
    for scheme in (MC, WT):
        a, b = out[(pic.PIC_FP32_MIXED, scheme)], out[(pic.PIC_FP64, scheme)]
        err = np.max(np.abs(a[1:] - b[1:]) / b[1:])
        print("scheme", scheme, "max relative E/E0 difference FP32 vs FP64: %.2e" % err)
        assert err < 1e-2
    assert out[(pic.PIC_FP64, MC)][-1] > 1e2 * out[(pic.PIC_FP64, WT)][-1]
