"""Asymptotic growth rate of the numerical Cherenkov instability (Sec. 2, Eq. NCI-Xu2013; App. A)
for an ultra-relativistic cold beam drifting along x1, evaluated with the interpolation tensors
of the MC scheme (Eq. shapeEB-org) or the WT scheme (Eq. shapeEB, Eq. tau_l), on a 2D grid
(k3 = 0, so only the (S_B3 xi_0 - S_E2 [k]_B1) term is present).

Host-side analysis (numpy); it needs no GPU and does not touch the simulation path.

Notation (c = 1):
  k'_1 = k_1 + nu_1 2 pi / dx_1 (aliasing order nu_1; nu_2 = nu_3 = 0), omega' = k'_1 on the
  beam resonance; s_{l,i} = sinc(k'_i dx_i / 2)^(l+1); tau_{l,i} = sinc(k'_i dx_i / 2)^l
  sinc(k'_i dt); eta_i = (-1)^nu_i; xi_0 = sin(k'_1 dt / 2) / (dt / 2); xi_1 = cos(k'_1 dt / 2);
  [k]_Bi = sin(k_i dx_i / 2) / (dx_i / 2); [k]_Ei = A_i [k]_Bi with A_i of Eq. Maxwell-A.
  S_J1 (not printed in the paper) is taken from the discrete continuity equation, which the
  Esirkepov deposit satisfies exactly: for charge deposited with W_l (S_rho = s_{l,1} s_{l,2})
  moving along x1, xi_0 S_rho = [k]_B1 S_J1, so S_J1 = S_rho xi_0 / [k]_B1.
"""
from __future__ import annotations

import math

import numpy as np

MC, WT = 0, 1
YEE, M4 = 0, 1


def _sinc(x):
    return np.sinc(np.asarray(x) / math.pi)  # sin(x) / x


def faraday_factor(solver: int, cdt: float, k1, k2, dx=(1.0, 1.0)):
    """A_1, A_2 of Eq. Maxwell-A (2D, k3 = 0): 1 for Yee; for M4 the App. C coefficients
    beta_ij = (c dt / dx_j)^2 / 12, delta_i = ((c dt / dx_i)^2 - 1) / 12."""
    if solver == YEE:
        one = np.ones(np.broadcast(k1, k2).shape)
        return one, one
    r1, r2 = cdt / dx[0], cdt / dx[1]
    b12, b21 = r2 * r2 / 12.0, r1 * r1 / 12.0
    d1, d2 = (r1 * r1 - 1.0) / 12.0, (r2 * r2 - 1.0) / 12.0
    c1, c2 = 1.0 - np.cos(k1 * dx[0]), 1.0 - np.cos(k2 * dx[1])
    return 1.0 - 2.0 * b12 * c2 - 2.0 * d1 * c1, 1.0 - 2.0 * b21 * c1 - 2.0 * d2 * c2


def lowest_order_factor(scheme: int, l: int, cdt: float, k1, k2, nu1: int, dx=(1.0, 1.0)):
    """S_B3 xi_0 - S_E2 [k]_B1 on the beam resonance (the factor App. A shows to vanish for WT)."""
    k1p = k1 + nu1 * 2.0 * math.pi / dx[0]
    s1 = _sinc(k1p * dx[0] / 2.0) ** (l + 1)
    s2 = _sinc(k2 * dx[1] / 2.0) ** (l + 1)
    tau1 = _sinc(k1p * dx[0] / 2.0) ** l * _sinc(k1p * cdt)
    eta1 = (-1.0) ** nu1
    xi0 = np.sin(k1p * cdt / 2.0) / (cdt / 2.0)
    xi1 = np.cos(k1p * cdt / 2.0)
    kb1 = np.sin(k1 * dx[0] / 2.0) / (dx[0] / 2.0)
    s_b3 = xi1 * s1 * s2 * eta1                       # tau_{l,3} = s_{l,3} = eta_3 = 1 in 2D
    s_e2 = (tau1 if scheme == WT else s1) * s2        # eta_2 = 1 (nu_2 = 0)
    return s_b3 * xi0 - s_e2 * kb1


def growth_rate(scheme: int, solver: int, l: int, cdt: float, k1, k2, nu1: int, omega_p: float,
                dx=(1.0, 1.0)):
    """Gamma of Eq. NCI-Xu2013 at (k1, k2) and aliasing order nu1 (2D: the k3 term is zero)."""
    k1 = np.asarray(k1, dtype=np.float64)
    k2 = np.asarray(k2, dtype=np.float64)
    k1p = k1 + nu1 * 2.0 * math.pi / dx[0]
    xi0 = np.sin(k1p * cdt / 2.0) / (cdt / 2.0)
    xi1 = np.cos(k1p * cdt / 2.0)
    kb1 = np.sin(k1 * dx[0] / 2.0) / (dx[0] / 2.0)
    kb2 = np.sin(k2 * dx[1] / 2.0) / (dx[1] / 2.0)
    _, a2 = faraday_factor(solver, cdt, k1, k2, dx)
    ke2 = a2 * kb2
    s_rho = _sinc(k1p * dx[0] / 2.0) ** (l + 1) * _sinc(k2 * dx[1] / 2.0) ** (l + 1)
    with np.errstate(divide="ignore", invalid="ignore"):
        s_j1 = s_rho * xi0 / kb1
        f = lowest_order_factor(scheme, l, cdt, k1, k2, nu1, dx)
        g = omega_p ** 2 * s_j1 * f * ke2 * k2 / (2.0 * xi0 ** 2 * xi1)
    return (math.sqrt(3.0) / 2.0) * np.cbrt(np.abs(g))


def max_growth_rate(scheme: int, solver: int, l: int, cdt: float, omega_p: float, n: int = 128,
                    nus=(-2, -1, 1, 2), dx=(1.0, 1.0)):
    """Largest Gamma over a cell-centred n x n sample of the Brillouin zone (k1 = 0 excluded by
    the centring) and the aliasing orders nus; returns (Gamma, k1, k2, nu1)."""
    h = 2.0 * math.pi / n
    k = -math.pi + h * (np.arange(n) + 0.5)
    K1, K2 = np.meshgrid(k / dx[0], k / dx[1], indexing="ij")
    best = (0.0, 0.0, 0.0, 0)
    for nu in nus:
        g = growth_rate(scheme, solver, l, cdt, K1, K2, nu, omega_p, dx)
        g = np.where(np.isfinite(g), g, 0.0)
        i = np.unravel_index(np.argmax(g), g.shape)
        if g[i] > best[0]:
            best = (float(g[i]), float(K1[i]), float(K2[i]), nu)
    return best
