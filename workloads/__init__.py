"""Seeded synthetic workloads: the parameters of the drifting pair plasma of the paper's Table 1
at the sizes of the benchmark configurations.  Shared by the tests and the benchmark.

This module holds no arithmetic of the method.  It names each configuration (grid, cell size,
time step, spline order, scheme, drift gamma, co-moving spread u_th or temperature theta,
particles per cell, seed and random stream) and the constants of its two species: charge
-1 / +1, mass 1, and the macro-particle weight that gives the configuration's plasma frequency,
omega_p^2 = n q^2 / (gamma m) with n = (ppc / 2) w / V_c (when omega_p is not given, the grid
resolves the skin depth with 16 cells, c / omega_p = 16 dx, as in Table 1: 16 d_e over 256
cells).  Each species holds ppc / 2 particles in every cell.

The particles themselves are drawn by a loader that follows App. D from these parameters and
one counter-based generator (SplitMix64, Steele/Lea/Flood 2014; stream ids documented in
include/pic.h): the library's device loader (pic_load_drifting_plasma / _juttner) in the
product and the benchmark, the FP64 oracle's loader (oracle.load_drifting) in the tests.  The
two implement the generator each from its published definition, so they draw the same numbers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

BASE_SEED = 1909096130

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1


def _mix(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, *ids: int) -> int:
    """A 64-bit key for one random stream, derived from the seed and stream ids."""
    k = _mix(seed + _GOLDEN)
    for i in ids:
        k = _mix(k ^ ((i + 1) * _GOLDEN))
    return k


def uniform(key: int, counter: int) -> float:
    """U[0,1): 53 high bits of SplitMix64 at position `counter` of stream `key`."""
    return (_mix(counter * _GOLDEN + key) >> 11) * (1.0 / 9007199254740992.0)


@dataclass
class Species:
    q: float
    m: float
    w: float
    per_cell: int          # particles in every cell
    pos_species: int       # species whose positions this one takes (itself, or 0: neutral start)
    x: Optional[object] = None  # (dim, n) physical positions, once a loader has drawn them
    u: Optional[object] = None  # (3, n) u = gamma v


@dataclass
class Workload:
    name: str
    grid: tuple          # (nx, ny, nz), nz = 1 for 2D
    dx: tuple            # (dx, dy, dz)
    dt: float
    l: int
    scheme: int          # 0 = MC, 1 = WT
    gamma: float
    u_th: float
    ppc: int             # both species together
    omega_p: float
    steps: int
    seed: int = BASE_SEED
    run: int = 0         # random stream of this plasma
    theta: float = 0.0   # > 0: Juttner-Synge co-moving momenta of temperature theta
    species: List[Species] = field(default_factory=list)

    @property
    def dim(self) -> int:
        return 3 if self.grid[2] > 1 else 2

    @property
    def ncell(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def n_particles(self) -> int:
        return sum(self.ncell * s.per_cell for s in self.species)


def pair_plasma(grid: Sequence[int], dx: Sequence[float], dt: float, l: int, scheme: int,
                gamma: float, u_th: float, ppc: int, omega_p: Optional[float] = None,
                seed: int = BASE_SEED, run: int = 0, steps: int = 0,
                name: str = "pair_plasma", colocated: bool = False,
                theta: Optional[float] = None) -> Workload:
    """Drifting e-/e+ pair plasma along x1 (Table 1 set-up), ppc particles per cell in total.

    colocated: the positrons take the electrons' positions (a neutral start: rho = 0, so zero
    initial fields satisfy Gauss's law); momenta stay independent.  Otherwise every species
    draws its own positions.  theta: Juttner-Synge co-moving momenta of that temperature
    instead of the Gaussian of spread u_th."""
    grid = tuple(int(g) for g in grid) + (1,) * (3 - len(grid))
    dx = tuple(float(d) for d in dx) + (1.0,) * (3 - len(dx))
    dim = 3 if grid[2] > 1 else 2
    if ppc % 2:
        raise ValueError("ppc counts both species and must be even")
    per = ppc // 2
    vc = dx[0] * dx[1] * (dx[2] if dim == 3 else 1.0)
    if omega_p is None:
        omega_p = 1.0 / (16.0 * dx[0])
    w = omega_p * omega_p * gamma * vc / per if per > 0 else 0.0
    species = [Species(q=q, m=1.0, w=w, per_cell=per, pos_species=0 if colocated else s)
               for s, q in enumerate((-1.0, 1.0))]
    return Workload(name=name, grid=grid, dx=dx, dt=dt, l=l, scheme=scheme, gamma=gamma,
                    u_th=u_th, ppc=ppc, omega_p=omega_p, steps=steps, seed=seed, run=run,
                    theta=float(theta or 0.0), species=species)


# --- the benchmark configurations ----------------------------------------------------------

def config_small(scheme: int = 1, seed: int = BASE_SEED) -> Workload:
    """64x32, dx = 1, c dt = 0.35, quadratic, cold pair plasma at gamma = 20, 4 ppc,
    omega_p dt = 0.05, 200 steps (the parity and NCI case)."""
    dt = 0.35
    return pair_plasma((64, 32), (1.0, 1.0), dt, 2, scheme, 20.0, 0.0, 4, omega_p=0.05 / dt,
                       seed=seed, steps=200, name="pair_64x32_l2_cold_g20_ppc4")


def config_large(scheme: int = 1, seed: int = BASE_SEED, scale: int = 1) -> Workload:
    """2048x1024, cubic, gamma = 50, u_th = 0.01, 64 ppc (134,217,728 particles), c dt = 0.25,
    1000 steps.  `scale` divides both grid extents (a section of the same plasma, for
    reduced-size parity runs)."""
    nx, ny = 2048 // scale, 1024 // scale
    return pair_plasma((nx, ny), (1.0, 1.0), 0.25, 3, scheme, 50.0, 0.01, 64, seed=seed,
                       steps=1000, name="pair_%dx%d_l3_g50_uth0.01_ppc64" % (nx, ny))


def batched_runs(n_runs: int = 256, seed: int = BASE_SEED, max_nx: int = 512):
    """Parameters of the uneven batch: grids 64x32 .. 512x256, 4..32 ppc, l in {2,3}, c dt/dx
    uniform on [0.1, 0.7], gamma log-uniform on [10, 100], u_th = 0.01, WT, 500 steps."""
    key = stream_key(seed, 7777)
    runs = []
    for r in range(n_runs):
        v = [uniform(key, 6 * r + c) for c in range(6)]
        choices = [n for n in (64, 128, 256, 512) if n <= max_nx]
        nx = choices[min(int(v[0] * len(choices)), len(choices) - 1)]
        ppc = (4, 8, 16, 32)[min(int(v[1] * 4), 3)]
        l = (2, 3)[min(int(v[2] * 2), 1)]
        cdt = 0.1 + 0.6 * v[3]
        gamma = 10.0 ** (1.0 + v[4])
        runs.append(dict(grid=(nx, nx // 2, 1), dx=(1.0, 1.0, 1.0), dt=cdt, l=l, scheme=1,
                         gamma=gamma, u_th=0.01, ppc=ppc, steps=500, run=r))
    return runs


def served_requests(n_req: int = 48, seed: int = BASE_SEED, frac_3d: float = 0.1,
                    sizes_3d=((128, 32, 32), (256, 64, 64), (512, 128, 128)), steps: int = 500):
    """Parameters of the served stream: 90% from the batched distribution, 10% 3D runs (drift
    along x1, 8 particles per cell, quadratic, c dt = 0.4), in arrival order.  Arrival times
    are drawn by the caller from the measured service capacity."""
    key = stream_key(seed, 8888)
    base = batched_runs(n_req, seed=seed + 5)
    out = []
    for i, sp in enumerate(base):
        if uniform(key, 2 * i) < frac_3d:
            g = sizes_3d[min(int(uniform(key, 2 * i + 1) * len(sizes_3d)), len(sizes_3d) - 1)]
            out.append(dict(grid=g, dx=(1.0, 1.0, 1.0), dt=0.4, l=2, scheme=1,
                            gamma=sp["gamma"], u_th=0.01, ppc=8, steps=steps, run=i))
        else:
            out.append(dict(sp, steps=steps, run=i))
    return out
