"""Seeded synthetic workloads: the drifting pair plasma of the paper's Table 1, at the sizes of
the benchmark configurations.  Shared by the oracle tests, the CUDA tests and the benchmark.

This module holds no arithmetic of the PIC step.  It draws counter-based random numbers
(SplitMix64, Steele/Lea/Flood 2014: state += 0x9E3779B97F4A7C15, then the xor-shift-multiply
finaliser) and turns them into an initial particle state:

* positions: ppc/2 particles of each species per cell at uniform in-cell offsets (stratified
  per cell; independent per species, or with colocated=True the positrons on the electrons'
  positions, a neutral start);
* momenta: cold beam u = (sqrt(gamma^2 - 1), 0, 0), or a drifting Maxwellian loaded as in the
  paper's App. D -- Gaussian u' ~ N(0, u_th^2) per component in the co-moving frame
  (Box-Muller), the flip of u'_x that accounts for the volume transform (flip when the extra
  uniform X1 exceeds (1 + beta v'_x)/2, the reading under which the loaded density is
  proportional to 1 + beta v'_x as App. D requires), then the Lorentz boost along x1.

Tensors are torch float64 so the same code produces a small case on the CPU for the oracle and
a 134M-particle case directly on the GPU for the benchmark.  The integer stream is identical on
both; the Box-Muller log/cos/sqrt may differ in the last bit between devices, so a parity test
always hands the oracle and the CUDA path the very same arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import torch

BASE_SEED = 1909096130

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1


def _s64(v: int) -> int:
    """Reinterpret a 64-bit unsigned constant as a signed int64 (torch has no uint64 math)."""
    v &= _MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 lanes."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _s64(_M1)
    z = (z ^ _srl(z, 27)) * _s64(_M2)
    return z ^ _srl(z, 31)


def _mix_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, *ids: int) -> int:
    """A 64-bit key for one random stream, derived from the seed and stream ids."""
    k = _mix_int(seed + _GOLDEN)
    for i in ids:
        k = _mix_int(k ^ ((i + 1) * _GOLDEN))
    return k


def uniform(key: int, counter: torch.Tensor) -> torch.Tensor:
    """U[0,1) doubles: 53 high bits of SplitMix64 at position `counter` of stream `key`."""
    z = counter.to(torch.int64) * _s64(_GOLDEN) + _s64(key)
    z = _mix(z)
    return _srl(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def normal(key_a: int, key_b: int, counter: torch.Tensor) -> torch.Tensor:
    """Standard normal by Box-Muller from two independent uniform streams."""
    u1 = 1.0 - uniform(key_a, counter)  # (0, 1]
    u2 = uniform(key_b, counter)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


JUTTNER_ATTEMPTS = 128


def juttner_speeds(theta: float, key_x: Sequence[int], counter: torch.Tensor) -> torch.Tensor:
    """|u'| of the Juttner-Synge distribution f(u) ~ u^2 exp(-sqrt(1 + u^2)/theta) (App. D) by
    Sobol's rejection method: u = -theta ln(X1 X2 X3), eta = -theta ln(X1 X2 X3 X4), accepted
    when eta^2 - u^2 > 1.  Attempt a of particle p draws its four uniforms at counter
    p * JUTTNER_ATTEMPTS + a of the streams key_x[0..3]; the first accepted attempt is taken.
    Particles with no accepted attempt among JUTTNER_ATTEMPTS get NaN (theta >= 0.3 makes that
    a ~1e-14 event per particle)."""
    n = counter.numel()
    out = torch.full((n,), float("nan"), dtype=torch.float64, device=counter.device)
    todo = torch.ones(n, dtype=torch.bool, device=counter.device)
    base = counter.to(torch.int64) * JUTTNER_ATTEMPTS
    for a in range(JUTTNER_ATTEMPTS):
        idx = torch.nonzero(todo).flatten()
        if idx.numel() == 0:
            break
        c = base[idx] + a
        x = [1.0 - uniform(key_x[j], c) for j in range(4)]   # (0, 1]
        p3 = x[0] * x[1] * x[2]
        u = -theta * torch.log(p3)
        eta = -theta * torch.log(p3 * x[3])
        ok = eta * eta - u * u > 1.0
        out[idx[ok]] = u[ok]
        todo[idx[ok]] = False
    return out


@dataclass
class Species:
    q: float
    m: float
    w: float
    x: torch.Tensor  # (dim, n) physical positions
    u: torch.Tensor  # (3, n) u = gamma v


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
    species: List[Species] = field(default_factory=list)

    @property
    def dim(self) -> int:
        return 3 if self.grid[2] > 1 else 2

    @property
    def n_particles(self) -> int:
        return sum(int(s.x.shape[1]) for s in self.species)

    @property
    def ncell(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]


def pair_plasma(grid: Sequence[int], dx: Sequence[float], dt: float, l: int, scheme: int,
                gamma: float, u_th: float, ppc: int, omega_p: Optional[float] = None,
                seed: int = BASE_SEED, run: int = 0, device="cpu", steps: int = 0,
                name: str = "pair_plasma", colocated: bool = False,
                theta: Optional[float] = None) -> Workload:
    """Drifting e-/e+ pair plasma along x1 (Table 1 set-up), ppc particles per cell in total.

    omega_p is the relativistic plasma frequency of each species, omega_p^2 = n q^2/(gamma m)
    with n = (ppc/2) w / V_c (Sec. 4 normalisation); when omitted the grid resolves the skin
    depth with 16 cells, c/omega_p = 16 dx, as in Table 1 (16 d_e over 256 cells).

    colocated: the positrons start at the electrons' positions (a neutral start: rho = 0, so
    zero initial fields satisfy Gauss's law); momenta stay independent.  Otherwise every
    species draws its own positions.

    theta: when given, the co-moving momenta follow the Juttner-Synge distribution of
    temperature theta = kT / mc^2 (App. D, Sobol's method; isotropic directions), instead of
    the Gaussian of spread u_th.
    """
    grid = tuple(int(g) for g in grid) + (1,) * (3 - len(grid))
    dx = tuple(float(d) for d in dx) + (1.0,) * (3 - len(dx))
    dim = 3 if grid[2] > 1 else 2
    if ppc % 2:
        raise ValueError("ppc counts both species and must be even")
    per = ppc // 2
    ncell = grid[0] * grid[1] * grid[2]
    n = ncell * per
    vc = dx[0] * dx[1] * (dx[2] if dim == 3 else 1.0)
    if omega_p is None:
        omega_p = 1.0 / (16.0 * dx[0])
    w = omega_p * omega_p * gamma * vc / per
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    idx = torch.arange(n, dtype=torch.int64, device=device)
    cell = idx // per
    ci = [cell % grid[0], (cell // grid[0]) % grid[1], cell // (grid[0] * grid[1])]
    species = []
    for s, q in enumerate((-1.0, 1.0)):
        xs = []
        for a in range(dim):
            off = uniform(stream_key(seed, run, 0 if colocated else s, 10 + a), idx)
            L = grid[a] * dx[a]
            xa = (ci[a].to(torch.float64) + off) * dx[a]
            xa = torch.where(xa >= L, xa - L, xa)
            xs.append(xa)
        x = torch.stack(xs)
        if theta is not None or u_th > 0.0:
            if theta is not None:
                um = juttner_speeds(theta, [stream_key(seed, run, s, 40 + j) for j in range(4)], idx)
                x5 = uniform(stream_key(seed, run, s, 44), idx)
                x6 = uniform(stream_key(seed, run, s, 45), idx)
                ct = 2.0 * x5 - 1.0
                st = 2.0 * torch.sqrt(x5 * (1.0 - x5))
                ph = 2.0 * math.pi * x6
                up = torch.stack([um * ct, um * st * torch.cos(ph), um * st * torch.sin(ph)])
            else:
                up = torch.stack([u_th * normal(stream_key(seed, run, s, 20 + 2 * a),
                                                stream_key(seed, run, s, 21 + 2 * a), idx)
                                  for a in range(3)])
            e_prime = torch.sqrt(1.0 + (up * up).sum(0))
            x1 = uniform(stream_key(seed, run, s, 30), idx)
            flip = x1 > 0.5 * (1.0 + beta * up[0] / e_prime)
            upx = torch.where(flip, -up[0], up[0])
            ux = gamma * (upx + beta * e_prime)
            u = torch.stack([ux, up[1], up[2]])
        else:
            u = torch.zeros(3, n, dtype=torch.float64, device=device)
            u[0] = math.sqrt(gamma * gamma - 1.0)
        species.append(Species(q=q, m=1.0, w=w, x=x, u=u))
    return Workload(name=name, grid=grid, dx=dx, dt=dt, l=l, scheme=scheme, gamma=gamma,
                    u_th=u_th, ppc=ppc, omega_p=omega_p, steps=steps, species=species)


# --- the benchmark configurations ----------------------------------------------------------

def config_small(scheme: int = 1, device="cpu", seed: int = BASE_SEED) -> Workload:
    """64x32, dx = 1, c dt = 0.35, quadratic, cold pair plasma at gamma = 20, 4 ppc,
    omega_p dt = 0.05, 200 steps (the parity and NCI case)."""
    dt = 0.35
    return pair_plasma((64, 32), (1.0, 1.0), dt, 2, scheme, 20.0, 0.0, 4, omega_p=0.05 / dt,
                       seed=seed, device=device, steps=200, name="pair_64x32_l2_cold_g20_ppc4")


def config_large(scheme: int = 1, device="cpu", seed: int = BASE_SEED, scale: int = 1) -> Workload:
    """2048x1024, cubic, gamma = 50, u_th = 0.01, 64 ppc (134,217,728 particles), c dt = 0.25,
    1000 steps.  `scale` divides both grid extents (for reduced-size parity runs)."""
    nx, ny = 2048 // scale, 1024 // scale
    return pair_plasma((nx, ny), (1.0, 1.0), 0.25, 3, scheme, 50.0, 0.01, 64, seed=seed,
                       device=device, steps=1000,
                       name="pair_%dx%d_l3_g50_uth0.01_ppc64" % (nx, ny))


def batched_runs(n_runs: int = 256, seed: int = BASE_SEED, max_nx: int = 512):
    """Parameters of the uneven batch: grids 64x32 .. 512x256, 4..32 ppc, l in {2,3}, c dt/dx
    uniform on [0.1, 0.7], gamma log-uniform on [10, 100], u_th = 0.01, WT, 500 steps."""
    key = stream_key(seed, 7777)
    runs = []
    for r in range(n_runs):
        c = torch.arange(6, dtype=torch.int64) + 6 * r
        v = uniform(key, c).tolist()
        choices = [n for n in (64, 128, 256, 512) if n <= max_nx]
        nx = choices[min(int(v[0] * len(choices)), len(choices) - 1)]
        ppc = (4, 8, 16, 32)[min(int(v[1] * 4), 3)]
        l = (2, 3)[min(int(v[2] * 2), 1)]
        cdt = 0.1 + 0.6 * v[3]
        gamma = 10.0 ** (1.0 + v[4])
        runs.append(dict(grid=(nx, nx // 2, 1), dx=(1.0, 1.0, 1.0), dt=cdt, l=l, scheme=1,
                         gamma=gamma, u_th=0.01, ppc=ppc, steps=500, run=r))
    return runs
