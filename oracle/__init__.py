"""FP64 CPU oracle of the WT-scheme PIC step (arXiv:1909.09613) -- test infrastructure.

This package is the slow, plain, obviously-correct reference that the CUDA library is checked
against.  It is written from the paper (Sec. 2 for W_l, T_l and the WT gather of
Eq. interpolation-EB-real-mod; Sec. 1 for Boris, Esirkepov and Yee; App. B for Gauss's law;
App. D for loading a drifting plasma; App. E for the dimensionless equations) and shares no
code with the CUDA path.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.

The arithmetic lives in ``pic_oracle.c`` (plain C99, IEEE binary64, compiled with
``-ffp-contract=off``); this module only compiles it with gcc and marshals arrays through ctypes.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  W            closed forms, partition of unity, unit integral, convolution recurrence
  T            the paper's printed T_1..T_4, T_l(1/2) = W_l, partition of unity,
               dtt -> 0 limit, numerical Fourier transform = tau_l
  gather       brute force over all nodes; WT = MC at c dt = dx/2; Fourier symbol of every
               component (Eq. shapeEB); App. B self-force with transverse T
  boris        gyration angle and |u| conservation; E x B drift
  deposit      discrete continuity on every node; 1-D motion; static J_z closed form
  yee, M4      vacuum dispersion relation of App. C (A_i = 1 and the M4 A_i); fourth-order
               phase error of M4; Gauss's law conservation
  tile_sort    brute-force order check on small inputs
  load_drifting  App. D: the drift moment with and without the flip, the Juttner-Synge
               distribution (mean gamma, CDF, isotropy), the cold beam, the attempt bound
  step         composition of the above, brute-force tiny runs (whole-step parity has no
               printed worked example in the paper)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_LIB_TIMING = os.path.join(_LIBDIR, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_timing = None

MC, WT = 0, 1
YEE, M4 = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False, timing: bool = False) -> str:
    """Compile pic_oracle.c into oracle/_lib/liboracle.so (plain gcc, no CUDA): the parity build,
    -O2 with no fused multiply-add, single-threaded.  timing=True builds liboracle_omp.so, the
    same source at -O3 with OpenMP over particles (orc_particle_pass_threads), for the timed
    CPU baseline only."""
    os.makedirs(_LIBDIR, exist_ok=True)
    out = _LIB_TIMING if timing else _LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    opt = ["-O3", "-fopenmp"] if timing else ["-O2"]
    cmd = ["gcc"] + opt + ["-ffp-contract=off", "-std=c99", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def _load(timing: bool = False):
    global _lib, _lib_timing
    with _lock:
        if not timing and _lib is not None:
            return _lib
        if timing and _lib_timing is not None:
            return _lib_timing
        lib = ctypes.CDLL(build(timing=timing))
        lib.orc_W.restype = ctypes.c_double
        lib.orc_W.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.orc_T.restype = ctypes.c_double
        lib.orc_T.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.orc_T_paper.restype = ctypes.c_double
        lib.orc_T_paper.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [ctypes.c_int] * 2
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_add_species.restype = ctypes.c_int
        lib.orc_add_species.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_long, _dp, _dp]
        lib.orc_set_field.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        lib.orc_get_field.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        lib.orc_get_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp]
        lib.orc_set_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp]
        lib.orc_step_count.restype = ctypes.c_long
        lib.orc_step_count.argtypes = [ctypes.c_void_p]
        lib.orc_gather.argtypes = [ctypes.c_void_p, _dp, _dp]
        lib.orc_gather_brute.argtypes = [ctypes.c_void_p, _dp, _dp]
        lib.orc_boris.argtypes = [ctypes.c_double, _dp, _dp, _dp]
        lib.orc_deposit.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, _dp, _dp]
        lib.orc_rho.argtypes = [ctypes.c_void_p, _dp]
        lib.orc_yee_b.argtypes = [ctypes.c_void_p, ctypes.c_double]
        lib.orc_set_solver.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_yee_e.argtypes = [ctypes.c_void_p]
        lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.orc_push_particle.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _dp, _dp]
        lib.orc_particle_pass.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_long]
        lib.orc_diag.argtypes = [ctypes.c_void_p, _dp]
        lib.orc_gauss_residual.argtypes = [ctypes.c_void_p, _dp]
        lib.orc_tile_sort.restype = ctypes.c_long
        lib.orc_tile_sort.argtypes = [_ip, _ip, ctypes.c_int, ctypes.c_long, _lp, _lp, _lp]
        lib.orc_load_drifting.restype = ctypes.c_long
        lib.orc_load_drifting.argtypes = [ctypes.c_int, _ip, _dp, ctypes.c_long, ctypes.c_long,
                                          ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_ulonglong, ctypes.c_ulonglong,
                                          ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.orc_juttner_speeds.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_ulonglong,
                                           ctypes.c_ulonglong, ctypes.c_int, ctypes.c_long,
                                           ctypes.c_long, _dp]
        lib.orc_particle_pass_threads.restype = ctypes.c_int
        lib.orc_particle_pass_threads.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_long,
                                                  ctypes.c_int]
        if timing:
            _lib_timing = lib
        else:
            _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(_dp)


def W(l: int, x: float) -> float:
    """B-spline W_l(x), x in cell units (Sec. 2, Eq. shape-real)."""
    return _load().orc_W(int(l), float(x))


def T(l: int, dtt: float, x: float) -> float:
    """T_l(x; dtt) as the box average of W_{l-1} over [x - dtt, x + dtt] (Sec. 2, Eq. tau_l)."""
    return _load().orc_T(int(l), float(dtt), float(x))


def T_paper(l: int, dtt: float, x: float) -> float:
    """The paper's printed T_1..T_4 closed forms (Sec. 2), valid for dtt <= 1/2."""
    return _load().orc_T_paper(int(l), float(dtt), float(x))


def boris(qmdt: float, E, B, u) -> np.ndarray:
    """One relativistic Boris rotation u^{n-1/2} -> u^{n+1/2} (Sec. 1; App. E equations)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    out = np.array(u, dtype=np.float64)
    _load().orc_boris(float(qmdt), _d(E), _d(B), _d(out))
    return out


CELL_MAJOR, SLOT_MAJOR = 0, 1


def tile_sort(grid, tile, cells, order=CELL_MAJOR):
    """Reference tile-sort order; returns (perm, tile_start).
    CELL_MAJOR: (tile, cell-in-tile, slot); SLOT_MAJOR: (tile, slot, cell-in-tile), where slot
    is the particle's rank inside its cell in input order."""
    lib = _load()
    n = np.array(list(grid) + [1] * (3 - len(grid)), dtype=np.int32)
    t = np.array(list(tile) + [1] * (3 - len(tile)), dtype=np.int32)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    ntiles = int(np.prod((n.astype(np.int64) + t - 1) // t))
    perm = np.zeros(max(len(cells), 1), dtype=np.int64)
    ts = np.zeros(ntiles + 1, dtype=np.int64)
    lib.orc_tile_sort(n.ctypes.data_as(_ip), t.ctypes.data_as(_ip), int(order), len(cells),
                      cells.ctypes.data_as(_lp), perm.ctypes.data_as(_lp), ts.ctypes.data_as(_lp))
    return perm[:len(cells)], ts


def load_drifting(grid, dx, per_cell, gamma, u_th=0.0, theta=0.0, seed=0, run=0, species=0,
                  pos_species=None, first=0, count=None):
    """Particles first .. first + count - 1 of one species of the App. D drifting plasma along
    x1 (per_cell per cell, cells x1-fastest; Gaussian co-moving momenta of spread u_th, or
    Juttner-Synge ones of temperature theta > 0 by Sobol's method; the flip and the boost).
    Returns (x (dim, count) physical positions, u (3, count), particles without an accepted
    Sobol attempt)."""
    grid = list(grid)
    dim = 3 if len(grid) == 3 and grid[2] > 1 else 2
    n = np.array(grid + [1] * (3 - len(grid)), dtype=np.int32)
    d = np.array(list(dx) + [1.0] * (3 - len(dx)), dtype=np.float64)
    ncell = int(np.prod(n.astype(np.int64)))
    total = ncell * int(per_cell)
    if count is None:
        count = total - first
    x = np.zeros((dim, count))
    u = np.zeros((3, count))
    if count > 0:
        failed = _load().orc_load_drifting(
            dim, n.ctypes.data_as(_ip), _d(d), int(per_cell), int(first), int(count),
            float(gamma), float(u_th), float(theta), int(seed) & (2 ** 64 - 1),
            int(run) & (2 ** 64 - 1), int(species),
            int(species if pos_species is None else pos_species), _d(x), _d(u))
    else:
        failed = 0
    return x, u, int(failed)


JUTTNER_ATTEMPTS = 128


def juttner_speeds(theta, n, seed=0, run=0, species=0, attempts=JUTTNER_ATTEMPTS, first=0):
    """Co-moving |u'| of n particles drawn from the Juttner-Synge distribution (App. D,
    Eq. Maxwell-dist-relativistic) by Sobol's method with at most `attempts` attempts each
    (the streams the loader uses); NaN where no attempt was accepted."""
    out = np.zeros(n)
    _load().orc_juttner_speeds(float(theta), int(attempts), int(seed) & (2 ** 64 - 1),
                               int(run) & (2 ** 64 - 1), int(species), int(first), int(n), _d(out))
    out[out < 0.0] = np.nan
    return out


class Sim:
    """One periodic 2D (nz = 1) or 3D simulation held by the C oracle.

    Positions are physical, in [0, n_a dx_a); u = gamma v in units of c.
    Fields: comps 0..5 = E1 E2 E3 B1 B2 B3, 6..8 = J1 J2 J3, arrays shaped (nz, ny, nx).
    """

    def __init__(self, grid, dx, dt, l, scheme, solver=0, timing=False):
        grid = list(grid) + [1] * (3 - len(grid))
        dx = list(dx) + [1.0] * (3 - len(dx))
        self.grid = tuple(int(g) for g in grid)
        self.dx = tuple(float(d) for d in dx)
        self.dim = 3 if self.grid[2] > 1 else 2
        self.dt = float(dt)
        self.l = int(l)
        self.scheme = int(scheme)
        self._lib = _load(timing)
        self._h = self._lib.orc_create(*self.grid, *self.dx, self.dt, self.l, self.scheme)
        if not self._h:
            raise ValueError("oracle: bad arguments")
        self.solver = int(solver)
        self._lib.orc_set_solver(self._h, self.solver)
        self.nsp = 0
        self.counts = []

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.grid[2], self.grid[1], self.grid[0])

    def add_species(self, q, m, w, x, u):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.dim, -1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1)
        n = x.shape[1]
        sp = self._lib.orc_add_species(self._h, float(q), float(m), float(w), n, _d(x), _d(u))
        if sp < 0:
            raise ValueError("too many species")
        self.nsp += 1
        self.counts.append(n)
        return sp

    def set_field(self, comp, a):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
        self._lib.orc_set_field(self._h, int(comp), _d(a))

    def field(self, comp):
        out = np.zeros(self.shape, dtype=np.float64)
        self._lib.orc_get_field(self._h, int(comp), _d(out))
        return out

    def particles(self, sp):
        n = self.counts[sp]
        x = np.zeros((self.dim, n))
        u = np.zeros((3, n))
        self._lib.orc_get_particles(self._h, int(sp), _d(x), _d(u))
        return x, u

    def set_particles(self, sp, x, u):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.dim, -1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1)
        assert x.shape[1] == self.counts[sp]
        self._lib.orc_set_particles(self._h, int(sp), _d(x), _d(u))

    def gather(self, pos):
        p = np.zeros(3)
        p[:self.dim] = pos[:self.dim]
        out = np.zeros(6)
        self._lib.orc_gather(self._h, _d(p), _d(out))
        return out

    def gather_brute(self, pos):
        p = np.zeros(3)
        p[:self.dim] = pos[:self.dim]
        out = np.zeros(6)
        self._lib.orc_gather_brute(self._h, _d(p), _d(out))
        return out

    def push_particle(self, q, m, x, u):
        """Gather + Boris + move of one particle against the current fields (no deposit)."""
        xx = np.zeros(3)
        xx[:self.dim] = x[:self.dim]
        uu = np.array(u, dtype=np.float64)
        self._lib.orc_push_particle(self._h, float(q), float(m), _d(xx), _d(uu))
        return xx[:self.dim], uu

    def deposit(self, qw, xo, xn, v):
        a = np.zeros(3); a[:self.dim] = xo[:self.dim]
        b = np.zeros(3); b[:self.dim] = xn[:self.dim]
        vv = np.ascontiguousarray(v, dtype=np.float64)
        self._lib.orc_deposit(self._h, float(qw), _d(a), _d(b), _d(vv))

    def rho(self):
        out = np.zeros(self.shape)
        self._lib.orc_rho(self._h, _d(out))
        return out

    def yee_b(self, h):
        self._lib.orc_yee_b(self._h, float(h))

    def yee_e(self):
        self._lib.orc_yee_e(self._h)

    def step(self, n=1):
        self._lib.orc_step(self._h, int(n))

    def particle_pass(self, first, count):
        self._lib.orc_particle_pass(self._h, int(first), int(count))

    def particle_pass_threads(self, first, count, threads=0):
        """The particle pass over `threads` host threads (0: all OpenMP threads; the timing build
        only runs in parallel).  Returns the threads used."""
        return int(self._lib.orc_particle_pass_threads(self._h, int(first), int(count),
                                                       int(threads)))

    @property
    def step_count(self):
        return int(self._lib.orc_step_count(self._h))

    def diag(self):
        out = np.zeros(4)
        self._lib.orc_diag(self._h, _d(out))
        return {"field_energy": out[0], "kinetic_energy": out[1], "total_charge": out[2],
                "max_gauss_residual": out[3]}

    def gauss_residual(self):
        out = np.zeros(self.shape)
        self._lib.orc_gauss_residual(self._h, _d(out))
        return out
