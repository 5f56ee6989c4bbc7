"""Python binding of libpic, the GB300 (sm_103a) WT-scheme PIC step (arXiv:1909.09613).

Argument marshalling only: every step of the PIC path (gather, push, move, deposit, tile sort,
Yee, diagnostics) runs in the library's CUDA kernels.  PyTorch provides device memory and the
stream.  There is no CPU fallback: if libpic.so is missing or no CUDA device is present the
calls raise.

The module exposes the C-ABI functions of include/pic.h under the same names (pic_create,
pic_footprint, pic_bind_memory, pic_load_particles, pic_step, pic_read_fields, pic_diag, ...)
and a small convenience class `Run` that owns a context and its torch-allocated memory.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpic.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECFL, PIC_ECUDA = 0, -1, -2, -3, -4
PIC_EOVERFLOW, PIC_ETIMEOUT, PIC_ENAN, PIC_ESTATE = -5, -6, -7, -8
PIC_SCHEME_MC, PIC_SCHEME_WT = 0, 1
PIC_FP64, PIC_FP32_MIXED = 0, 1
PIC_SOLVER_YEE, PIC_SOLVER_M4 = 0, 1
PIC_ORDER_AUTO, PIC_ORDER_CELL, PIC_ORDER_SLOT = 0, 1, 2
PIC_ERR_OUTSIDE_TILE, PIC_ERR_NONFINITE, PIC_ERR_TIMEOUT = 1, 2, 4  # diag()["error_flags"] bits
PIC_MAX_SPECIES = 4
PIC_JUTTNER_MIN_THETA = 0.3

_c_dp = ctypes.POINTER(ctypes.c_double)
_c_lp = ctypes.POINTER(ctypes.c_int64)
_c_ip = ctypes.POINTER(ctypes.c_int32)


class pic_options(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32 * 3), ("sort_interval", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("n_species", ctypes.c_int32),
                ("capacity", ctypes.c_int64 * PIC_MAX_SPECIES), ("stream", ctypes.c_uint64),
                ("solver", ctypes.c_int32), ("tile_order", ctypes.c_int32),
                ("deterministic", ctypes.c_int32)]


class pic_batch_capacity(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_int32), ("cells", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("stage_bytes", ctypes.c_size_t), ("ctas_per_sm", ctypes.c_int32)]


class pic_diag_t(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("field_energy", ctypes.c_double),
                ("kinetic_energy", ctypes.c_double), ("total_charge", ctypes.c_double),
                ("max_gauss_residual", ctypes.c_double),
                ("max_continuity_residual", ctypes.c_double),
                ("max_gauss_residual_drift", ctypes.c_double), ("error_flags", ctypes.c_int32)]


class PicError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, pic_strerror(status), status))


_lib = None

# (name, restype, argtypes)
_SIGS = [
    ("pic_create", ctypes.c_int, [_c_ip, _c_dp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(pic_options), ctypes.POINTER(ctypes.c_void_p)]),
    ("pic_footprint", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("pic_bind_memory", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("pic_alloc", ctypes.c_int, [ctypes.c_void_p]),
    ("pic_load_particles", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                          _c_dp, _c_dp]),
    ("pic_load_particles_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    ("pic_load_drifting_plasma", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                ctypes.c_uint64, ctypes.c_int]),
    ("pic_load_drifting_juttner", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                 ctypes.c_uint64, ctypes.c_int]),
    ("pic_set_fields", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_dp, ctypes.c_size_t]),
    ("pic_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("pic_read_fields", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_dp, ctypes.c_size_t]),
    ("pic_read_particles", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_dp, _c_dp, _c_lp,
                                          ctypes.c_int64]),
    ("pic_read_tile_offsets", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_lp, ctypes.c_int64]),
    ("pic_tile_info", ctypes.c_int, [ctypes.c_void_p, _c_ip, _c_lp, _c_ip, _c_ip]),
    ("pic_smem_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    ("pic_sort", ctypes.c_int, [ctypes.c_void_p]),
    ("pic_diag", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pic_diag_t)]),
    ("pic_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("pic_batch_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("pic_batch_reserve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pic_batch_capacity)]),
    ("pic_batch_set_runs", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.c_int]),
    ("pic_batch_footprint", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    ("pic_batch_bind_memory", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("pic_batch_alloc", ctypes.c_int, [ctypes.c_void_p]),
    ("pic_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("pic_batch_time_gpp", ctypes.c_int, [ctypes.c_void_p, _c_dp]),
    ("pic_batch_info", ctypes.c_int, [ctypes.c_void_p, _c_lp, _c_lp]),
    ("pic_batch_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("pic_batch_destroy", None, [ctypes.c_void_p]),
    ("pic_last_gpp_ms", ctypes.c_int, [ctypes.c_void_p, _c_dp, _c_lp]),
    ("pic_kernel_launches", ctypes.c_int, [ctypes.c_void_p, _c_lp]),
    ("pic_probe_fma_peak", ctypes.c_int, [ctypes.c_int, _c_dp]),
    ("pic_tile_sort_noalloc", ctypes.c_int, [_c_ip, _c_ip, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    ("pic_destroy", None, [ctypes.c_void_p]),
    ("pic_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("pic_axis_weights", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, _c_dp, _c_ip, _c_ip]),
]


def exported_names():
    return [n for n, _, _ in _SIGS]


def load_library(path: Optional[str] = None):
    """Load libpic.so (built by paper_1909_09613_gb300._build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libpic.so not built (%s): run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    for name, res, args in _SIGS:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def pic_strerror(status: int) -> str:
    try:
        return load_library().pic_strerror(int(status)).decode()
    except Exception:
        return "status %d" % status


def _check(status: int, what: str):
    if status != PIC_OK:
        raise PicError(status, what)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_c_dp)


# ---- thin wrappers with the C names --------------------------------------------------------

def pic_create(grid, dx, dt, spline_order, scheme, opt: Optional[pic_options] = None):
    lib = load_library()
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid])
    d = (ctypes.c_double * 3)(*[float(v) for v in dx])
    out = ctypes.c_void_p()
    st = lib.pic_create(g, d, float(dt), int(spline_order), int(scheme),
                        ctypes.byref(opt) if opt is not None else None, ctypes.byref(out))
    _check(st, "pic_create")
    return out.value


def pic_footprint(ctx) -> int:
    b = ctypes.c_size_t()
    _check(load_library().pic_footprint(ctx, ctypes.byref(b)), "pic_footprint")
    return int(b.value)


def pic_bind_memory(ctx, ptr: int, nbytes: int):
    _check(load_library().pic_bind_memory(ctx, ctypes.c_void_p(ptr), nbytes), "pic_bind_memory")


def pic_load_particles(ctx, species, q, m, w, x: np.ndarray, u: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.shape[-1]
    _check(load_library().pic_load_particles(ctx, int(species), float(q), float(m), float(w), n,
                                             _dptr(x), _dptr(u)), "pic_load_particles")


def pic_load_particles_device(ctx, species, q, m, w, x_ptr: int, u_ptr: int, n: int):
    _check(load_library().pic_load_particles_device(ctx, int(species), float(q), float(m),
                                                    float(w), int(n), ctypes.c_void_p(x_ptr),
                                                    ctypes.c_void_p(u_ptr)),
           "pic_load_particles_device")


def pic_load_drifting_plasma(ctx, species, q, m, w, per_cell, gamma, u_th, seed, run,
                             pos_species):
    _check(load_library().pic_load_drifting_plasma(ctx, int(species), float(q), float(m),
                                                   float(w), int(per_cell), float(gamma),
                                                   float(u_th), int(seed) & (2**64 - 1),
                                                   int(run) & (2**64 - 1), int(pos_species)),
           "pic_load_drifting_plasma")


def pic_load_drifting_juttner(ctx, species, q, m, w, per_cell, gamma, theta, seed, run,
                              pos_species):
    _check(load_library().pic_load_drifting_juttner(ctx, int(species), float(q), float(m),
                                                    float(w), int(per_cell), float(gamma),
                                                    float(theta), int(seed) & (2**64 - 1),
                                                    int(run) & (2**64 - 1), int(pos_species)),
           "pic_load_drifting_juttner")


def pic_set_fields(ctx, comp, a: np.ndarray):
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    _check(load_library().pic_set_fields(ctx, int(comp), _dptr(a), a.size), "pic_set_fields")


def pic_step(ctx, nsteps: int):
    _check(load_library().pic_step(ctx, int(nsteps)), "pic_step")


def pic_read_fields(ctx, comp, ncell) -> np.ndarray:
    out = np.empty(ncell, dtype=np.float64)
    _check(load_library().pic_read_fields(ctx, int(comp), _dptr(out), ncell), "pic_read_fields")
    return out


def pic_read_particles(ctx, species, n, dim):
    x = np.empty((dim, n), dtype=np.float64)
    u = np.empty((3, n), dtype=np.float64)
    cell = np.empty(n, dtype=np.int64)
    _check(load_library().pic_read_particles(ctx, int(species), _dptr(x), _dptr(u),
                                             cell.ctypes.data_as(_c_lp), n), "pic_read_particles")
    return x, u, cell


def pic_read_tile_offsets(ctx, species, ntiles) -> np.ndarray:
    out = np.empty(ntiles + 1, dtype=np.int64)
    _check(load_library().pic_read_tile_offsets(ctx, int(species), out.ctypes.data_as(_c_lp),
                                                ntiles + 1), "pic_read_tile_offsets")
    return out


def pic_tile_info(ctx):
    """(tile extent, number of tiles, sort interval, slot-major order flag)"""
    t = (ctypes.c_int32 * 3)()
    nt = ctypes.c_int64()
    si = ctypes.c_int32()
    sm = ctypes.c_int32()
    _check(load_library().pic_tile_info(ctx, t, ctypes.byref(nt), ctypes.byref(si),
                                        ctypes.byref(sm)), "pic_tile_info")
    return tuple(t), int(nt.value), int(si.value), int(sm.value)


def pic_smem_info(ctx):
    """(own kernel's shared memory per CTA, batched kernel's for this run, two-per-SM limit)"""
    a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(load_library().pic_smem_info(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "pic_smem_info")
    return int(a.value), int(b.value), int(c.value)


def pic_sort(ctx):
    _check(load_library().pic_sort(ctx), "pic_sort")


def pic_sync(ctx):
    _check(load_library().pic_sync(ctx), "pic_sync")


def pic_diag(ctx) -> dict:
    d = pic_diag_t()
    st = load_library().pic_diag(ctx, ctypes.byref(d))
    out = {"step": d.step, "field_energy": d.field_energy, "kinetic_energy": d.kinetic_energy,
           "total_charge": d.total_charge, "max_gauss_residual": d.max_gauss_residual,
           "max_continuity_residual": d.max_continuity_residual,
           "max_gauss_residual_drift": d.max_gauss_residual_drift,
           "error_flags": d.error_flags, "status": st}
    return out


class Batch:
    """Batched form: advance many `Run`s (2D, FP32 form, same stream) together with one
    persistent particle kernel per step, replayed from a CUDA graph (pic_batch_*).
    `capacity` (a pic_batch_capacity, or None for the initial set's sizes) leaves room for the
    other run sets `set_runs` may install later without a new graph."""

    def __init__(self, runs, capacity: Optional[pic_batch_capacity] = None):
        import torch
        self.runs = list(runs)
        arr = (ctypes.c_void_p * len(self.runs))(*[r.ctx for r in self.runs])
        h = ctypes.c_void_p()
        lib = load_library()
        _check(lib.pic_batch_create(arr, len(self.runs), ctypes.byref(h)), "pic_batch_create")
        self.h = h.value
        if capacity is not None:
            st = lib.pic_batch_reserve(self.h, ctypes.byref(capacity))
            if st != PIC_OK:
                lib.pic_batch_destroy(self.h)
                self.h = None
                raise PicError(st, "pic_batch_reserve")
        nb = ctypes.c_size_t()
        _check(lib.pic_batch_footprint(self.h, ctypes.byref(nb)), "pic_batch_footprint")
        self.mem = torch.empty(int(nb.value), dtype=torch.uint8, device=self.runs[0].device)
        _check(lib.pic_batch_bind_memory(self.h, ctypes.c_void_p(self.mem.data_ptr()), nb.value),
               "pic_batch_bind_memory")

    def set_runs(self, runs) -> bool:
        """Install another run set (the old runs' state is written back first).  False when the
        set does not fit the batch's capacities (the batch keeps its old runs then)."""
        runs = list(runs)
        arr = (ctypes.c_void_p * max(len(runs), 1))(*[r.ctx for r in runs])
        st = load_library().pic_batch_set_runs(self.h, arr, len(runs))
        if st == PIC_ENOMEM:
            return False
        _check(st, "pic_batch_set_runs")
        self.runs = runs
        return True

    def step(self, n=1):
        _check(load_library().pic_batch_step(self.h, int(n)), "pic_batch_step")

    def time_gpp(self):
        ms = ctypes.c_double()
        _check(load_library().pic_batch_time_gpp(self.h, ctypes.byref(ms)), "pic_batch_time_gpp")
        return float(ms.value)

    def info(self):
        a = ctypes.c_int64()
        b = ctypes.c_int64()
        _check(load_library().pic_batch_info(self.h, ctypes.byref(a), ctypes.byref(b)), "pic_batch_info")
        return int(a.value), int(b.value)

    def sync(self):
        _check(load_library().pic_batch_sync(self.h), "pic_batch_sync")

    def close(self):
        if getattr(self, "h", None):
            load_library().pic_batch_destroy(self.h)
            self.h = None
            self.mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pic_last_gpp_ms(ctx):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load_library().pic_last_gpp_ms(ctx, ctypes.byref(ms), ctypes.byref(n)), "pic_last_gpp_ms")
    return float(ms.value), int(n.value)


def pic_kernel_launches(ctx) -> int:
    n = ctypes.c_int64()
    _check(load_library().pic_kernel_launches(ctx, ctypes.byref(n)), "pic_kernel_launches")
    return int(n.value)


def pic_probe_fma_peak(kind: int) -> float:
    v = ctypes.c_double()
    _check(load_library().pic_probe_fma_peak(int(kind), ctypes.byref(v)), "pic_probe_fma_peak")
    return float(v.value)


def pic_tile_sort_noalloc(grid, tile, cells, stream=None):
    """Cell-major tile order of `cells` (a CUDA int32 tensor) without any device allocation
    inside the library; returns (perm, tile_start) as CUDA int64 tensors (allocated here by
    torch, i.e. by the caller of the C entry point).  perm positions past tile_start[-1] (cells
    outside the grid) hold -1.  The call runs with the tensors' device current."""
    import torch
    with torch.cuda.device(cells.device):
        return _tile_sort_noalloc(grid, tile, cells, stream)


def _tile_sort_noalloc(grid, tile, cells, stream):
    import torch
    g = (ctypes.c_int32 * 3)(*[int(v) for v in grid])
    t = (ctypes.c_int32 * 3)(*[int(v) for v in tile])
    ntiles = 1
    for a in range(3):
        ntiles *= (int(grid[a]) + int(tile[a]) - 1) // int(tile[a])
    cells = cells.contiguous()
    perm = torch.empty(cells.numel(), dtype=torch.int64, device=cells.device)
    ts = torch.empty(ntiles + 1, dtype=torch.int64, device=cells.device)
    st = stream if stream is not None else torch.cuda.current_stream(cells.device).cuda_stream
    _check(load_library().pic_tile_sort_noalloc(g, t, cells.numel(), cells.data_ptr(),
                                                perm.data_ptr(), ts.data_ptr(), int(st)),
           "pic_tile_sort_noalloc")
    return perm, ts


def pic_destroy(ctx):
    if ctx:
        load_library().pic_destroy(ctx)


def pic_axis_weights(spline_order, scheme, dtt, delta):
    """Host evaluation of the integer-node interpolation weights the kernels use along one
    axis (T_l for WT, W_l for MC).  Returns (first_node, weights)."""
    w = np.zeros(8)
    b = ctypes.c_int32()
    k = ctypes.c_int32()
    _check(load_library().pic_axis_weights(int(spline_order), int(scheme), float(dtt),
                                           float(delta), _dptr(w), ctypes.byref(b),
                                           ctypes.byref(k)), "pic_axis_weights")
    return int(b.value), w[:k.value].copy()


# ---- convenience wrapper ---------------------------------------------------------------------

class Run:
    """One PIC run: a libpic context plus the torch-allocated device buffer bound to it."""

    def __init__(self, grid, dx, dt, l, scheme, precision=PIC_FP64, capacity=(0, 0),
                 tile=None, sort_interval=0, stream=None, device=None, solver=PIC_SOLVER_YEE,
                 tile_order=PIC_ORDER_AUTO, deterministic=False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libpic needs a CUDA device")
        grid = list(grid) + [1] * (3 - len(grid))
        dx = list(dx) + [1.0] * (3 - len(dx))
        self.grid = tuple(int(g) for g in grid)
        self.dx = tuple(float(d) for d in dx)
        self.dim = 3 if self.grid[2] > 1 else 2
        self.ncell = self.grid[0] * self.grid[1] * self.grid[2]
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        opt = pic_options()
        if tile is not None:
            for a, t in enumerate(tile):
                opt.tile[a] = int(t)
        opt.sort_interval = int(sort_interval)
        opt.precision = int(precision)
        opt.n_species = len(capacity)
        for s, c in enumerate(capacity):
            opt.capacity[s] = int(c)
        opt.stream = int(self.stream.cuda_stream)
        opt.solver = int(solver)
        opt.tile_order = int(tile_order)
        opt.deterministic = 1 if deterministic else 0
        self.ctx = pic_create(self.grid, self.dx, dt, l, scheme, opt)
        self.nbytes = pic_footprint(self.ctx)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        pic_bind_memory(self.ctx, self.mem.data_ptr(), self.nbytes)
        self.counts = [0] * len(capacity)
        self.tile, self.ntiles, self.sort_interval, self.slot_major = pic_tile_info(self.ctx)

    def load(self, species, q, m, w, x, u):
        import torch
        if isinstance(x, torch.Tensor) and x.is_cuda:
            x = x.contiguous().to(torch.float64)
            u = u.contiguous().to(torch.float64)
            n = int(u.shape[-1])
            pic_load_particles_device(self.ctx, species, q, m, w, x.data_ptr(), u.data_ptr(), n)
        else:
            if isinstance(x, torch.Tensor):
                x, u = x.numpy(), u.numpy()
            n = int(np.asarray(u).shape[-1])
            pic_load_particles(self.ctx, species, q, m, w, x, u)
        self.counts[species] = n

    def load_drifting_plasma(self, species, q, m, w, per_cell, gamma, u_th, seed, run=0,
                             pos_species=None):
        """Generate species `species` on the device (App. D drifting plasma, pic.h)."""
        pic_load_drifting_plasma(self.ctx, species, q, m, w, per_cell, gamma, u_th, seed, run,
                                 species if pos_species is None else pos_species)
        self.counts[species] = int(np.prod(self.grid)) * int(per_cell)

    def load_drifting_juttner(self, species, q, m, w, per_cell, gamma, theta, seed, run=0,
                              pos_species=None):
        """Same with Juttner-Synge co-moving momenta of temperature theta (Sobol's method)."""
        pic_load_drifting_juttner(self.ctx, species, q, m, w, per_cell, gamma, theta, seed, run,
                                  species if pos_species is None else pos_species)
        self.counts[species] = int(np.prod(self.grid)) * int(per_cell)

    def set_field(self, comp, a):
        pic_set_fields(self.ctx, comp, a)

    def step(self, n=1):
        pic_step(self.ctx, n)

    def field(self, comp):
        return pic_read_fields(self.ctx, comp, self.ncell).reshape(self.grid[2], self.grid[1],
                                                                   self.grid[0])

    def particles(self, species):
        return pic_read_particles(self.ctx, species, self.counts[species], self.dim)

    def tile_offsets(self, species):
        return pic_read_tile_offsets(self.ctx, species, self.ntiles)

    def diag(self):
        return pic_diag(self.ctx)

    def sync(self):
        pic_sync(self.ctx)

    def sort(self):
        pic_sort(self.ctx)

    def gpp_ms(self):
        return pic_last_gpp_ms(self.ctx)

    def kernel_launches(self):
        return pic_kernel_launches(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            pic_destroy(self.ctx)
            self.ctx = None
            self.mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
