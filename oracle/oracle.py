"""Python access to the plain FP64 CPU oracle of the D2Q37 time step (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may import this
module. It loads oracle/liboracle_d2q37.so (built from d2q37_oracle.c by oracle/build.py) and
exposes it on numpy arrays. It never touches the CUDA path.

Layouts: the oracle is site-major, ``f[Ly, Lx, 37]`` (its own velocity order, see
``velocity_set``). ``to_planes`` / ``from_planes`` convert to and from the plane-major
``f[37, Ly, Lx]`` layout in any other velocity order, matching populations by their velocity
vector, so the oracle and a caller never need to agree on an index order.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NPOP = 37

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.or_npop.restype = C.c_int
        L.or_velocity_set.argtypes = [ip, ip, dp, C.POINTER(C.c_double)]
        L.or_equilibrium.argtypes = [C.c_size_t, dp, dp, dp, dp, dp]
        L.or_moments.argtypes = [C.c_size_t, dp, dp, dp, dp, dp]
        L.or_collide.argtypes = [C.c_size_t, dp, C.c_double, C.c_double, C.c_double, C.c_int]
        L.or_propagate.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int]
        L.or_walls.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, dp]
        L.or_run.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                             C.c_double, C.c_int, C.c_int, C.c_int, dp, dp]
        L.or_run.restype = C.c_int
        L.or_walls_mirror.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, dp]
        L.or_moments_half_step.argtypes = [C.c_size_t, dp, C.c_double, C.c_double, dp, dp, dp, dp]
        L.or_run_walls.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp]
        L.or_run_walls.restype = C.c_int
        _lib = L
    return _lib


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def velocity_set():
    """(cx[37], cy[37], w[37], r): the oracle's velocity table, weights and thermal scale."""
    cx = np.zeros(NPOP, np.int32)
    cy = np.zeros(NPOP, np.int32)
    w = np.zeros(NPOP, np.float64)
    r = C.c_double()
    lib().or_velocity_set(cx, cy, w, C.byref(r))
    return cx, cy, w, r.value


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def equilibrium(rho, ux, uy, T) -> np.ndarray:
    """Equilibrium populations, shape rho.shape + (37,), oracle order."""
    rho, ux, uy, T = (_c(np.broadcast_to(v, np.shape(rho))) for v in (rho, ux, uy, T))
    out = np.empty(rho.shape + (NPOP,), np.float64)
    lib().or_equilibrium(rho.size, rho.ravel(), ux.ravel(), uy.ravel(), T.ravel(), out.reshape(-1))
    return out


def moments(f):
    """(rho, ux, uy, T) of site-major populations f[..., 37]."""
    f = _c(f)
    shape = f.shape[:-1]
    n = int(np.prod(shape))
    outs = [np.empty(n, np.float64) for _ in range(4)]
    lib().or_moments(n, f.reshape(-1), *outs)
    return tuple(o.reshape(shape) for o in outs)


def collide(f, tau: float, gx: float = 0.0, gy: float = 0.0, nthreads: int = 1) -> np.ndarray:
    """Collided copy of site-major populations f[..., 37]."""
    out = _c(f).copy()
    lib().or_collide(out.size // NPOP, out.reshape(-1), tau, gx, gy, nthreads)
    return out


def propagate(src_full, Lx: int, Ly: int, y_periodic: bool, nthreads: int = 1) -> np.ndarray:
    """Pull propagate of src_full[Ly+6, Lx, 37] (halo rows included); returns the interior
    result [Ly, Lx, 37]."""
    src_full = _c(src_full)
    assert src_full.shape == (Ly + 6, Lx, NPOP)
    dst = np.zeros_like(src_full)
    lib().or_propagate(Lx, Ly, int(bool(y_periodic)), src_full.reshape(-1), dst.reshape(-1), nthreads)
    return dst[3:Ly + 3]


WALL_MODES = {"rest": 0, "mirror": 1}


def with_walls(f_int, T_top: float, T_bottom: float, wall_mode: str = "rest") -> np.ndarray:
    """Interior populations [Ly, Lx, 37] -> full array [Ly+6, Lx, 37] with wall halo rows."""
    f_int = _c(f_int)
    Ly, Lx, _ = f_int.shape
    full = np.zeros((Ly + 6, Lx, NPOP), np.float64)
    full[3:Ly + 3] = f_int
    walls = lib().or_walls_mirror if WALL_MODES[wall_mode] == 1 else lib().or_walls
    walls(Lx, Ly, T_top, T_bottom, full.reshape(-1))
    return full


def moments_half_step(f, gx: float = 0.0, gy: float = 0.0):
    """Half-step fields (rho, ux, uy, T) of post-collision populations f[..., 37]."""
    f = _c(f)
    shape = f.shape[:-1]
    n = int(np.prod(shape))
    out = [np.empty(n) for _ in range(4)]
    lib().or_moments_half_step(n, f.reshape(-1), gx, gy, *out)
    return tuple(o.reshape(shape) for o in out)


def run(f0, tau: float, nsteps: int, gy: float = 0.0, T_top: float = 1.0, T_bottom: float = 1.0,
        y_periodic: bool = False, gx: float = 0.0, nthreads: int | None = None,
        wall_mode: str = "rest") -> np.ndarray:
    """nsteps time steps (wall halos, pull, collide) from interior populations f0[Ly, Lx, 37]."""
    f0 = _c(f0)
    Ly, Lx, npop = f0.shape
    assert npop == NPOP
    out = np.empty_like(f0)
    nt = default_threads() if nthreads is None else nthreads
    rc = lib().or_run_walls(Lx, Ly, tau, gx, gy, T_top, T_bottom, int(bool(y_periodic)),
                            WALL_MODES[wall_mode], nsteps, nt, f0.reshape(-1), out.reshape(-1))
    if rc != 0:
        raise MemoryError("oracle could not allocate its lattice")
    return out


def init_fields(fields) -> np.ndarray:
    """Site-major equilibrium populations [Ly, Lx, 37] of an inputs.RTFields."""
    return equilibrium(fields.rho, fields.ux, fields.uy, fields.T)


def order_map(cx_other, cy_other) -> np.ndarray:
    """perm such that oracle population perm[j] has the velocity of population j of the other
    table; raises if the two tables are not the same set of velocities."""
    cx, cy, _, _ = velocity_set()
    index = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(cx, cy))}
    perm = np.array([index[(int(a), int(b))] for a, b in zip(cx_other, cy_other)], np.int64)
    if sorted(perm.tolist()) != list(range(NPOP)):
        raise ValueError("velocity tables differ")
    return perm


def to_planes(f_site, cx_other, cy_other) -> np.ndarray:
    """Oracle site-major f[Ly, Lx, 37] -> plane-major f[37, Ly, Lx] in the other table's order."""
    perm = order_map(cx_other, cy_other)
    return np.ascontiguousarray(np.moveaxis(np.asarray(f_site)[..., perm], -1, 0))


def from_planes(f_planes, cx_other, cy_other) -> np.ndarray:
    """Plane-major f[37, Ly, Lx] in the other table's order -> oracle site-major f[Ly, Lx, 37]."""
    perm = order_map(cx_other, cy_other)
    site = np.moveaxis(np.asarray(f_planes, dtype=np.float64), 0, -1)
    out = np.empty_like(site)
    out[..., perm] = site
    return np.ascontiguousarray(out)
