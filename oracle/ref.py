"""ctypes wrapper of the FP64 CPU oracle (``libfdlbm_ref.so``).

TEST INFRASTRUCTURE ONLY: the plain reference that the CUDA library is checked
against.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product package never does.

The oracle follows the paper step by step (Sec. 1, 1-a, 2 and Eq. 1-2 of
Dubois, Lallemand, Obrecht, Tekitek, "Lattice Boltzmann model approximated
with finite difference expressions"); see ``fdlbm_ref.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fdlbm_ref.c")
HDR = os.path.join(HERE, "fdlbm_ref.h")
LIB = os.path.join(HERE, "libfdlbm_ref.so")

FD3, FD5, FD9, MRT, LWACM = 3, 5, 9, 100, 200
PERIODIC, WALLS_Y = 0, 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("scheme", ctypes.c_int32), ("boundary", ctypes.c_int32),
        ("s_xx", ctypes.c_double), ("s_e", ctypes.c_double),
        ("s_q", ctypes.c_double), ("s_eps", ctypes.c_double),
        ("wall_xi", ctypes.c_double),
        ("force_x", ctypes.c_double), ("force_y", ctypes.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(Params)
            i64p = ctypes.POINTER(ctypes.c_int64)
            L.fdlbm_ref_set_threads.argtypes = [ctypes.c_int]
            L.fdlbm_ref_get_threads.restype = ctypes.c_int
            L.fdlbm_ref_moment_matrix.argtypes = [dp, dp]
            L.fdlbm_ref_fd_step.argtypes = [pp, dp, dp, dp, ctypes.c_int64]
            L.fdlbm_ref_fd_step_points.argtypes = [pp, dp, dp, dp, ctypes.c_int64, i64p, dp]
            L.fdlbm_ref_fd_fstar.argtypes = [pp, dp, dp, dp, ctypes.c_int32, ctypes.c_int32, dp]
            L.fdlbm_ref_mrt_init.argtypes = [pp, dp, dp, dp, dp]
            L.fdlbm_ref_mrt_step.argtypes = [pp, dp, ctypes.c_int64]
            L.fdlbm_ref_mrt_moments.argtypes = [pp, dp, dp, dp, dp]
            L.fdlbm_ref_mrt_step_points_from_eq.argtypes = [pp, dp, dp, dp, ctypes.c_int64,
                                                             i64p, dp]
            L.fdlbm_ref_lwacm_step.argtypes = [pp, dp, dp, dp, ctypes.c_int64]
            L.fdlbm_ref_lwacm_step_points.argtypes = [pp, dp, dp, dp, ctypes.c_int64, i64p, dp]
            u8p, i8p = ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int8)
            L.fdlbm_ref_fd_step_walls.argtypes = [pp, u8p, ctypes.c_int64, i64p, i8p, dp,
                                                  dp, dp, dp, ctypes.c_int64]
            for name in ("fdlbm_ref_fd_step", "fdlbm_ref_fd_step_points", "fdlbm_ref_fd_fstar",
                         "fdlbm_ref_mrt_init", "fdlbm_ref_mrt_step", "fdlbm_ref_mrt_moments",
                         "fdlbm_ref_mrt_step_points_from_eq", "fdlbm_ref_lwacm_step",
                         "fdlbm_ref_lwacm_step_points", "fdlbm_ref_fd_step_walls"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def params(nx, ny, scheme, s_xx, s_e=1.5, s_q=1.0, s_eps=1.5, boundary=PERIODIC, wall_xi=0.5,
           force=(0.0, 0.0)) -> Params:
    return Params(int(nx), int(ny), int(scheme), int(boundary), float(s_xx), float(s_e),
                  float(s_q), float(s_eps), float(wall_xi), float(force[0]), float(force[1]))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64).copy()
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def set_threads(n: int) -> None:
    lib().fdlbm_ref_set_threads(int(n))


def get_threads() -> int:
    return int(lib().fdlbm_ref_get_threads())


def moment_matrix():
    M = np.zeros(81)
    Minv = np.zeros(81)
    lib().fdlbm_ref_moment_matrix(_dptr(M), _dptr(Minv))
    return M.reshape(9, 9), Minv.reshape(9, 9)


def fd_run(p: Params, rho, ux, uy, nsteps: int):
    """FD-LBM: return (rho, ux, uy) after nsteps, FP64 copies of the inputs."""
    shape = (p.ny, p.nx)
    r, x, y = _f64(rho, shape), _f64(ux, shape), _f64(uy, shape)
    _check(lib().fdlbm_ref_fd_step(ctypes.byref(p), _dptr(r), _dptr(x), _dptr(y), int(nsteps)),
           "fd_step")
    return r, x, y


def fd_run_walls(p: Params, walls, rho, ux, uy, nsteps: int):
    """FD-LBM with curved walls (Sec. 3-b): `walls` carries kind [ny][nx]
    (0 fluid, 1 virtual, 2 unused) and the virtual-node table (node, link,
    xi).  Returns (rho, ux, uy) after nsteps; only fluid nodes change."""
    shape = (p.ny, p.nx)
    r, x, y = _f64(rho, shape), _f64(ux, shape), _f64(uy, shape)
    kind = np.ascontiguousarray(walls.kind, dtype=np.uint8)
    node = np.ascontiguousarray(walls.node, dtype=np.int64)
    link = np.ascontiguousarray(walls.link, dtype=np.int8)
    xi = np.ascontiguousarray(walls.xi, dtype=np.float64)
    assert kind.shape == shape
    _check(lib().fdlbm_ref_fd_step_walls(
        ctypes.byref(p), kind.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), node.size,
        node.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        link.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), _dptr(xi), _dptr(r), _dptr(x),
        _dptr(y), int(nsteps)), "fd_step_walls")
    return r, x, y


def fd_step_points(p: Params, rho, ux, uy, idx):
    shape = (p.ny, p.nx)
    r, x, y = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    assert r.shape == shape and x.shape == shape and y.shape == shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((idx.size, 3))
    _check(lib().fdlbm_ref_fd_step_points(
        ctypes.byref(p), _dptr(r), _dptr(x), _dptr(y), idx.size,
        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(out)), "fd_step_points")
    return out


def fd_fstar(p: Params, rho, ux, uy, i: int, j: int):
    shape = (p.ny, p.nx)
    r, x, y = _f64(rho, shape), _f64(ux, shape), _f64(uy, shape)
    out = np.zeros(9)
    _check(lib().fdlbm_ref_fd_fstar(ctypes.byref(p), _dptr(r), _dptr(x), _dptr(y), int(i),
                                    int(j), _dptr(out)), "fd_fstar")
    return out


def mrt_init(p: Params, rho, ux, uy):
    shape = (p.ny, p.nx)
    r, x, y = _f64(rho, shape), _f64(ux, shape), _f64(uy, shape)
    f = np.zeros((9,) + shape)
    _check(lib().fdlbm_ref_mrt_init(ctypes.byref(p), _dptr(r), _dptr(x), _dptr(y), _dptr(f)),
           "mrt_init")
    return f


def mrt_step(p: Params, f, nsteps: int):
    f = _f64(f, (9, p.ny, p.nx))
    _check(lib().fdlbm_ref_mrt_step(ctypes.byref(p), _dptr(f), int(nsteps)), "mrt_step")
    return f


def mrt_moments(p: Params, f):
    f = _f64(f, (9, p.ny, p.nx))
    shape = (p.ny, p.nx)
    r, x, y = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    _check(lib().fdlbm_ref_mrt_moments(ctypes.byref(p), _dptr(f), _dptr(r), _dptr(x), _dptr(y)),
           "mrt_moments")
    return r, x, y


def mrt_run(p: Params, rho, ux, uy, nsteps: int):
    """MRT from equilibrium at (rho, u): return (rho, ux, uy) after nsteps."""
    f = mrt_step(p, mrt_init(p, rho, ux, uy), nsteps)
    return mrt_moments(p, f)


def mrt_step_points_from_eq(p: Params, rho, ux, uy, idx):
    shape = (p.ny, p.nx)
    r, x, y = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    assert r.shape == shape and x.shape == shape and y.shape == shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((idx.size, 3))
    _check(lib().fdlbm_ref_mrt_step_points_from_eq(
        ctypes.byref(p), _dptr(r), _dptr(x), _dptr(y), idx.size,
        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(out)), "mrt_step_points")
    return out


def lwacm_run(p: Params, rho, ux, uy, nsteps: int):
    """LW-ACM (Sec. 1-b): return (rho, ux, uy) after nsteps, FP64 copies of the inputs."""
    shape = (p.ny, p.nx)
    r, x, y = _f64(rho, shape), _f64(ux, shape), _f64(uy, shape)
    _check(lib().fdlbm_ref_lwacm_step(ctypes.byref(p), _dptr(r), _dptr(x), _dptr(y),
                                      int(nsteps)), "lwacm_step")
    return r, x, y


def lwacm_step_points(p: Params, rho, ux, uy, idx):
    shape = (p.ny, p.nx)
    r, x, y = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, ux, uy))
    assert r.shape == shape and x.shape == shape and y.shape == shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros((idx.size, 3))
    _check(lib().fdlbm_ref_lwacm_step_points(
        ctypes.byref(p), _dptr(r), _dptr(x), _dptr(y), idx.size,
        idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(out)), "lwacm_step_points")
    return out


def run(p: Params, rho, ux, uy, nsteps: int):
    """Any scheme from primitive fields; returns (rho, ux, uy)."""
    if p.scheme == MRT:
        return mrt_run(p, rho, ux, uy, nsteps)
    if p.scheme == LWACM:
        return lwacm_run(p, rho, ux, uy, nsteps)
    return fd_run(p, rho, ux, uy, nsteps)
