"""Python binding of the C-ABI library ``libfdlbm.so`` (include/fdlbm.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  PyTorch provides device memory (the workspace and
field tensors) and CUDA streams.  There is no fallback: if the library is
missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdlbm.so")

# include/fdlbm.h constants
OK, ERR_INVALID, ERR_UNSUPPORTED, ERR_NOMEM, ERR_CUDA, ERR_DIVERGED, ERR_TIMEOUT, ERR_RANGE = (
    0, -1, -2, -3, -4, -5, -6, -7)
SCHEMES = {"fd3": 3, "fd5": 5, "fd9": 9, "mrt": 100, "lwacm": 200}
BOUNDARIES = {"periodic": 0, "walls_y": 1}
STORAGES = {"f32": 0, "f16": 1, "bf16": 2, "i16": 3}
REDUCE = {"mass": 0, "momentum": 1, "energy": 2, "mode": 3, "maxabs": 4}
FLAG_TILED = 1
FLAG_STREAM = 2
S_Q_QUARTIC = 0.0


class FdlbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("scheme", ctypes.c_int32), ("boundary", ctypes.c_int32),
        ("storage", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("s_xx", ctypes.c_double), ("s_e", ctypes.c_double),
        ("s_q", ctypes.c_double), ("s_eps", ctypes.c_double),
        ("wall_xi", ctypes.c_double),
        ("force_x", ctypes.c_double), ("force_y", ctypes.c_double),
        ("storage_range", ctypes.c_double),
    ]


class BatchParams(ctypes.Structure):
    _fields_ = [
        ("scheme", ctypes.c_int32), ("max_lattices", ctypes.c_int32),
        ("arena_bytes", ctypes.c_int64), ("max_side", ctypes.c_int32),
        ("flags", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load libfdlbm.so (built by paper_1803_00437_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise FdlbmError(ERR_CUDA, f"{p} is missing: build it with "
                             "`python -m paper_1803_00437_gb300.build`")
        L = ctypes.CDLL(p)
        vp, cp = ctypes.c_void_p, ctypes.c_char_p
        pp = ctypes.POINTER(Params)
        fp = ctypes.c_void_p  # float* / double* passed as addresses
        L.fdlbm_workspace_size.argtypes = [pp]
        L.fdlbm_workspace_size.restype = ctypes.c_size_t
        L.fdlbm_create.argtypes = [pp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.fdlbm_destroy.argtypes = [vp]
        L.fdlbm_destroy.restype = None
        L.fdlbm_set_stream.argtypes = [vp, vp]
        L.fdlbm_init.argtypes = [vp, fp, fp, fp]
        L.fdlbm_init_host.argtypes = [vp, fp, fp, fp]
        L.fdlbm_init_modes.argtypes = [vp, ctypes.c_int32, fp, ctypes.c_double, ctypes.c_double]
        L.fdlbm_step.argtypes = [vp, ctypes.c_int64]
        L.fdlbm_moments.argtypes = [vp, fp, fp, fp]
        L.fdlbm_moments_host.argtypes = [vp, fp, fp, fp]
        L.fdlbm_reduce.argtypes = [vp, ctypes.c_int32, fp, fp]
        L.fdlbm_sync.argtypes = [vp]
        L.fdlbm_selftest_wait_timeout.argtypes = [vp, ctypes.c_int32]
        L.fdlbm_selftest_wait_timeout.restype = ctypes.c_int
        L.fdlbm_last_error.argtypes = [vp]
        L.fdlbm_last_error.restype = cp
        L.fdlbm_status_string.argtypes = [ctypes.c_int]
        L.fdlbm_status_string.restype = cp
        L.fdlbm_launch_count.argtypes = [vp]
        L.fdlbm_launch_count.restype = ctypes.c_int64
        bp = ctypes.POINTER(BatchParams)
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        L.fdlbm_batch_workspace_size.argtypes = [bp]
        L.fdlbm_batch_workspace_size.restype = ctypes.c_size_t
        L.fdlbm_batch_create.argtypes = [bp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.fdlbm_batch_destroy.argtypes = [vp]
        L.fdlbm_batch_destroy.restype = None
        L.fdlbm_batch_add.argtypes = [vp, pp, ctypes.POINTER(i32)]
        L.fdlbm_batch_remove.argtypes = [vp, i32]
        L.fdlbm_batch_init.argtypes = [vp, i32, fp, fp, fp]
        L.fdlbm_batch_init_modes.argtypes = [vp, i32, i32, fp, ctypes.c_double, ctypes.c_double]
        L.fdlbm_batch_step.argtypes = [vp, i64, fp]
        L.fdlbm_batch_moments.argtypes = [vp, i32, fp, fp, fp]
        L.fdlbm_batch_reduce.argtypes = [vp, i32, i32, fp, fp]
        L.fdlbm_batch_sync.argtypes = [vp]
        L.fdlbm_batch_set_segment_rows.argtypes = [vp, i32]
        L.fdlbm_batch_set_grid.argtypes = [vp, i32]
        L.fdlbm_batch_set_narrow_strips.argtypes = [vp, i32]
        L.fdlbm_stream_plan.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(i32)]
        L.fdlbm_stream_plan.restype = ctypes.c_int
        L.fdlbm_stream_plan_candidates.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(i32),
                                                   i32, ctypes.POINTER(i32)]
        L.fdlbm_stream_plan_candidates.restype = ctypes.c_int
        L.fdlbm_set_stream_plan.argtypes = [vp, i32, i32, i32]
        L.fdlbm_set_stream_plan.restype = ctypes.c_int
        L.fdlbm_get_stream_plan.argtypes = [vp, ctypes.POINTER(i32)]
        L.fdlbm_get_stream_plan.restype = ctypes.c_int
        L.fdlbm_batch_last_error.argtypes = [vp]
        L.fdlbm_batch_last_error.restype = cp
        L.fdlbm_batch_launch_count.argtypes = [vp]
        L.fdlbm_batch_launch_count.restype = i64
        L.fdlbm_batch_count.argtypes = [vp]
        L.fdlbm_batch_count.restype = i32
        for name in ("fdlbm_batch_create", "fdlbm_batch_add", "fdlbm_batch_remove",
                     "fdlbm_batch_init", "fdlbm_batch_init_modes", "fdlbm_batch_step",
                     "fdlbm_batch_moments", "fdlbm_batch_reduce", "fdlbm_batch_sync",
                     "fdlbm_batch_set_segment_rows", "fdlbm_batch_set_grid",
                     "fdlbm_batch_set_narrow_strips"):
            getattr(L, name).restype = ctypes.c_int
        L.fdlbm_get_populations.argtypes = [vp, fp]
        L.fdlbm_get_populations.restype = ctypes.c_int
        L.fdlbm_set_populations.argtypes = [vp, fp]
        L.fdlbm_set_populations.restype = ctypes.c_int
        L.fdlbm_walls_table_bytes.argtypes = [pp]
        L.fdlbm_walls_table_bytes.restype = ctypes.c_size_t
        L.fdlbm_set_walls.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_size_t]
        L.fdlbm_set_walls.restype = ctypes.c_int
        L.fdlbm_reduce_fields_static.argtypes = [fp, fp, fp, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32, fp, fp, vp]
        L.fdlbm_reduce_fields_static.restype = ctypes.c_int
        for name in ("fdlbm_create", "fdlbm_set_stream", "fdlbm_init", "fdlbm_init_host",
                     "fdlbm_init_modes", "fdlbm_step", "fdlbm_moments", "fdlbm_moments_host",
                     "fdlbm_reduce", "fdlbm_sync"):
            getattr(L, name).restype = ctypes.c_int
        if path is None:
            _lib = L
        return L


def status_string(status: int) -> str:
    return load_library().fdlbm_status_string(int(status)).decode()


def stream_plan(nx: int, ny: int, scheme: str = "fd5", storage: str = "f32",
                resident_ctas: int = 152 * 8) -> dict:
    """The streaming step's launch plan (fdlbm_stream_plan) for an nx x ny
    lattice: rows per long segment and their number, rows per short segment
    and their number (0 if all segments are equal), CTA strips and CTAs;
    host-only."""
    lib = load_library()
    out = (ctypes.c_int32 * 6)()
    rc = lib.fdlbm_stream_plan(int(nx), int(ny), SCHEMES[scheme], STORAGES[storage],
                               int(resident_ctas), out)
    if rc != OK:
        raise FdlbmError(rc, f"stream plan: {status_string(rc)}")
    return {"seg_rows": out[0], "nsegs": out[1], "tail_rows": out[2], "ntail": out[3],
            "strips": out[4], "ctas": out[5]}


def stream_plan_candidates(nx: int, ny: int, scheme: str = "fd5", storage: str = "f32",
                           resident_ctas: int = 152 * 8, max_candidates: int = 32) -> list:
    """Candidate plans of the streaming step (fdlbm_stream_plan_candidates):
    (rows per long segment, long segments, rows per short segment) tuples,
    the model's plan first; host-only."""
    lib = load_library()
    out = (ctypes.c_int32 * (3 * max_candidates))()
    n = ctypes.c_int32()
    rc = lib.fdlbm_stream_plan_candidates(int(nx), int(ny), SCHEMES[scheme], STORAGES[storage],
                                          int(resident_ctas), out, int(max_candidates),
                                          ctypes.byref(n))
    if rc != OK:
        raise FdlbmError(rc, f"stream plan candidates: {status_string(rc)}")
    return [(out[3 * i], out[3 * i + 1], out[3 * i + 2]) for i in range(n.value)]


def nu_to_s(nu: float) -> float:
    """Sec. 1-a: nu = (1/s_xx - 1/2)/3, so s_xx = 1 / (3 nu + 1/2)."""
    return 1.0 / (3.0 * nu + 0.5)


@dataclass
class LatticeConfig:
    nx: int
    ny: int
    scheme: str = "fd5"
    boundary: str = "periodic"
    storage: str = "f32"
    s_xx: float = 1.85
    s_e: float = 1.5
    s_q: float | None = None  # None: FDLBM_S_Q_QUARTIC (MRT: the library applies Eq. sigsig)
    s_eps: float = 1.5
    wall_xi: float = 0.5
    force: tuple = (0.0, 0.0)
    flags: int = 0
    storage_range: float = 0.0  # "i16" storage: largest |value| representable


    def params(self) -> Params:
        s_q = self.s_q if self.s_q is not None else S_Q_QUARTIC
        return Params(int(self.nx), int(self.ny), SCHEMES[self.scheme],
                      BOUNDARIES[self.boundary], STORAGES[self.storage], int(self.flags),
                      float(self.s_xx), float(self.s_e), float(s_q), float(self.s_eps),
                      float(self.wall_xi), float(self.force[0]), float(self.force[1]),
                      float(self.storage_range))


def workspace_size(cfg: LatticeConfig) -> int:
    p = cfg.params()
    return int(load_library().fdlbm_workspace_size(ctypes.byref(p)))


def _addr(t) -> int:
    import torch
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    raise TypeError("expected a torch tensor")


class Lattice:
    """One D2Q9 lattice (FD-LBM or MRT) on one GPU.

    The workspace is a torch uint8 tensor on the device (allocated here unless
    given); every call is enqueued on `stream` (a torch.cuda.Stream; default:
    the current stream of the device)."""

    def __init__(self, cfg: LatticeConfig, device=None, stream=None, workspace=None):
        import torch
        self.cfg = cfg
        self.lib = load_library()
        self.params = cfg.params()
        nbytes = int(self.lib.fdlbm_workspace_size(ctypes.byref(self.params)))
        if nbytes == 0:
            raise FdlbmError(ERR_INVALID, f"invalid lattice parameters {cfg}")
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        if workspace.numel() * workspace.element_size() < nbytes:
            raise FdlbmError(ERR_NOMEM, "workspace too small")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.fdlbm_create(ctypes.byref(self.params), ctypes.c_void_p(_addr(workspace)),
                                       nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(self._h))
        if rc != OK:
            raise FdlbmError(rc, f"fdlbm_create failed: {status_string(rc)}")
        self.workspace_bytes = nbytes

    # -- helpers --------------------------------------------------------------------
    def _check(self, rc: int, what: str):
        if rc != OK:
            msg = self.lib.fdlbm_last_error(self._h).decode()
            raise FdlbmError(rc, f"{what}: {status_string(rc)}: {msg}")

    def _field(self, t):
        import torch
        if not (isinstance(t, torch.Tensor) and t.dtype == torch.float32 and t.is_cuda
                and t.device == self.device and t.is_contiguous()
                and t.numel() == self.cfg.nx * self.cfg.ny):
            raise ValueError("fields must be contiguous float32 CUDA tensors of nx*ny elements "
                             "on the lattice's device")
        return ctypes.c_void_p(t.data_ptr())

    @staticmethod
    def _host(a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        return a, ctypes.c_void_p(a.ctypes.data)

    # -- API ------------------------------------------------------------------------
    def set_stream(self, stream):
        self.stream = stream
        self._check(self.lib.fdlbm_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)),
                    "set_stream")

    def init(self, drho, ux, uy):
        """drho, ux, uy: float32 CUDA tensors [ny, nx]."""
        self._check(self.lib.fdlbm_init(self._h, self._field(drho), self._field(ux),
                                        self._field(uy)), "init")

    def populations(self):
        """MRT state (fdlbm_get_populations): a float32 CUDA tensor [9, ny, nx]
        of f_a - w_a."""
        import torch
        f = torch.empty((9, self.cfg.ny, self.cfg.nx), dtype=torch.float32, device=self.device)
        self._check(self.lib.fdlbm_get_populations(self._h, ctypes.c_void_p(f.data_ptr())),
                    "get_populations")
        return f

    def set_populations(self, f):
        """Replace the MRT state by f (float32 CUDA tensor [9, ny, nx], as
        returned by populations())."""
        import torch
        if not (isinstance(f, torch.Tensor) and f.dtype == torch.float32 and f.is_cuda
                and f.is_contiguous() and tuple(f.shape) == (9, self.cfg.ny, self.cfg.nx)):
            raise ValueError("populations must be a contiguous float32 CUDA tensor [9, ny, nx]")
        self._check(self.lib.fdlbm_set_populations(self._h, ctypes.c_void_p(f.data_ptr())),
                    "set_populations")

    def set_walls(self, walls):
        """Curved walls (Sec. 3-b, fdlbm_set_walls): `walls` carries kind
        [ny, nx] (0 fluid, 1 virtual, 2 unused) and, per virtual node, node
        (flat index), link (1..8) and xi; None removes them.  The device
        table is a torch uint8 tensor kept with the lattice."""
        import torch
        if walls is None:
            self._check(self.lib.fdlbm_set_walls(self._h, None, 0, None, None, None, None, 0),
                        "set_walls")
            self._walls_table = None
            return
        kind = np.ascontiguousarray(walls.kind, dtype=np.uint8)
        node = np.ascontiguousarray(walls.node, dtype=np.int64)
        link = np.ascontiguousarray(walls.link, dtype=np.int8)
        xi = np.ascontiguousarray(walls.xi, dtype=np.float64)
        if kind.shape != (self.cfg.ny, self.cfg.nx):
            raise ValueError("kind must be [ny, nx]")
        nbytes = int(self.lib.fdlbm_walls_table_bytes(ctypes.byref(self.params)))
        table = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=self.device)
        self._check(self.lib.fdlbm_set_walls(
            self._h, ctypes.c_void_p(kind.ctypes.data), node.size,
            ctypes.c_void_p(node.ctypes.data), ctypes.c_void_p(link.ctypes.data),
            ctypes.c_void_p(xi.ctypes.data), ctypes.c_void_p(table.data_ptr()), nbytes),
            "set_walls")
        self._walls_table = table

    def init_host(self, drho, ux, uy):
        """drho, ux, uy: host arrays [ny, nx] (converted to float32)."""
        n = self.cfg.nx * self.cfg.ny
        arrs = [self._host(np.asarray(a).reshape(-1)) for a in (drho, ux, uy)]
        for a, _ in arrs:
            if a.size != n:
                raise ValueError("fields must have nx*ny elements")
        self._check(self.lib.fdlbm_init_host(self._h, *[p for _, p in arrs]), "init_host")

    def init_modes(self, modes, mean_velocity=(0.0, 0.0)):
        """modes: iterable of (m, n, amplitude, phase) (e.g. inputs.Mode)."""
        rec = np.ascontiguousarray(
            [[float(md[0]), float(md[1]), float(md[2]), float(md[3])] if not hasattr(md, "m")
             else [float(md.m), float(md.n), float(md.amp), float(md.phase)] for md in modes],
            dtype=np.float64).reshape(-1)
        ptr = ctypes.c_void_p(rec.ctypes.data) if rec.size else None
        self._check(self.lib.fdlbm_init_modes(self._h, rec.size // 4, ptr,
                                              float(mean_velocity[0]), float(mean_velocity[1])),
                    "init_modes")

    def step(self, nsteps: int = 1):
        self._check(self.lib.fdlbm_step(self._h, int(nsteps)), "step")

    def moments(self, out=None):
        """(drho, ux, uy) as float32 CUDA tensors [ny, nx]."""
        import torch
        if out is None:
            out = [torch.empty((self.cfg.ny, self.cfg.nx), dtype=torch.float32,
                               device=self.device) for _ in range(3)]
        self._check(self.lib.fdlbm_moments(self._h, *[self._field(t) for t in out]), "moments")
        return tuple(out)

    def moments_host(self):
        out = [np.empty((self.cfg.ny, self.cfg.nx), dtype=np.float32) for _ in range(3)]
        self._check(self.lib.fdlbm_moments_host(
            self._h, *[ctypes.c_void_p(a.ctypes.data) for a in out]), "moments_host")
        return tuple(out)

    def reduce(self, what: str, args=None) -> np.ndarray:
        out = np.zeros(4, dtype=np.float64)
        a = None
        if args is not None:
            a = np.ascontiguousarray(args, dtype=np.float64)
        rc = self.lib.fdlbm_reduce(self._h, REDUCE[what],
                                   ctypes.c_void_p(a.ctypes.data) if a is not None else None,
                                   ctypes.c_void_p(out.ctypes.data))
        self._check(rc, f"reduce({what})")
        n = 2 if what in ("momentum", "mode", "maxabs") else 1
        return out[:n].copy()

    def sync(self):
        self._check(self.lib.fdlbm_sync(self._h), "sync")

    def selftest_wait_timeout(self, tries: int = 1000):
        """Enqueue the failure-detection self test (a bounded device wait that
        runs out); the next sync() or reduce() raises FdlbmError with status
        ERR_TIMEOUT."""
        self._check(self.lib.fdlbm_selftest_wait_timeout(self._h, int(tries)), "selftest")

    @property
    def launches(self) -> int:
        return int(self.lib.fdlbm_launch_count(self._h))

    def set_stream_plan(self, seg_rows: int = 0, nsegs: int = 0, tail_rows: int = 0):
        """Row segments of the streaming step (fdlbm_set_stream_plan); no
        arguments: back to the model's plan."""
        self._check(self.lib.fdlbm_set_stream_plan(self._h, int(seg_rows), int(nsegs),
                                                   int(tail_rows)), "set_stream_plan")

    def stream_plan(self):
        """The streaming step's plan in use (fdlbm_get_stream_plan) as a dict,
        or None if the lattice has not stepped or does not stream."""
        out = (ctypes.c_int32 * 7)()
        if self.lib.fdlbm_get_stream_plan(self._h, out) != OK:
            return None
        return {"seg_rows": out[0], "nsegs": out[1], "tail_rows": out[2], "ntail": out[3],
                "strips": out[4], "ctas": out[5], "resident_ctas": out[6]}

    _tuned: dict = {}

    def tune(self, steps: int = 10, max_candidates: int = 32):
        """Autotuner over the streaming step's row segments: times `steps`
        steps under each candidate plan of fdlbm_stream_plan_candidates,
        keeps the fastest (cached per device, size, scheme, storage and
        boundary) and returns it as (seg_rows, nsegs, tail_rows) with the
        timings in milliseconds per step; None for a lattice that does not
        run on the streaming kernel.  The lattice's state is saved before and
        restored after (the moments are the whole FD-LBM state), so tuning
        does not advance it."""
        import torch
        cfg = self.cfg
        key = (torch.cuda.get_device_name(self.device), cfg.nx, cfg.ny, cfg.scheme,
               cfg.storage, cfg.boundary)
        if key in Lattice._tuned:
            best, timings = Lattice._tuned[key]
            self.set_stream_plan(*best)
            return best, timings
        saved = [t.clone() for t in self.moments()]
        self.step(1)
        plan = self.stream_plan()
        if plan is None:
            self.init(*saved)
            return None
        cands = stream_plan_candidates(cfg.nx, cfg.ny, cfg.scheme, cfg.storage,
                                       plan["resident_ctas"], max_candidates)
        timings = {}
        for cand in cands:
            self.set_stream_plan(*cand)
            self.step(2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            self.step(steps)
            e1.record(self.stream)
            self.sync()
            timings[cand] = e0.elapsed_time(e1) / steps
        best = min(timings, key=timings.get)
        Lattice._tuned[key] = (best, timings)
        self.set_stream_plan(*best)
        self.init(*saved)
        self.sync()
        return best, timings

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.fdlbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reduce_fields_static(drho, ux, uy, what: str, args=None, out=None, stream=None):
    """fdlbm_reduce_fields_static: FP64 reductions of device fields (float32
    CUDA tensors [ny, nx]) without a handle or workspace.  Returns the device
    tensor `out` (4 doubles: results, 0, count of non-finite nodes); the work
    is asynchronous on `stream` (default: the current stream)."""
    import torch
    lib = load_library()
    ny, nx = drho.shape
    for t in (drho, ux, uy):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                and tuple(t.shape) == (ny, nx)):
            raise ValueError("fields must be contiguous float32 CUDA tensors of one shape")
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=drho.device)
    a = None if args is None else np.ascontiguousarray(args, dtype=np.float64)
    s = stream if stream is not None else torch.cuda.current_stream(drho.device)
    with torch.cuda.device(drho.device):  # the library works on the current device
        rc = lib.fdlbm_reduce_fields_static(
            ctypes.c_void_p(drho.data_ptr()), ctypes.c_void_p(ux.data_ptr()),
            ctypes.c_void_p(uy.data_ptr()), int(nx), int(ny), REDUCE[what],
            ctypes.c_void_p(a.ctypes.data) if a is not None else None,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if rc != OK:
        raise FdlbmError(rc, f"fdlbm_reduce_fields_static({what}): {status_string(rc)}")
    return out


def _mode_records(modes):
    rec = np.ascontiguousarray(
        [[float(md[0]), float(md[1]), float(md[2]), float(md[3])] if not hasattr(md, "m")
         else [float(md.m), float(md.n), float(md.amp), float(md.phase)] for md in modes],
        dtype=np.float64).reshape(-1)
    return rec


class Batch:
    """Many independent lattices stepped together (fdlbm_batch_* in the C ABI).

    Slots take LatticeConfig's of the batch's scheme with FP32 storage, any
    size 16..max_side, periodic or walls in y, each with its own rates and
    force.  The workspace (arena + tables) is a torch uint8 CUDA tensor."""

    # (segment length, narrow last strips) measured best per (device, scheme,
    # size class), with every candidate's time; filled by tune()
    _tuned: dict = {}

    def __init__(self, scheme="fd5", max_lattices=64, arena_bytes=1 << 30, max_side=512,
                 device=None, stream=None):
        import torch
        self.lib = load_library()
        self.scheme = scheme
        self.bp = BatchParams(SCHEMES[scheme], int(max_lattices), int(arena_bytes),
                              int(max_side), 0)
        nbytes = int(self.lib.fdlbm_batch_workspace_size(ctypes.byref(self.bp)))
        if nbytes == 0:
            raise FdlbmError(ERR_INVALID, "invalid batch parameters")
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.fdlbm_batch_create(ctypes.byref(self.bp),
                                             ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                             ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.byref(self._h))
        if rc != OK:
            raise FdlbmError(rc, f"fdlbm_batch_create failed: {status_string(rc)}")
        self.max_lattices = int(max_lattices)
        self.configs = {}

    def _check(self, rc, what):
        if rc != OK:
            msg = self.lib.fdlbm_batch_last_error(self._h).decode()
            raise FdlbmError(rc, f"{what}: {status_string(rc)}: {msg}")

    def add(self, cfg: LatticeConfig) -> int:
        p = cfg.params()
        slot = ctypes.c_int32()
        self._check(self.lib.fdlbm_batch_add(self._h, ctypes.byref(p), ctypes.byref(slot)), "add")
        self.configs[slot.value] = cfg
        return slot.value

    def remove(self, slot: int):
        self._check(self.lib.fdlbm_batch_remove(self._h, int(slot)), "remove")
        self.configs.pop(slot, None)

    def init(self, slot, drho, ux, uy):
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (drho, ux, uy)]
        self._check(self.lib.fdlbm_batch_init(self._h, int(slot), *ptrs), "init")

    def init_modes(self, slot, modes, mean_velocity=(0.0, 0.0)):
        rec = _mode_records(modes)
        ptr = ctypes.c_void_p(rec.ctypes.data) if rec.size else None
        self._check(self.lib.fdlbm_batch_init_modes(self._h, int(slot), rec.size // 4, ptr,
                                                    float(mean_velocity[0]),
                                                    float(mean_velocity[1])), "init_modes")

    def step(self, nsteps: int, slot_steps=None):
        """Advance every slot by nsteps, or slot s by min(slot_steps[s], nsteps)
        (slot_steps: dict slot -> steps or an array of max_lattices counts)."""
        arr = None
        if slot_steps is not None:
            arr = np.zeros(self.max_lattices, dtype=np.int64)
            if isinstance(slot_steps, dict):
                for k, v in slot_steps.items():
                    arr[int(k)] = int(v)
            else:
                arr[:len(slot_steps)] = np.asarray(slot_steps, dtype=np.int64)
        self._check(self.lib.fdlbm_batch_step(
            self._h, int(nsteps), ctypes.c_void_p(arr.ctypes.data) if arr is not None else None),
            "step")

    def moments(self, slot):
        import torch
        cfg = self.configs[slot]
        out = [torch.empty((cfg.ny, cfg.nx), dtype=torch.float32, device=self.device)
               for _ in range(3)]
        self._check(self.lib.fdlbm_batch_moments(
            self._h, int(slot), *[ctypes.c_void_p(t.data_ptr()) for t in out]), "moments")
        return tuple(out)

    def reduce(self, slot, what, args=None):
        out = np.zeros(4, dtype=np.float64)
        a = None if args is None else np.ascontiguousarray(args, dtype=np.float64)
        self._check(self.lib.fdlbm_batch_reduce(
            self._h, int(slot), REDUCE[what], ctypes.c_void_p(a.ctypes.data) if a is not None
            else None, ctypes.c_void_p(out.ctypes.data)), f"reduce({what})")
        n = 2 if what in ("momentum", "mode", "maxabs") else 1
        return out[:n].copy()

    def sync(self):
        self._check(self.lib.fdlbm_batch_sync(self._h), "sync")

    def set_segment_rows(self, rows: int):
        self._check(self.lib.fdlbm_batch_set_segment_rows(self._h, int(rows)), "segment rows")

    def set_grid(self, ctas: int):
        self._check(self.lib.fdlbm_batch_set_grid(self._h, int(ctas)), "grid")

    def set_narrow_strips(self, on: bool):
        self._check(self.lib.fdlbm_batch_set_narrow_strips(self._h, int(bool(on))), "strips")

    @property
    def count(self) -> int:
        return int(self.lib.fdlbm_batch_count(self._h))

    @property
    def launches(self) -> int:
        return int(self.lib.fdlbm_batch_launch_count(self._h))

    def _size_class(self):
        sides = [max(c.nx, c.ny) for c in self.configs.values()] or [0]
        return int(2 ** round(np.log2(max(16, float(np.mean(sides))))))

    def tune(self, steps: int = 8, candidates=(16, 32, 64, 128, 256), strips=(True, False)) -> int:
        """Autotuner over the tile shape: times `steps` steps of the current
        slots for each row-segment length and each form of the lattices' last
        strips (2-column lanes for a last strip of <= 56 columns, or 4-column
        lanes throughout), keeps the fastest pair (cached per device, scheme
        and size class) and returns its segment length.  The slots' states
        advance while tuning: call it before initialising them, or
        re-initialise afterwards."""
        import torch
        key = (torch.cuda.get_device_name(self.device), self.scheme, self._size_class())
        if key in Batch._tuned:
            rows, narrow = Batch._tuned[key][0]
            self.set_segment_rows(rows)
            self.set_narrow_strips(narrow)
            return rows
        timings = {}
        for narrow in strips:
            self.set_narrow_strips(narrow)
            for rows in candidates:
                self.set_segment_rows(rows)
                self.step(1)  # work list and graph for this choice
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                self.step(steps)
                e1.record(self.stream)
                self.sync()
                timings[(rows, narrow)] = e0.elapsed_time(e1) / steps
        best = min(timings, key=timings.get)
        Batch._tuned[key] = (best, timings)
        self.set_segment_rows(best[0])
        self.set_narrow_strips(best[1])
        return best[0]

    @property
    def tuned(self):
        """The autotuner's choice for this batch's size class, (rows, narrow
        strips), or None before tune()."""
        import torch
        key = (torch.cuda.get_device_name(self.device), self.scheme, self._size_class())
        return Batch._tuned.get(key, (None,))[0]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.fdlbm_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
