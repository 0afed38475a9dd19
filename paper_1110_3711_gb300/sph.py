"""Python binding of libsph (``include/sph.h``): the same calls, argument
marshalling only.  Every stage of the time step runs in the CUDA kernels of
``csrc/``; there is no CPU path.  Loading fails loudly when the shared library
has not been built (``paper_1110_3711_gb300.build.build()``).

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); particle
arrays are float64 in persistent-id order, fluid first.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

SPH_FP64 = 0
SPH_FP32_SPLIT = 1
PRECISIONS = {"fp64": SPH_FP64, "fp32": SPH_FP32_SPLIT, "fp32_split": SPH_FP32_SPLIT}
PI_KERNELS = {"warp": 0, "thread": 1, "thread_fastcells": 2, "warp_sym": 3}
FLAG_OUT_OF_GRID = 1
FLAG_NAN = 2
FLAG_DT_TOO_SMALL = 4

_lock = threading.Lock()
_lib = None


class SphError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = lib().sph_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})")


class sph_params(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("cell_size", C.c_double),
                ("rho0", C.c_double), ("gamma", C.c_double), ("c0", C.c_double),
                ("alpha", C.c_double), ("eta2_coef", C.c_double), ("cfl", C.c_double),
                ("mass", C.c_double), ("g", C.c_double * 3), ("dom_min", C.c_double * 3),
                ("dom_max", C.c_double * 3), ("verlet_euler_every", C.c_int64),
                ("fixed_dt", C.c_double), ("clamp_boundary_rho", C.c_int64),
                ("precision", C.c_int32), ("pi_kernel", C.c_int32),
                ("tensile_eps", C.c_double), ("tensile_pos", C.c_double),
                ("tensile_n", C.c_int64)]


def make_params(run_params, precision, pi_kernel="warp") -> sph_params:
    """Fill ``sph_params`` from any object with the same field names."""
    prec = PRECISIONS.get(precision, precision)
    p = sph_params()
    for name in ("dp", "h", "cell_size", "rho0", "gamma", "c0", "alpha", "eta2_coef", "cfl",
                 "mass", "fixed_dt"):
        setattr(p, name, float(getattr(run_params, name)))
    for name in ("g", "dom_min", "dom_max"):
        arr = getattr(p, name)
        for k, v in enumerate(getattr(run_params, name)):
            arr[k] = float(v)
    p.verlet_euler_every = int(run_params.verlet_euler_every)
    p.clamp_boundary_rho = int(run_params.clamp_boundary_rho)
    p.precision = int(prec)
    p.pi_kernel = int(PI_KERNELS.get(pi_kernel, pi_kernel))
    p.tensile_eps = float(getattr(run_params, "tensile_eps", 0.0))
    p.tensile_pos = float(getattr(run_params, "tensile_pos", 0.0))
    p.tensile_n = int(getattr(run_params, "tensile_n", 4))
    return p


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libsph.so; raises if it was not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libsph.so not built ({path}); run "
                                   "paper_1110_3711_gb300.build.build() first")
            L = C.CDLL(path)
            vp, i64, i32, sz = C.c_void_p, C.c_int64, C.c_int, C.c_size_t
            pp = C.POINTER(sph_params)
            sig = {
                "sph_workspace_bytes": ([pp, i64, i64, C.POINTER(sz)], i32),
                "sph_create": ([pp, i64, i64, vp, vp, vp, vp, sz, vp, C.POINTER(vp)], i32),
                "sph_neighbour_list": ([vp], i32),
                "sph_interact": ([vp], i32),
                "sph_update": ([vp, vp], i32),
                "sph_run": ([vp, i64], i32),
                "sph_run_graph": ([vp, i64], i32),
                "sph_get_state": ([vp, vp, vp, vp, vp, vp], i32),
                "sph_set_state": ([vp, vp, vp, vp, vp, vp], i32),
                "sph_get_time": ([vp, vp, vp, vp], i32),
                "sph_status": ([vp, vp, i32], i32),
                "sph_get_neighbour_list": ([vp, vp, vp, vp], i32),
                "sph_get_grid": ([vp, vp], i32),
                "sph_get_forces": ([vp, vp, vp, vp], i32),
                "sph_count_work": ([vp, vp], i32),
                "sph_launch_count": ([vp], i64),
                "sph_checkpoint_bytes": ([vp, C.POINTER(sz)], i32),
                "sph_save_state": ([vp, vp], i32),
                "sph_load_state": ([vp, vp], i32),
                "sph_neighbour_list_static": ([pp, i64, vp, vp, vp, vp, vp], i32),
                "sph_fma_rate": ([i32, vp, vp, C.POINTER(C.c_double)], i32),
                "sph_sensor_pressure": ([vp, vp, i64, vp], i32),
                "sph_sensor_adjoint": ([vp, vp, i64, vp, vp], i32),
                "sph_front_position": ([vp, C.c_double, vp], i32),
                "sph_front_adjoint": ([vp, C.c_double, C.c_double, vp], i32),
                "sph_adjoint_step": ([vp, vp, vp, vp], i32),
                "sph_error_string": ([i32], C.c_char_p),
                "sph_destroy": ([vp], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def exported_symbols():
    """Names the binding expects the library to export (all of include/sph.h)."""
    return ["sph_workspace_bytes", "sph_create", "sph_neighbour_list", "sph_interact",
            "sph_update", "sph_run", "sph_run_graph", "sph_get_state", "sph_set_state", "sph_get_time",
            "sph_status", "sph_get_neighbour_list", "sph_get_grid", "sph_get_forces",
            "sph_count_work", "sph_launch_count", "sph_checkpoint_bytes", "sph_save_state",
            "sph_load_state", "sph_neighbour_list_static", "sph_sensor_pressure",
            "sph_sensor_adjoint", "sph_front_position", "sph_front_adjoint", "sph_adjoint_step",
            "sph_fma_rate", "sph_error_string", "sph_destroy"]


def _check(code, what):
    if code != 0:
        raise SphError(code, what)


def _ptr(a, dtype=None, count=None, writable=False):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        if count is not None and a.size != count:
            raise ValueError(f"expected {count} elements, got {a.size}")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("array is read-only")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None:
            tdt = {np.float64: torch.float64, np.uint32: torch.uint32 if hasattr(torch, "uint32") else torch.int32,
                   np.int32: torch.int32, np.uint8: torch.uint8}.get(np.dtype(dtype).type)
            if tdt is not None and a.dtype != tdt and a.element_size() != np.dtype(dtype).itemsize:
                raise TypeError(f"expected {dtype}, got {a.dtype}")
        if count is not None and a.numel() != count:
            raise ValueError(f"expected {count} elements, got {a.numel()}")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


# ---------------------------------------------------------------- raw calls --

def sph_workspace_bytes(p: sph_params, n_f: int, n_b: int) -> int:
    out = C.c_size_t(0)
    _check(lib().sph_workspace_bytes(C.byref(p), n_f, n_b, C.byref(out)), "sph_workspace_bytes")
    return out.value


def sph_create(p: sph_params, n_f, n_b, pos, vel, rho, workspace, ws_bytes, stream):
    n = n_f + n_b
    h = C.c_void_p()
    _check(lib().sph_create(C.byref(p), n_f, n_b, _ptr(pos, np.float64, 3 * n),
                            _ptr(vel, np.float64, 3 * n), _ptr(rho, np.float64, n),
                            _ptr(workspace), ws_bytes, stream, C.byref(h)), "sph_create")
    return h


def sph_neighbour_list(ctx):
    _check(lib().sph_neighbour_list(ctx), "sph_neighbour_list")


def sph_interact(ctx):
    _check(lib().sph_interact(ctx), "sph_interact")


def sph_update(ctx, want_dt=False):
    if want_dt:
        dt = C.c_double(0.0)
        _check(lib().sph_update(ctx, C.byref(dt)), "sph_update")
        return dt.value
    _check(lib().sph_update(ctx, None), "sph_update")
    return None


def sph_run(ctx, n_steps):
    _check(lib().sph_run(ctx, int(n_steps)), "sph_run")


def sph_run_graph(ctx, n_steps):
    _check(lib().sph_run_graph(ctx, int(n_steps)), "sph_run_graph")


def sph_get_state(ctx, n, pos=None, vel=None, rho=None, vel_prev=None, rho_prev=None):
    _check(lib().sph_get_state(ctx, _ptr(pos, np.float64, 3 * n, True),
                               _ptr(vel, np.float64, 3 * n, True), _ptr(rho, np.float64, n, True),
                               _ptr(vel_prev, np.float64, 3 * n, True),
                               _ptr(rho_prev, np.float64, n, True)), "sph_get_state")


def sph_set_state(ctx, n, pos, vel, rho, vel_prev=None, rho_prev=None):
    _check(lib().sph_set_state(ctx, _ptr(pos, np.float64, 3 * n), _ptr(vel, np.float64, 3 * n),
                               _ptr(rho, np.float64, n), _ptr(vel_prev, np.float64, 3 * n),
                               _ptr(rho_prev, np.float64, n)), "sph_set_state")


def sph_get_time(ctx):
    t, dt, st = C.c_double(), C.c_double(), C.c_int64()
    _check(lib().sph_get_time(ctx, C.byref(t), C.byref(dt), C.byref(st)), "sph_get_time")
    return t.value, dt.value, st.value


def sph_status(ctx, clear=False):
    f = C.c_uint32(0)
    _check(lib().sph_status(ctx, C.byref(f), 1 if clear else 0), "sph_status")
    return f.value


def sph_get_grid(ctx):
    d = np.zeros(3, np.int64)
    _check(lib().sph_get_grid(ctx, d.ctypes.data), "sph_get_grid")
    return d


def sph_get_neighbour_list(ctx, n_f):
    dims = sph_get_grid(ctx)
    nc = int(dims.prod())
    ids = np.zeros(n_f, np.uint32)
    cell = np.zeros(n_f, np.uint32)
    start = np.zeros(nc + 2, np.int32)
    _check(lib().sph_get_neighbour_list(ctx, ids.ctypes.data, cell.ctypes.data,
                                        start.ctypes.data), "sph_get_neighbour_list")
    return ids, cell, start


def sph_get_forces(ctx, n_f, n_b):
    ace = np.zeros((n_f, 3), np.float64)
    ar = np.zeros(n_f + n_b, np.float64)
    mx = np.zeros(3, np.float64)
    _check(lib().sph_get_forces(ctx, ace.ctypes.data, ar.ctypes.data, mx.ctypes.data),
           "sph_get_forces")
    return ace, ar, mx


def sph_count_work(ctx):
    c = np.zeros(4, np.int64)
    _check(lib().sph_count_work(ctx, c.ctypes.data), "sph_count_work")
    return c


def sph_launch_count(ctx) -> int:
    return int(lib().sph_launch_count(ctx))


def sph_checkpoint_bytes(ctx) -> int:
    out = C.c_size_t(0)
    _check(lib().sph_checkpoint_bytes(ctx, C.byref(out)), "sph_checkpoint_bytes")
    return out.value


def sph_save_state(ctx, dst):
    _check(lib().sph_save_state(ctx, _ptr(dst)), "sph_save_state")


def sph_load_state(ctx, src):
    _check(lib().sph_load_state(ctx, _ptr(src)), "sph_load_state")


def sph_sensor_pressure(ctx, sensors, n_sensors, out):
    _check(lib().sph_sensor_pressure(ctx, _ptr(sensors), int(n_sensors), _ptr(out)),
           "sph_sensor_pressure")


def sph_sensor_adjoint(ctx, sensors, n_sensors, dj_dp, lam):
    _check(lib().sph_sensor_adjoint(ctx, _ptr(sensors), int(n_sensors), _ptr(dj_dp), _ptr(lam)),
           "sph_sensor_adjoint")


def sph_front_position(ctx, tau, out):
    _check(lib().sph_front_position(ctx, float(tau), _ptr(out)), "sph_front_position")


def sph_front_adjoint(ctx, tau, dj, lam):
    _check(lib().sph_front_adjoint(ctx, float(tau), float(dj), _ptr(lam)), "sph_front_adjoint")


def sph_adjoint_step(ctx, lam_next, lam, dalpha):
    _check(lib().sph_adjoint_step(ctx, _ptr(lam_next), _ptr(lam), _ptr(dalpha)),
           "sph_adjoint_step")


STATIC_MAX_POINTS = 524288
STATIC_MAX_CELLS = 16777216


def static_grid_cells(p: sph_params) -> int:
    """Number of cells of the grid that sph_neighbour_list_static builds for p
    (ceil(span / cell_size) per axis), i.e. cell_start holds this + 2 entries."""
    n = 1
    for d in range(3):
        n *= int(math.ceil((p.dom_max[d] - p.dom_min[d]) / p.cell_size))
    return n


def sph_neighbour_list_static(p: sph_params, n, pos, sorted_id, cell, cell_start, stream=None):
    """Neighbour list of n points with no device allocation (see include/sph.h):
    pos and the three outputs are CUDA tensors the caller owns, of exactly
    the sizes the call reads and writes (float64 [n][3]; 32-bit [n], [n];
    int32 [n_cells + 2])."""
    import torch
    n = int(n)
    if n < 0:
        raise ValueError("n must be >= 0")
    bufs = {"pos": pos, "sorted_id": sorted_id, "cell": cell, "cell_start": cell_start}
    for name, t in bufs.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
    if pos.dtype != torch.float64:
        raise TypeError(f"pos must be float64, got {pos.dtype}")
    u32 = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())
    for name in ("sorted_id", "cell"):
        if bufs[name].dtype not in u32:
            raise TypeError(f"{name} must be a 32-bit integer tensor, got {bufs[name].dtype}")
    if cell_start.dtype != torch.int32:
        raise TypeError(f"cell_start must be int32, got {cell_start.dtype}")
    ncells = static_grid_cells(p)
    _check(lib().sph_neighbour_list_static(C.byref(p), n, _ptr(pos, np.float64, 3 * n),
                                           _ptr(sorted_id, np.uint32, n), _ptr(cell, np.uint32, n),
                                           _ptr(cell_start, np.int32, ncells + 2), stream),
           "sph_neighbour_list_static")


def sph_fma_rate(precision, scratch, stream=None):
    """Measured rate (FLOP/s, 2 per FMA) of float32 ("fp32") or float64
    ("fp64") fused multiply-adds on the current device; scratch is a device
    buffer of at least 8 bytes."""
    out = C.c_double(0.0)
    code = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().sph_fma_rate(code, _ptr(scratch), stream, C.byref(out)), "sph_fma_rate")
    return out.value


def sph_destroy(ctx):
    if ctx:
        lib().sph_destroy(ctx)


# ------------------------------------------------------------ convenience --

class Simulation:
    """One context with a torch-allocated device workspace on torch's current
    stream (or a given one).  Memory and streams come from torch; every stage
    runs in libsph."""

    def __init__(self, run_params, n_f, n_b, pos, vel, rho, precision="fp32", device=None,
                 stream=None, pi_kernel="warp"):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.params = make_params(run_params, precision, pi_kernel)
        self.n_f, self.n_b = int(n_f), int(n_b)
        self.n = self.n_f + self.n_b
        self.ws_bytes = sph_workspace_bytes(self.params, self.n_f, self.n_b)
        with torch.cuda.device(self.device):
            raw = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        off = (-raw.data_ptr()) % 256
        self._raw = raw
        self.workspace = raw[off:off + self.ws_bytes]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        pos = np.ascontiguousarray(pos, np.float64) if isinstance(pos, np.ndarray) else pos
        vel = np.ascontiguousarray(vel, np.float64) if isinstance(vel, np.ndarray) else vel
        rho = np.ascontiguousarray(rho, np.float64) if isinstance(rho, np.ndarray) else rho
        with torch.cuda.device(self.device):
            self.ctx = sph_create(self.params, self.n_f, self.n_b, pos, vel, rho,
                                  self.workspace.data_ptr(), self.ws_bytes,
                                  self.stream.cuda_stream)

    @classmethod
    def from_case(cls, case, precision="fp32", **kw):
        return cls(case.params, case.n_f, case.n_b, case.pos, case.vel, case.rho,
                   precision=precision, **kw)

    def neighbour_list(self):
        sph_neighbour_list(self.ctx)

    def interact(self):
        sph_interact(self.ctx)

    def update(self, want_dt=False):
        return sph_update(self.ctx, want_dt)

    def step(self, want_dt=False):
        sph_neighbour_list(self.ctx)
        sph_interact(self.ctx)
        return sph_update(self.ctx, want_dt)

    def run(self, n_steps):
        sph_run(self.ctx, n_steps)

    def run_graph(self, n_steps):
        sph_run_graph(self.ctx, n_steps)

    def get_state(self, with_prev=False):
        n = self.n
        pos = np.zeros((n, 3)); vel = np.zeros((n, 3)); rho = np.zeros(n)
        vp = np.zeros((n, 3)) if with_prev else None
        rp = np.zeros(n) if with_prev else None
        sph_get_state(self.ctx, n, pos, vel, rho, vp, rp)
        return (pos, vel, rho, vp, rp) if with_prev else (pos, vel, rho)

    def set_state(self, pos, vel, rho, vel_prev=None, rho_prev=None):
        sph_set_state(self.ctx, self.n, pos, vel, rho, vel_prev, rho_prev)

    def time(self):
        return sph_get_time(self.ctx)

    def status(self, clear=False):
        return sph_status(self.ctx, clear)

    def grid(self):
        return sph_get_grid(self.ctx)

    def neighbour_list_arrays(self):
        return sph_get_neighbour_list(self.ctx, self.n_f)

    def forces(self):
        return sph_get_forces(self.ctx, self.n_f, self.n_b)

    def count_work(self):
        return sph_count_work(self.ctx)

    @property
    def launches(self):
        return sph_launch_count(self.ctx)

    def checkpoint_bytes(self):
        return sph_checkpoint_bytes(self.ctx)

    def save_state(self, dst):
        sph_save_state(self.ctx, dst)

    def load_state(self, src):
        sph_load_state(self.ctx, src)

    def close(self):
        if getattr(self, "ctx", None):
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
