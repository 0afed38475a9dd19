"""ctypes front end of the FP64 CPU oracle (``sph_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The library in ``paper_1110_3711_gb300``
never imports it.

State arrays are numpy float64 in persistent-id order: ``pos``/``vel`` ``[N, 3]``,
``rho`` ``[N]``; fluid particles come first, then boundary particles.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrParams(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("cell_size", C.c_double),
                ("rho0", C.c_double), ("gamma", C.c_double), ("c0", C.c_double),
                ("alpha", C.c_double), ("eta2_coef", C.c_double), ("cfl", C.c_double),
                ("mass", C.c_double), ("g", C.c_double * 3),
                ("dom_min", C.c_double * 3), ("dom_max", C.c_double * 3),
                ("verlet_euler_every", C.c_int64), ("fixed_dt", C.c_double),
                ("clamp_boundary_rho", C.c_int64), ("tensile_eps", C.c_double),
                ("tensile_pos", C.c_double), ("tensile_n", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER
            d, i64, vp = C.c_double, C.c_int64, C.c_void_p
            pp = P(OrParams)
            L.or_grid.argtypes = [pp, vp]; L.or_grid.restype = C.c_int
            L.or_cells.argtypes = [pp, i64, vp, vp]; L.or_cells.restype = None
            L.or_list.argtypes = [pp, i64, vp, vp, vp]; L.or_list.restype = C.c_int
            L.or_kernel_w.argtypes = [d, d]; L.or_kernel_w.restype = d
            L.or_kernel_f.argtypes = [d, d]; L.or_kernel_f.restype = d
            L.or_pressure.argtypes = [pp, d]; L.or_pressure.restype = d
            L.or_sound.argtypes = [pp, d]; L.or_sound.restype = d
            L.or_pairs.argtypes = [pp, i64, i64, vp, vp, vp, i64, vp]; L.or_pairs.restype = C.c_int
            L.or_interact.argtypes = [pp, i64, i64, vp, vp, vp, vp, vp, vp, vp, C.c_int]
            L.or_interact.restype = i64
            L.or_interact_sampled.argtypes = [pp, i64, i64, vp, vp, vp, vp, vp, vp, vp, C.c_int,
                                              i64, vp]
            L.or_interact_sampled.restype = i64
            L.or_dt.argtypes = [pp, i64, i64, vp, vp, vp, d]; L.or_dt.restype = d
            L.or_update.argtypes = [pp, i64, i64, i64, d, vp, vp, vp, vp, vp, vp, vp]
            L.or_update.restype = None
            L.or_step.argtypes = [pp, i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, C.c_int]
            L.or_step.restype = i64
            L.or_sensor_pressure.argtypes = [pp, i64, vp, vp, i64, vp, vp]
            L.or_sensor_pressure.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def params(p) -> OrParams:
    """Build the oracle's own parameter struct from a ``RunParams``-like object."""
    o = OrParams()
    for name in ("dp", "h", "cell_size", "rho0", "gamma", "c0", "alpha", "eta2_coef",
                 "cfl", "mass", "fixed_dt"):
        setattr(o, name, float(getattr(p, name)))
    for name in ("g", "dom_min", "dom_max"):
        arr = getattr(o, name)
        for k, v in enumerate(getattr(p, name)):
            arr[k] = float(v)
    o.verlet_euler_every = int(p.verlet_euler_every)
    o.clamp_boundary_rho = int(p.clamp_boundary_rho)
    o.tensile_eps = float(getattr(p, "tensile_eps", 0.0))
    o.tensile_pos = float(getattr(p, "tensile_pos", 0.0))
    o.tensile_n = int(getattr(p, "tensile_n", 4))
    return o


def _searchable(p):
    """Parameters for a call that searches neighbours: the oracle visits the 27
    cells around a particle, which hold its whole support only when the cell
    edge is at least 2h."""
    if not p.cell_size >= 2.0 * p.h * (1.0 - 1e-12):
        raise ValueError("oracle neighbour search needs cell_size >= 2h")
    return params(p)


def grid(p):
    dims = np.zeros(3, np.int64)
    rc = lib().or_grid(C.byref(params(p)), _ptr(dims))
    if rc:
        raise ValueError("invalid cell grid")
    return dims


def cells(p, pos):
    pos = np.ascontiguousarray(pos, np.float64)
    out = np.zeros(pos.shape[0], np.int64)
    lib().or_cells(C.byref(params(p)), pos.shape[0], _ptr(pos), _ptr(out))
    return out


def cell_list(p, cell):
    """(order, start) of the stable (cell, id) sort; start has n_cells + 2 entries."""
    dims = grid(p)
    nc = int(dims.prod())
    cell = np.ascontiguousarray(cell, np.int64)
    order = np.zeros(cell.shape[0], np.int64)
    start = np.zeros(nc + 2, np.int64)
    rc = lib().or_list(C.byref(params(p)), cell.shape[0], _ptr(cell), _ptr(order), _ptr(start))
    if rc:
        raise MemoryError("or_list")
    return order, start


def kernel_w(h, r):
    return lib().or_kernel_w(float(h), float(r))


def kernel_f(h, r):
    return lib().or_kernel_f(float(h), float(r))


def pressure(p, rho):
    return lib().or_pressure(C.byref(params(p)), float(rho))


def sound(p, rho):
    return lib().or_sound(C.byref(params(p)), float(rho))


def pairs(p, n_f, n_b, pos, cap=None):
    """All ordered interacting pairs (a, b) found through the cell lists."""
    pos = np.ascontiguousarray(pos, np.float64)
    n = n_f + n_b
    cap = cap or max(1024, n * 200)
    pa = np.zeros(cap, np.int64)
    pb = np.zeros(cap, np.int64)
    cnt = np.zeros(1, np.int64)
    rc = lib().or_pairs(C.byref(_searchable(p)), n_f, n_b, _ptr(pos), _ptr(pa), _ptr(pb), cap, _ptr(cnt))
    if rc:
        raise MemoryError("or_pairs")
    k = int(cnt[0])
    if k > cap:
        return pairs(p, n_f, n_b, pos, cap=k)
    return pa[:k].copy(), pb[:k].copy()


def interact(p, n_f, n_b, pos, vel, rho, nthreads=0):
    """PI: returns (ace [n_f,3], ar [N], viscdt_max, counts[4], n_out)."""
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    n = n_f + n_b
    ace = np.zeros((max(n_f, 1), 3), np.float64)
    ar = np.zeros(max(n, 1), np.float64)
    vm = np.zeros(1, np.float64)
    counts = np.zeros(4, np.int64)
    nout = lib().or_interact(C.byref(_searchable(p)), n_f, n_b, _ptr(pos), _ptr(vel), _ptr(rho),
                             _ptr(ace), _ptr(ar), _ptr(vm), _ptr(counts), int(nthreads))
    if nout < 0:
        raise MemoryError("or_interact")
    return ace[:n_f], ar[:n], float(vm[0]), counts, int(nout)


def interact_sampled(p, n_f, n_b, pos, vel, rho, stride, nthreads=0):
    """PI on every stride-th target; returns (ace, ar, viscdt_max, counts, n_out,
    seconds[2] = list build, interaction loop)."""
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    n = n_f + n_b
    ace = np.zeros((max(n_f, 1), 3), np.float64)
    ar = np.zeros(max(n, 1), np.float64)
    vm = np.zeros(1, np.float64)
    counts = np.zeros(4, np.int64)
    secs = np.zeros(2, np.float64)
    nout = lib().or_interact_sampled(C.byref(_searchable(p)), n_f, n_b, _ptr(pos), _ptr(vel), _ptr(rho),
                                     _ptr(ace), _ptr(ar), _ptr(vm), _ptr(counts), int(nthreads),
                                     int(stride), _ptr(secs))
    if nout < 0:
        raise MemoryError("or_interact_sampled")
    return ace[:n_f], ar[:n], float(vm[0]), counts, int(nout), secs


def update(p, n_f, n_b, step, dt, pos, vel, velm1, rho, rhom1, ace, ar):
    """SU in place on the given arrays."""
    ace = np.ascontiguousarray(ace, np.float64).reshape(-1)
    if ace.size == 0:
        ace = np.zeros(3, np.float64)
    for a in (pos, vel, velm1, rho, rhom1):
        assert a.flags["C_CONTIGUOUS"] and a.dtype == np.float64
    lib().or_update(C.byref(params(p)), n_f, n_b, int(step), float(dt), _ptr(pos), _ptr(vel),
                    _ptr(velm1), _ptr(rho), _ptr(rhom1), _ptr(ace),
                    _ptr(np.ascontiguousarray(ar, np.float64)))


def time_step(p, n_f, n_b, pos, ace, rho, viscdt_max):
    pos = np.ascontiguousarray(pos, np.float64)
    ace = np.ascontiguousarray(ace, np.float64).reshape(-1)
    if ace.size == 0:
        ace = np.zeros(3, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    return lib().or_dt(C.byref(params(p)), n_f, n_b, _ptr(pos), _ptr(ace), _ptr(rho),
                       float(viscdt_max))


class State:
    """Oracle state in persistent-id order (fluid first, then boundary)."""

    def __init__(self, case, *, params_override=None):
        self.p = params_override or case.params
        self.n_f, self.n_b = case.n_f, case.n_b
        self.pos = np.array(case.pos, np.float64, copy=True)
        self.vel = np.array(case.vel, np.float64, copy=True)
        self.velm1 = self.vel.copy()
        self.rho = np.array(case.rho, np.float64, copy=True)
        self.rhom1 = self.rho.copy()
        self.step_index = 0
        self.time = 0.0
        self.last_counts = np.zeros(4, np.int64)
        self.n_out = 0

    def step(self, nthreads=0):
        """One NL -> PI -> SU step; returns dt."""
        dt = np.zeros(1, np.float64)
        counts = np.zeros(4, np.int64)
        nout = lib().or_step(C.byref(_searchable(self.p)), self.n_f, self.n_b, self.step_index,
                             _ptr(self.pos), _ptr(self.vel), _ptr(self.velm1),
                             _ptr(self.rho), _ptr(self.rhom1), _ptr(dt), _ptr(counts),
                             int(nthreads))
        if nout < 0:
            raise MemoryError("or_step")
        self.n_out = int(nout)
        self.last_counts = counts
        self.step_index += 1
        self.time += float(dt[0])
        return float(dt[0])

    def run(self, steps, nthreads=0):
        return [self.step(nthreads) for _ in range(steps)]

    def copy(self):
        o = State.__new__(State)
        o.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                           for k, v in self.__dict__.items()})
        return o


def sensor_pressure(p, n_f, pos, rho, spos):
    pos = np.ascontiguousarray(pos, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    spos = np.ascontiguousarray(spos, np.float64)
    out = np.zeros(spos.shape[0], np.float64)
    lib().or_sensor_pressure(C.byref(_searchable(p)), n_f, _ptr(pos), _ptr(rho), spos.shape[0],
                             _ptr(spos), _ptr(out))
    return out
