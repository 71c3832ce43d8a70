"""Plain FP64 CPU oracle of the RiemannProblem fluid step (Sec. 3, Algorithm 1).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package; the
product library never does.  It shares no code with the CUDA path.

The arithmetic lives in ``fv_oracle.c`` (plain C, compiled with
``-O2 -ffp-contract=off``); this module only compiles it on first use and
marshals numpy arrays.  States are ghosted arrays of shape
``(5, nz+4, ny+4, nx+4)`` (rho, rho*vx, rho*vy, rho*vz, E), x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "fv_oracle.c"), os.path.join(_HERE, "fv_oracle.h")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_fv.so")
_lock = threading.Lock()
_lib = None

BC_OUTFLOW = 0
BC_PERIODIC = 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle_fv.so`` (gcc)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    newest_src = max(os.path.getmtime(p) for p in _SRC)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= newest_src):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("gamma", ctypes.c_double), ("theta", ctypes.c_double),
                ("bc", ctypes.c_int * 3)]


def mesh(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, gamma=1.4, theta=2.0,
         bc=(BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW)) -> Mesh:
    m = Mesh()
    m.nx, m.ny, m.nz = int(nx), int(ny), int(nz)
    m.lx, m.ly, m.lz = float(lx), float(ly), float(lz)
    m.gamma, m.theta = float(gamma), float(theta)
    for a in range(3):
        m.bc[a] = int(bc[a])
    return m


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # a test may point this at a deliberately mutated copy of the
            # oracle to check that the pins catch planted mistakes
            path = os.environ.get("ORACLE_LIB_OVERRIDE") or build()
            lib = ctypes.CDLL(path)
            MP = ctypes.POINTER(Mesh)
            lib.orc_field_size.argtypes = [MP]
            lib.orc_field_size.restype = ctypes.c_size_t
            lib.orc_fill_ghosts.argtypes = [MP, _D]
            lib.orc_fill_ghosts.restype = None
            lib.orc_cons_to_prim.argtypes = [ctypes.c_double, _D, _D]
            lib.orc_prim_to_cons.argtypes = [ctypes.c_double, _D, _D]
            lib.orc_minmod3.argtypes = [ctypes.c_double] * 3
            lib.orc_minmod3.restype = ctypes.c_double
            lib.orc_limited_slope.argtypes = [ctypes.c_double] * 3
            lib.orc_limited_slope.restype = ctypes.c_double
            lib.orc_hll_flux.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D, _D]
            lib.orc_hll_flux.restype = None
            lib.orc_reduce_dt.argtypes = [MP, _D, ctypes.c_double, _D, _D]
            lib.orc_reduce_dt.restype = ctypes.c_long
            lib.orc_compute_update.argtypes = [MP, _D, ctypes.c_double, _D,
                                               ctypes.POINTER(ctypes.c_long)]
            lib.orc_compute_update.restype = ctypes.c_long
            lib.orc_step.argtypes = [MP, _D, ctypes.c_double, ctypes.POINTER(ctypes.c_long)]
            lib.orc_step.restype = ctypes.c_long
            lib.orc_conserved_sums.argtypes = [MP, _D, _D]
            lib.orc_conserved_sums.restype = None
            lib.orc_pairwise_sum.argtypes = [_D, ctypes.c_size_t]
            lib.orc_pairwise_sum.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _check_state(m: Mesh, U: np.ndarray):
    shape = (5, m.nz + 4, m.ny + 4, m.nx + 4)
    if U.shape != shape or U.dtype != np.float64 or not U.flags["C_CONTIGUOUS"]:
        raise ValueError(f"state must be C-contiguous float64 {shape}, got {U.shape} {U.dtype}")


def ghosted_from_interior(m: Mesh, interior: np.ndarray) -> np.ndarray:
    """Embed a (5, nz, ny, nx) interior state in a ghosted array and fill ghosts."""
    U = np.zeros((5, m.nz + 4, m.ny + 4, m.nx + 4))
    U[:, 2:-2, 2:-2, 2:-2] = interior
    fill_ghosts(m, U)
    return U


def interior(U: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(U[:, 2:-2, 2:-2, 2:-2])


def fill_ghosts(m: Mesh, U: np.ndarray) -> None:
    _check_state(m, U)
    _load().orc_fill_ghosts(ctypes.byref(m), _ptr(U))


def cons_to_prim(gamma: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.empty(5)
    _load().orc_cons_to_prim(gamma, _ptr(u), _ptr(w))
    return w


def prim_to_cons(gamma: float, w) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.empty(5)
    _load().orc_prim_to_cons(gamma, _ptr(w), _ptr(u))
    return u


def minmod3(a, b, c) -> float:
    return _load().orc_minmod3(a, b, c)


def limited_slope(theta, d_minus, d_plus) -> float:
    return _load().orc_limited_slope(theta, d_minus, d_plus)


def hll_flux(axis: int, gamma: float, wl, wr) -> np.ndarray:
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.empty(5)
    _load().orc_hll_flux(axis, gamma, _ptr(wl), _ptr(wr), _ptr(f))
    return f


def reduce_dt(m: Mesh, U: np.ndarray, cfl: float):
    """Returns (dt, smax, n_nonphysical)."""
    _check_state(m, U)
    dt = ctypes.c_double()
    smax = ctypes.c_double()
    bad = _load().orc_reduce_dt(ctypes.byref(m), _ptr(U), cfl, ctypes.byref(dt),
                                ctypes.byref(smax))
    return dt.value, smax.value, bad


def compute_update(m: Mesh, U: np.ndarray, dt: float):
    """Returns (dU, n_nonphysical, n_face_fallback) for one substep."""
    _check_state(m, U)
    dU = np.empty_like(U)
    fb = ctypes.c_long()
    bad = _load().orc_compute_update(ctypes.byref(m), _ptr(U), dt, _ptr(dU), ctypes.byref(fb))
    return dU, bad, fb.value


def step(m: Mesh, U: np.ndarray, dt: float):
    """One RK2 step in place; returns (n_nonphysical, n_face_fallback)."""
    _check_state(m, U)
    fb = ctypes.c_long()
    bad = _load().orc_step(ctypes.byref(m), _ptr(U), dt, ctypes.byref(fb))
    return bad, fb.value


def conserved_sums(m: Mesh, U: np.ndarray) -> np.ndarray:
    _check_state(m, U)
    out = np.empty(5)
    _load().orc_conserved_sums(ctypes.byref(m), _ptr(U), _ptr(out))
    return out


def pairwise_sum(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _load().orc_pairwise_sum(_ptr(v), v.size)


def evolve(m: Mesh, U: np.ndarray, cfl: float, t_end: float | None = None,
           nsteps: int | None = None):
    """Algorithm 1's time loop: dt = min(ComputeTimeStep, t_end - t); step.

    Stops at t_end or after nsteps steps, whichever comes first.  Returns
    (t, steps_taken, dts)."""
    t, n, dts = 0.0, 0, []
    while True:
        if t_end is not None and not t < t_end:
            break
        if nsteps is not None and n >= nsteps:
            break
        dt, _, bad = reduce_dt(m, U, cfl)
        if bad:
            raise FloatingPointError(f"non-physical state before step {n}")
        if t_end is not None and dt > t_end - t:
            dt = t_end - t
        bad, _ = step(m, U, dt)
        if bad:
            raise FloatingPointError(f"non-physical state in step {n}")
        dts.append(dt)
        t += dt
        n += 1
    return t, n, dts
