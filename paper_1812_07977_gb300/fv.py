"""Python binding of the C ABI in include/fv.h (argument marshalling only).

Every stage of the step runs in the CUDA kernels of ``libfvgb.so``; this
module converts arguments, checks shapes and raises :class:`FvError` on a
non-OK status.  It never computes anything itself and has no CPU path: if
the library is missing it raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfvgb.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_BAD_HANDLE = range(7)
BC = {"outflow": 0, "periodic": 1}
PRECISION = {"fp64": 0, "fp32_bulk": 1, "fp64_fma": 2, "fp64_ff": 3}

# Every entry point declared in include/fv.h.
ABI_SYMBOLS = (
    "fv_create_mesh", "fv_destroy_mesh", "fv_set_state", "fv_get_state",
    "fv_get_ghosted_state", "fv_reduce_dt", "fv_step", "fv_substep", "fv_fill_ghosts",
    "fv_conserved_sums", "fv_get_counters", "fv_get_face_counts", "fv_set_tuning",
    "fv_profile_enable",
    "fv_profile_read",
    "fv_mesh_info", "fv_status_string", "fv_last_error", "fv_conserved_sums_noalloc",
    "fv_batch_create", "fv_batch_destroy", "fv_batch_set_state", "fv_batch_get_state",
    "fv_batch_step", "fv_batch_get_dt", "fv_batch_set_tuning", "fv_batch_autotune",
    "fv_batch_get_counters", "fv_batch_info", "fv_batch_set_class_tuning",
    "fv_batch_get_class_tuning",
    "fv_net_param_count", "fv_net_create", "fv_net_destroy", "fv_net_set_params",
    "fv_net_get_params", "fv_net_set_scales", "fv_net_forward", "fv_net_train_step",
    "fv_net_take_loss",
    "fv_step_learned", "fv_net_get_buffer",
)
KERNEL_CLASSES = ("prim", "sweep_x", "sweep_y", "sweep_z", "fused", "ghost", "dt", "other")


class FvError(RuntimeError):
    def __init__(self, status: int, call: str, detail: str):
        self.status = status
        super().__init__(f"{call}: {_status_name(status)}: {detail}")


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("gamma", ctypes.c_double), ("theta", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("precision", ctypes.c_int)]


_lib = None


# fv_tuning_key (include/fv.h) by short name
TUNING_KEYS = {"kchunk": 0, "vacuum_ratio": 1, "occupancy": 2, "sweep_segments": 3,
               "tile_y": 4, "fp64_fused": 5, "tile_x": 6, "plane_skip": 7}


def load_library(path: str | None = None):
    """Load libfvgb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CUDA library {p} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, dp, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    d = ctypes.c_double
    sig = {
        "fv_create_mesh": ([ctypes.POINTER(MeshDesc), vp, ctypes.POINTER(vp)], i),
        "fv_destroy_mesh": ([vp], i),
        "fv_set_state": ([vp, vp, i], i),
        "fv_get_state": ([vp, vp, i], i),
        "fv_get_ghosted_state": ([vp, vp, i], i),
        "fv_reduce_dt": ([vp, d, dp], i),
        "fv_step": ([vp, d], i),
        "fv_substep": ([vp, i, d], i),
        "fv_fill_ghosts": ([vp], i),
        "fv_conserved_sums": ([vp, dp], i),
        "fv_get_counters": ([vp, ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong)], i),
        "fv_get_face_counts": ([vp, ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_longlong)], i),
        "fv_set_tuning": ([vp, i, d], i),
        "fv_profile_enable": ([vp, i], i),
        "fv_profile_read": ([vp, dp, ctypes.POINTER(ctypes.c_longlong)], i),
        "fv_mesh_info": ([vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)], i),
        "fv_conserved_sums_noalloc": ([vp, i, i, i, d, d, d, vp, dp], i),
        "fv_batch_create": ([ctypes.POINTER(MeshDesc), i, vp, ctypes.POINTER(vp)], i),
        "fv_batch_destroy": ([vp], i),
        "fv_batch_set_state": ([vp, i, vp, i], i),
        "fv_batch_get_state": ([vp, i, vp, i], i),
        "fv_batch_step": ([vp, d, i], i),
        "fv_batch_get_dt": ([vp, dp], i),
        "fv_batch_set_tuning": ([vp, i, i, i], i),
        "fv_batch_autotune": ([vp, d, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                               dp], i),
        "fv_batch_set_class_tuning": ([vp, i, i, i, i, i], i),
        "fv_batch_get_class_tuning": ([vp, i] + [ctypes.POINTER(i)] * 5, i),
        "fv_batch_get_counters": ([vp, ctypes.POINTER(ctypes.c_longlong),
                                   ctypes.POINTER(ctypes.c_longlong)], i),
        "fv_batch_info": ([vp, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong),
                           ctypes.POINTER(ctypes.c_longlong)], i),
        "fv_net_param_count": ([], ctypes.c_size_t),
        "fv_net_create": ([ctypes.POINTER(vp)], i),
        "fv_net_destroy": ([vp], i),
        "fv_net_set_params": ([vp, vp], i),
        "fv_net_get_params": ([vp, vp, vp], i),
        "fv_net_set_scales": ([vp, dp, dp, dp, dp], i),
        "fv_net_forward": ([vp, vp, vp], i),
        "fv_net_train_step": ([vp, vp, vp, d, d, dp], i),
        "fv_net_take_loss": ([vp, dp, ctypes.POINTER(ctypes.c_longlong)], i),
        "fv_step_learned": ([vp, vp, d], i),
        "fv_net_get_buffer": ([vp, i, vp, ctypes.c_size_t], i),
        "fv_status_string": ([i], ctypes.c_char_p),
        "fv_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


def _status_name(s: int) -> str:
    names = ["FV_OK", "FV_ERR_INVALID_ARG", "FV_ERR_OOM", "FV_ERR_CUDA",
             "FV_ERR_NONPHYSICAL", "FV_ERR_TIMEOUT", "FV_ERR_BAD_HANDLE"]
    return names[s] if 0 <= s < len(names) else f"status {s}"


def _check(status: int, call: str):
    if status != OK:
        raise FvError(status, call, load_library().fv_last_error().decode())


def _torch():
    import torch
    return torch


class Mesh:
    """One mesh of the RK2 finite-volume step on the current CUDA device.

    States are (5, nz, ny, nx) float64 arrays of conserved variables
    (rho, rho*vx, rho*vy, rho*vz, E): torch CUDA tensors are passed by
    device pointer, numpy arrays / CPU tensors through host memory.
    """

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, gamma=1.4, theta=2.0,
                 bc=("outflow", "outflow", "outflow"), precision="fp64", stream=None):
        self._lib = load_library()
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        d = MeshDesc()
        d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
        d.lx, d.ly, d.lz = float(lx), float(ly), float(lz)
        d.gamma, d.theta = float(gamma), float(theta)
        for a in range(3):
            d.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
        d.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self.desc = d
        self.shape = (5, d.nz, d.ny, d.nx)
        self.ghosted_shape = (5, d.nz + 4, d.ny + 4, d.nx + 4)
        self.device = torch.cuda.current_device()
        h = ctypes.c_void_p()
        _check(self._lib.fv_create_mesh(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                                        ctypes.byref(h)), "fv_create_mesh")
        self._h = h

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(self._lib.fv_destroy_mesh(self._h), "fv_destroy_mesh")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- state
    def _buffer(self, U, shape, writable):
        torch = _torch()
        if isinstance(U, torch.Tensor):
            if tuple(U.shape) != shape or U.dtype != torch.float64 or not U.is_contiguous():
                raise ValueError(f"expected a contiguous float64 tensor of shape {shape}")
            if U.is_cuda:
                # the library reads/writes U on its own stream, asynchronously:
                # order it after the work queued on the caller's stream and keep
                # the tensor's memory from being reused before that work is done
                cur = torch.cuda.current_stream(U.device)
                if self.stream.cuda_stream != cur.cuda_stream:
                    self.stream.wait_stream(cur)
                    U.record_stream(self.stream)
                return ctypes.c_void_p(U.data_ptr()), 1
            return ctypes.c_void_p(U.data_ptr()), 0
        if isinstance(U, np.ndarray):
            if U.shape != shape or U.dtype != np.float64 or not U.flags["C_CONTIGUOUS"]:
                raise ValueError(f"expected a C-contiguous float64 array of shape {shape}")
            if writable and not U.flags["WRITEABLE"]:
                raise ValueError("output array is read-only")
            return ctypes.c_void_p(U.ctypes.data), 0
        raise TypeError("state must be a torch tensor or a numpy array")

    def set_state(self, U):
        ptr, dev = self._buffer(U, self.shape, False)
        _check(self._lib.fv_set_state(self._h, ptr, dev), "fv_set_state")

    def get_state(self, out=None):
        """Interior state; into `out` if given, else a new CUDA tensor."""
        if out is None:
            out = _torch().empty(self.shape, dtype=_torch().float64, device=f"cuda:{self.device}")
        ptr, dev = self._buffer(out, self.shape, True)
        _check(self._lib.fv_get_state(self._h, ptr, dev), "fv_get_state")
        return out

    def get_ghosted_state(self, out=None):
        if out is None:
            out = _torch().empty(self.ghosted_shape, dtype=_torch().float64,
                                 device=f"cuda:{self.device}")
        ptr, dev = self._buffer(out, self.ghosted_shape, True)
        _check(self._lib.fv_get_ghosted_state(self._h, ptr, dev), "fv_get_ghosted_state")
        return out

    # -- the method
    def reduce_dt(self, cfl: float) -> float:
        dt = ctypes.c_double()
        _check(self._lib.fv_reduce_dt(self._h, float(cfl), ctypes.byref(dt)), "fv_reduce_dt")
        return dt.value

    def step(self, dt: float):
        _check(self._lib.fv_step(self._h, float(dt)), "fv_step")

    def substep(self, stage: int, dt: float):
        _check(self._lib.fv_substep(self._h, int(stage), float(dt)), "fv_substep")

    def fill_ghosts(self):
        _check(self._lib.fv_fill_ghosts(self._h), "fv_fill_ghosts")

    def conserved_sums(self) -> np.ndarray:
        out = (ctypes.c_double * 5)()
        _check(self._lib.fv_conserved_sums(self._h, out), "fv_conserved_sums")
        return np.array(out[:])

    def counters(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.fv_get_counters(self._h, ctypes.byref(a), ctypes.byref(b)),
               "fv_get_counters")
        return a.value, b.value

    def face_counts(self):
        """(evaluated, defined) face fluxes since the last set_state."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.fv_get_face_counts(self._h, ctypes.byref(a), ctypes.byref(b)),
               "fv_get_face_counts")
        return a.value, b.value

    def set_tuning(self, key: str, value):
        _check(self._lib.fv_set_tuning(self._h, TUNING_KEYS[key], float(value)),
               "fv_set_tuning")

    def profile(self, on: bool = True):
        _check(self._lib.fv_profile_enable(self._h, int(bool(on))), "fv_profile_enable")

    def read_profile(self):
        """{class: (device ms, launches)} since the last read; resets."""
        n = len(KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        _check(self._lib.fv_profile_read(self._h, ms, cnt), "fv_profile_read")
        return {c: (ms[k], cnt[k]) for k, c in enumerate(KERNEL_CLASSES)}

    def evolve(self, cfl: float, t_end: float | None = None, nsteps: int | None = None):
        """Algorithm 1's time loop: dt = min(ComputeTimeStep, t_end - t), step.
        Returns (t, steps, dts)."""
        t, n, dts = 0.0, 0, []
        while True:
            if t_end is not None and not t < t_end:
                break
            if nsteps is not None and n >= nsteps:
                break
            dt = self.reduce_dt(cfl)
            if t_end is not None and dt > t_end - t:
                dt = t_end - t
            self.step(dt)
            dts.append(dt)
            t += dt
            n += 1
        return t, n, dts

    # short names: set(U), dt(cfl), step(dt), get()
    def set(self, U):
        self.set_state(U)

    def get(self, out=None):
        return self.get_state(out)

    def dt(self, cfl: float) -> float:
        return self.reduce_dt(cfl)


def conserved_sums_noalloc(U, lx=1.0, ly=1.0, lz=1.0, stream=None):
    """Conservation sums of a caller-held (5, nz, ny, nx) float64 CUDA tensor
    through fv_conserved_sums_noalloc, which allocates no device memory (for
    callers whose device memory is managed elsewhere)."""
    torch = _torch()
    if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == torch.float64
            and U.is_contiguous() and U.dim() == 4 and U.shape[0] == 5):
        raise ValueError("U must be a contiguous float64 CUDA tensor of shape (5, nz, ny, nx)")
    if stream is None:
        stream = torch.cuda.current_stream(U.device)
    _, nz, ny, nx = U.shape
    out = (ctypes.c_double * 5)()
    lib = load_library()
    _check(lib.fv_conserved_sums_noalloc(ctypes.c_void_p(U.data_ptr()), nx, ny, nz, float(lx),
                                         float(ly), float(lz),
                                         ctypes.c_void_p(stream.cuda_stream), out),
           "fv_conserved_sums_noalloc")
    return np.array(out[:])


class Batch:
    """Many independent meshes advanced together by the FP32-bulk step
    (fv_batch_* in include/fv.h).  `shapes` is a list of (nx, ny, nz) on the
    unit cube (or pass `descs` kwargs per mesh)."""

    def __init__(self, shapes, gamma=1.4, theta=2.0, bc=("outflow",) * 3, stream=None,
                 extents=None):
        self._lib = load_library()
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        arr = (MeshDesc * len(self.shapes))()
        for m, (nx, ny, nz) in enumerate(self.shapes):
            d = arr[m]
            d.nx, d.ny, d.nz = nx, ny, nz
            l = extents[m] if extents else (1.0, 1.0, 1.0)
            d.lx, d.ly, d.lz = (float(v) for v in l)
            d.gamma, d.theta = float(gamma), float(theta)
            for a in range(3):
                d.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
            d.precision = PRECISION["fp32_bulk"]
        self.device = _torch().cuda.current_device()
        if stream is None:  # a stream of its own: capturable, unlike the default one
            stream = _torch().cuda.Stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self._lib.fv_batch_create(arr, len(self.shapes), ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.byref(h)), "fv_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(self._lib.fv_batch_destroy(self._h), "fv_batch_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _buf(self, m, U, writable):
        if not 0 <= m < len(self.shapes):   # let the library report the bad index
            return None, 0
        nx, ny, nz = self.shapes[m]
        return Mesh._buffer(self, U, (5, nz, ny, nx), writable)

    def set_state(self, m, U):
        ptr, dev = self._buf(m, U, False)
        _check(self._lib.fv_batch_set_state(self._h, int(m), ptr, dev), "fv_batch_set_state")

    def get_state(self, m, out=None):
        nx, ny, nz = self.shapes[m] if 0 <= m < len(self.shapes) else (1, 1, 1)
        if out is None:
            out = _torch().empty((5, nz, ny, nx), dtype=_torch().float64,
                                 device=f"cuda:{self.device}")
        ptr, dev = self._buf(m, out, True)
        _check(self._lib.fv_batch_get_state(self._h, int(m), ptr, dev), "fv_batch_get_state")
        return out

    def step(self, cfl=0.4, use_graph=True):
        _check(self._lib.fv_batch_step(self._h, float(cfl), int(bool(use_graph))),
               "fv_batch_step")

    def dts(self):
        out = (ctypes.c_double * len(self.shapes))()
        _check(self._lib.fv_batch_get_dt(self._h, out), "fv_batch_get_dt")
        return np.array(out[:])

    def set_tuning(self, kchunk, occupancy=2, tile_y=8):
        _check(self._lib.fv_batch_set_tuning(self._h, int(kchunk), int(occupancy), int(tile_y)),
               "fv_batch_set_tuning")

    def set_class_tuning(self, cls, tile_x, tile_y, occupancy, kchunk):
        _check(self._lib.fv_batch_set_class_tuning(self._h, int(cls), int(tile_x), int(tile_y),
                                                   int(occupancy), int(kchunk)),
               "fv_batch_set_class_tuning")

    def class_tuning(self, cls):
        """{tile_x, tile_y, occupancy, kchunk, meshes} of size class cls."""
        v = [ctypes.c_int() for _ in range(5)]
        _check(self._lib.fv_batch_get_class_tuning(self._h, int(cls),
                                                   *[ctypes.byref(x) for x in v]),
               "fv_batch_get_class_tuning")
        return dict(zip(("tile_x", "tile_y", "occupancy", "kchunk", "meshes"),
                        (x.value for x in v)))

    def autotune(self, cfl=0.4):
        """(kchunk, occupancy, tile_y, ms per step) of the fastest configuration."""
        kc, occ, ty, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(self._lib.fv_batch_autotune(self._h, float(cfl), ctypes.byref(kc),
                                           ctypes.byref(occ), ctypes.byref(ty), ctypes.byref(ms)),
               "fv_batch_autotune")
        return kc.value, occ.value, ty.value, ms.value

    def counters(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.fv_batch_get_counters(self._h, ctypes.byref(a), ctypes.byref(b)),
               "fv_batch_get_counters")
        return a.value, b.value

    def info(self):
        n, c, w = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(self._lib.fv_batch_info(self._h, ctypes.byref(n), ctypes.byref(c),
                                       ctypes.byref(w)), "fv_batch_info")
        return n.value, c.value, w.value


class Net:
    """The learned flux correction (fv_net_* in include/fv.h): three 3x3x3
    convolutions 5 -> 32 -> 32 -> 5, BF16 weights, FP32 accumulation."""

    def __init__(self):
        self._lib = load_library()
        self.nparam = int(self._lib.fv_net_param_count())
        h = ctypes.c_void_p()
        _check(self._lib.fv_net_create(ctypes.byref(h)), "fv_net_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(self._lib.fv_net_destroy(self._h), "fv_net_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparam
        _check(self._lib.fv_net_set_params(self._h, ctypes.c_void_p(a.ctypes.data)),
               "fv_net_set_params")

    def params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        _check(self._lib.fv_net_get_params(self._h, ctypes.c_void_p(p.ctypes.data), None),
               "fv_net_get_params")
        return p

    def grads(self):
        g = np.empty(self.nparam, dtype=np.float32)
        _check(self._lib.fv_net_get_params(self._h, None, ctypes.c_void_p(g.ctypes.data)),
               "fv_net_get_params")
        return g

    def set_scales(self, in_mean, in_scale, out_scale, res_scale):
        arrs = [(ctypes.c_double * 5)(*[float(v) for v in a])
                for a in (in_mean, in_scale, out_scale, res_scale)]
        _check(self._lib.fv_net_set_scales(self._h, *arrs), "fv_net_set_scales")

    def forward(self, mesh):
        torch = _torch()
        out = torch.empty((5,) + mesh.shape[1:], dtype=torch.float32,
                          device=f"cuda:{mesh.device}")
        _check(self._lib.fv_net_forward(self._h, mesh.handle, ctypes.c_void_p(out.data_ptr())),
               "fv_net_forward")
        return out

    def train_step(self, mesh, residual, dt, lr, sync=True):
        """One training step; returns its loss (sync), or None and adds the
        loss to the device-side sum that take_loss() returns (sync=False: no
        host wait)."""
        torch = _torch()
        assert isinstance(residual, torch.Tensor) and residual.is_cuda
        assert residual.dtype == torch.float64 and tuple(residual.shape) == mesh.shape
        loss = ctypes.c_double()
        _check(self._lib.fv_net_train_step(self._h, mesh.handle,
                                           ctypes.c_void_p(residual.data_ptr()), float(dt),
                                           float(lr), ctypes.byref(loss) if sync else None),
               "fv_net_train_step")
        return loss.value if sync else None

    def take_loss(self):
        """(sum of the asynchronous steps' losses, their number); clears."""
        total, n = ctypes.c_double(), ctypes.c_longlong()
        _check(self._lib.fv_net_take_loss(self._h, ctypes.byref(total), ctypes.byref(n)),
               "fv_net_take_loss")
        return total.value, n.value

    def step(self, mesh, dt):
        _check(self._lib.fv_step_learned(mesh.handle, self._h, float(dt)), "fv_step_learned")

    # buffer name: (enum value, torch dtype name, channel-last pitch or None)
    BUFFERS = {"features": (0, "bfloat16", 8), "h1": (1, "bfloat16", 32),
               "h2": (2, "bfloat16", 32), "out": (3, "float32", None),
               "grad_out": (4, "float32", None), "grad_a2": (5, "float32", 32),
               "grad_a1": (6, "float32", 32)}

    def buffer(self, name, mesh):
        """An intermediate buffer of the last pass on `mesh`
        (fv_net_get_buffer), as a CUDA tensor of shape (C, nz, ny, nx):
        channel-last buffers are returned transposed to channel-first."""
        torch = _torch()
        which, dtype, pitch = self.BUFFERS[name]
        _, nz, ny, nx = mesh.shape
        shape = (nz * ny * nx, pitch) if pitch else (5, nz, ny, nx)
        out = torch.empty(shape, dtype=getattr(torch, dtype), device=f"cuda:{mesh.device}")
        _check(self._lib.fv_net_get_buffer(self._h, which, ctypes.c_void_p(out.data_ptr()),
                                           out.numel() * out.element_size()),
               "fv_net_get_buffer")
        if pitch:
            out = out.t().reshape(pitch, nz, ny, nx)
        return out
