"""Python binding of the C ABI in include/fv.h (argument marshalling only).

Every step of the finite-volume method runs in the CUDA kernels of
libfv.so; this module converts Python values and torch tensors into the
plain pointers and sizes the ABI takes.  It never computes anything itself
and raises if the library is missing: there is no CPU fallback.

Function names follow the ABI: fv_init, fv_set_state, fv_step, fv_run,
fv_get_state, fv_totals, fv_time, fv_set_time, fv_lambda_max,
fv_kernel_info, fv_gauss_legendre, fv_snapshot, fv_snapshot_wait,
fv_prefetch_state, fv_set_state_prefetched, fv_destroy, plus the batched
fv_batch_*.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

FV_OK, FV_ERR_INVALID_ARG, FV_ERR_CUDA, FV_ERR_OOM = 0, 1, 2, 3
FV_ERR_CFL, FV_ERR_NONPHYSICAL, FV_ERR_TIMEOUT, FV_ERR_STATE = 4, 5, 6, 7
FV_ADVECTION, FV_EULER, FV_SPRAY = 0, 1, 2
FV_F64, FV_F32, FV_BF16 = 0, 1, 2
FV_BC_PERIODIC, FV_BC_TRANSMISSIVE, FV_BC_DIRICHLET = 0, 1, 2
FV_CONSERVED, FV_PRIMITIVE = 0, 1

SYSTEMS = {"advection": FV_ADVECTION, "euler": FV_EULER, "spray": FV_SPRAY}
BCS = {"periodic": FV_BC_PERIODIC, "transmissive": FV_BC_TRANSMISSIVE, "dirichlet": FV_BC_DIRICHLET}
PRECISIONS = {"f64": FV_F64, "f32": FV_F32, "bf16": FV_BF16}
NVAR = {FV_ADVECTION: 1, FV_EULER: 4, FV_SPRAY: 6}


class FvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class fv_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("npart_x", ctypes.c_int), ("npart_y", ctypes.c_int),
        ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
        ("ymin", ctypes.c_double), ("ymax", ctypes.c_double),
        ("system", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("bc", ctypes.c_int * 4),
        ("bc_state", (ctypes.c_double * 8) * 4),
        ("cfl", ctypes.c_double),
        ("fixed_dt", ctypes.c_double),
        ("params", ctypes.c_double * 8),
        ("stream", ctypes.c_void_p),
        ("tune", ctypes.c_int),
    ]


_lib = None

EXPORTS = ("fv_status_string", "fv_last_error", "fv_init", "fv_destroy", "fv_set_state", "fv_step",
           "fv_run", "fv_get_state", "fv_totals", "fv_time", "fv_set_time", "fv_lambda_max",
           "fv_kernel_info", "fv_kernel_candidate", "fv_gauss_legendre", "fv_snapshot",
           "fv_snapshot_wait", "fv_set_inplace", "fv_set_time_blocking", "fv_kernel_info_two_step",
           "fv_prefetch_state", "fv_set_state_prefetched")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfv.so (building it first if needed) and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libfv.so is not built; run paper_1701_05431_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    L.fv_status_string.restype = ctypes.c_char_p
    L.fv_status_string.argtypes = [ctypes.c_int]
    L.fv_last_error.restype = ctypes.c_char_p
    L.fv_last_error.argtypes = [vp]
    L.fv_init.argtypes = [ctypes.POINTER(fv_config), ctypes.POINTER(vp)]
    L.fv_destroy.argtypes = [vp]
    L.fv_destroy.restype = None
    L.fv_set_state.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.fv_step.argtypes = [vp, dp]
    L.fv_run.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp]
    L.fv_get_state.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
    L.fv_totals.argtypes = [vp, dp]
    L.fv_snapshot.argtypes = [vp, vp, ctypes.c_int]
    L.fv_snapshot_wait.argtypes = [vp]
    L.fv_prefetch_state.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
    L.fv_set_state_prefetched.argtypes = [vp]
    L.fv_set_inplace.argtypes = [vp, ctypes.c_int]
    L.fv_set_time_blocking.argtypes = [vp, ctypes.c_int]
    L.fv_kernel_info_two_step.argtypes = [vp]
    L.fv_kernel_info_two_step.restype = ctypes.c_char_p
    L.fv_time.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong)]
    L.fv_set_time.argtypes = [vp, ctypes.c_double, ctypes.c_longlong]
    L.fv_lambda_max.argtypes = [vp, dp]
    L.fv_kernel_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_char_p)]
    L.fv_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
    L.fv_kernel_candidate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p)]
    for name in EXPORTS:
        if name not in ("fv_status_string", "fv_last_error", "fv_destroy", "fv_kernel_info_two_step"):
            getattr(L, name).restype = ctypes.c_int
    L.fv_totals_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, vp, vp]
    L.fv_totals_noalloc.restype = ctypes.c_int
    L.fv_kernel_choice.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p)]
    L.fv_kernel_choice.restype = ctypes.c_int
    L.fv_fma_peak.argtypes = [ctypes.c_int, ctypes.c_double, dp, vp]
    L.fv_fma_peak.restype = ctypes.c_int
    _declare_batch(L)
    _lib = L
    return L


def _declare_batch(L):
    if not hasattr(L, "fv_batch_init"):
        return
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    L.fv_batch_init.argtypes = [ctypes.POINTER(fv_config), ctypes.c_int, ctypes.POINTER(vp)]
    L.fv_batch_init.restype = ctypes.c_int
    L.fv_batch_destroy.argtypes = [vp]
    L.fv_batch_destroy.restype = None
    L.fv_batch_set_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.fv_batch_set_state.restype = ctypes.c_int
    L.fv_batch_run.argtypes = [vp, ctypes.c_int]
    L.fv_batch_run.restype = ctypes.c_int
    L.fv_batch_get_state.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int]
    L.fv_batch_get_state.restype = ctypes.c_int
    L.fv_batch_time.argtypes = [vp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_longlong)]
    L.fv_batch_time.restype = ctypes.c_int
    L.fv_batch_last_error.argtypes = [vp]
    L.fv_batch_last_error.restype = ctypes.c_char_p
    L.fv_batch_kernel_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_char_p)]
    L.fv_batch_kernel_info.restype = ctypes.c_int
    L.fv_batch_kernel_choice.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p)]
    L.fv_batch_kernel_choice.restype = ctypes.c_int
    L.fv_batch_set_wait_limit.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    L.fv_batch_set_wait_limit.restype = ctypes.c_int
    L.fv_batch_set_dataflow.argtypes = [vp, ctypes.c_int]
    L.fv_batch_set_dataflow.restype = ctypes.c_int


def make_config(d: dict, precision: str = "f64", stream: int = 0, tune: int = 0) -> fv_config:
    """fv_config from a plain problem description (see workloads.problem)."""
    c = fv_config()
    c.nx, c.ny = int(d["nx"]), int(d["ny"])
    c.npart_x, c.npart_y = int(d.get("npart_x", 1)), int(d.get("npart_y", 1))
    c.xmin, c.xmax = float(d.get("xmin", 0.0)), float(d.get("xmax", 1.0))
    c.ymin, c.ymax = float(d.get("ymin", 0.0)), float(d.get("ymax", 1.0))
    c.system = SYSTEMS[d["system"]]
    c.precision = PRECISIONS[precision]
    for k, b in enumerate(d["bc"]):
        c.bc[k] = BCS[b]
    for s, st in enumerate(d.get("bc_state", ())):
        for v, val in enumerate(st):
            c.bc_state[s][v] = float(val)
    c.cfl = float(d.get("cfl", 0.4))
    c.fixed_dt = float(d.get("fixed_dt", 0.0))
    for k, val in enumerate(d["params"]):
        c.params[k] = float(val)
    c.stream = stream
    c.tune = int(tune)
    return c


def _check(st: int, ctx=None, lib=None):
    if st != FV_OK:
        L = lib or load()
        msg = L.fv_last_error(ctx).decode() if ctx is not None else L.fv_last_error(None).decode()
        raise FvError(st, msg or L.fv_status_string(st).decode())


def _ptr(x):
    """(address, is_device) of a torch tensor or numpy array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return x.data_ptr(), 1 if x.is_cuda else 0
    except ImportError:
        pass
    import numpy as np
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    raise TypeError(f"unsupported buffer type {type(x)}")


def _numel(x) -> int:
    n = x.numel() if hasattr(x, "numel") else x.size
    return int(n)


def _dtype_code(x) -> int:
    s = str(x.dtype)
    if s.endswith("float64"):
        return FV_F64
    if s.endswith("float32"):
        return FV_F32
    raise TypeError(f"unsupported dtype {x.dtype}")


class Solver:
    """Thin owner of one fv_ctx; methods map one-to-one onto the ABI."""

    def __init__(self, problem: dict, precision: str = "f64", stream: int = 0, tune: int = 0):
        self.lib = load()
        self.cfg = make_config(problem, precision, stream, tune)
        self.nvar = NVAR[self.cfg.system]
        self.nx, self.ny = self.cfg.nx, self.cfg.ny
        h = ctypes.c_void_p()
        _check(self.lib.fv_init(ctypes.byref(self.cfg), ctypes.byref(h)), None, self.lib)
        self.ctx = h

    def close(self):
        if self.ctx:
            self.lib.fv_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _need(self, x):
        if _numel(x) != self.nvar * self.ny * self.nx:
            raise ValueError(f"expected {self.nvar} x {self.ny} x {self.nx} values, got {_numel(x)}")

    def set_state(self, src, primitive: bool = False, check: bool = True) -> int:
        self._need(src)
        p, dev = _ptr(src)
        st = self.lib.fv_set_state(self.ctx, p, dev, _dtype_code(src), 1 if primitive else 0)
        if check:
            _check(st, self.ctx, self.lib)
        return st

    def run(self, nsteps: int, t_end: float = 0.0, check: bool = True):
        t = ctypes.c_double(0)
        st = self.lib.fv_run(self.ctx, int(nsteps), float(t_end), ctypes.byref(t))
        if check:
            _check(st, self.ctx, self.lib)
        return (st, t.value) if not check else t.value

    def step(self, check: bool = True):
        dt = ctypes.c_double(0)
        st = self.lib.fv_step(self.ctx, ctypes.byref(dt))
        if check:
            _check(st, self.ctx, self.lib)
        return dt.value

    def get_state(self, dst):
        self._need(dst)
        p, dev = _ptr(dst)
        _check(self.lib.fv_get_state(self.ctx, p, dev, _dtype_code(dst)), self.ctx, self.lib)
        return dst

    def state(self, dtype="float64"):
        import numpy as np
        out = np.empty((self.nvar, self.ny, self.nx), dtype=dtype)
        return self.get_state(out)

    def snapshot(self, dst):
        """Queue an asynchronous copy of the current state into host memory
        `dst` (float32/float64, shape (nvar, ny, nx); pinned memory lets later
        steps overlap the copy).  Do not read dst before snapshot_wait()."""
        self._need(dst)
        p, dev = _ptr(dst)
        if dev:
            raise ValueError("snapshot target must be host memory")
        _check(self.lib.fv_snapshot(self.ctx, p, _dtype_code(dst)), self.ctx, self.lib)
        return dst

    def set_time_blocking(self, steps_per_pass: int = 2):
        """Two time steps per kernel launch (fixed dt, periodic grids; same
        results as one step per launch)."""
        _check(self.lib.fv_set_time_blocking(self.ctx, int(steps_per_pass)), self.ctx, self.lib)

    def two_step_kernel(self):
        """Description of the two-step kernel in use, or None."""
        d = self.lib.fv_kernel_info_two_step(self.ctx)
        return d.decode() if d else None

    def set_inplace(self, on: bool = True):
        """One state buffer updated in place, halos from overlap strips
        (same results as the default two-buffer mode)."""
        _check(self.lib.fv_set_inplace(self.ctx, 1 if on else 0), self.ctx, self.lib)

    def snapshot_wait(self):
        _check(self.lib.fv_snapshot_wait(self.ctx), self.ctx, self.lib)

    def prefetch_state(self, src, primitive: bool = False):
        """Queue an asynchronous copy of a state from host memory `src`
        (float32/float64, shape (nvar, ny, nx); pinned memory lets the steps
        already queued overlap the copy).  Keep src unchanged until
        set_state_prefetched()."""
        self._need(src)
        p, dev = _ptr(src)
        if dev:
            raise ValueError("prefetch source must be host memory")
        _check(self.lib.fv_prefetch_state(self.ctx, p, _dtype_code(src), 1 if primitive else 0),
               self.ctx, self.lib)
        return src

    def set_state_prefetched(self, check: bool = True) -> int:
        """set_state from the last prefetch_state (same results)."""
        st = self.lib.fv_set_state_prefetched(self.ctx)
        if check:
            _check(st, self.ctx, self.lib)
        return st

    def totals(self):
        import numpy as np
        out = np.zeros(self.nvar)
        _check(self.lib.fv_totals(self.ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               self.ctx, self.lib)
        return out

    def time(self):
        t = ctypes.c_double(0)
        s = ctypes.c_longlong(0)
        _check(self.lib.fv_time(self.ctx, ctypes.byref(t), ctypes.byref(s)), self.ctx, self.lib)
        return t.value, s.value

    def set_time(self, t: float, step: int):
        _check(self.lib.fv_set_time(self.ctx, float(t), int(step)), self.ctx, self.lib)

    def lambda_max(self) -> float:
        out = ctypes.c_double(0)
        _check(self.lib.fv_lambda_max(self.ctx, ctypes.byref(out)), self.ctx, self.lib)
        return out.value

    def kernel_choice(self, two_step: bool = False) -> str:
        """How the step kernel (or the two-step kernel) was chosen: the
        recorded table entry, the heuristic, autotuning or a forced index."""
        h = ctypes.c_char_p()
        _check(self.lib.fv_kernel_choice(self.ctx, 1 if two_step else 0, ctypes.byref(h)), self.ctx, self.lib)
        return h.value.decode()

    def kernel_info(self):
        v = ctypes.c_int(0)
        d = ctypes.c_char_p()
        _check(self.lib.fv_kernel_info(self.ctx, ctypes.byref(v), ctypes.byref(d)), self.ctx, self.lib)
        return v.value, d.value.decode()


def totals_noalloc(state, totals, cell_area: float, stream: int = 0) -> int:
    """fv_totals_noalloc on a device state tensor (nvar, ny, nx) into a device
    tensor of nvar float64 values; returns the status."""
    L = load()
    nvar, ny, nx = state.shape
    p, dev = _ptr(state)
    q, _ = _ptr(totals)
    return L.fv_totals_noalloc(p, _dtype_code(state), int(nvar), int(nx), int(ny), float(cell_area), q, stream)


def fma_peak(precision: str = "f64", seconds: float = 0.05, stream: int = 0) -> float:
    """Measured FMA instructions retired per second by the GPU's FP64
    (precision "f64") or FP32 ("f32") pipe: fv_fma_peak."""
    L = load()
    r = ctypes.c_double(0)
    _check(L.fv_fma_peak(PRECISIONS[precision], float(seconds), ctypes.byref(r), stream), None, L)
    return r.value


def kernel_candidates(system: str, precision: str):
    """Descriptions of the compiled step-kernel candidates, in index order."""
    L = load()
    out = []
    d = ctypes.c_char_p()
    while L.fv_kernel_candidate(SYSTEMS[system], PRECISIONS[precision], len(out), ctypes.byref(d)) == FV_OK:
        out.append(d.value.decode())
    return out


def gauss_legendre(Q: int):
    import numpy as np
    L = load()
    x = np.zeros(Q)
    w = np.zeros(Q)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(L.fv_gauss_legendre(int(Q), x.ctypes.data_as(dp), w.ctypes.data_as(dp)), None, L)
    return x, w


class Batch:
    """Thin owner of one fv_batch (independent instances, one persistent
    launch per run); methods map one-to-one onto the fv_batch_* ABI."""

    def __init__(self, problems, precision: str = "f32", stream: int = 0, tune: int = 0):
        self.lib = load()
        n = len(problems)
        arr = (fv_config * n)()
        for k, d in enumerate(problems):
            arr[k] = make_config(d, precision, stream, tune)
        self.shapes = [(NVAR[arr[k].system], arr[k].ny, arr[k].nx) for k in range(n)]
        h = ctypes.c_void_p()
        st = self.lib.fv_batch_init(arr, n, ctypes.byref(h))
        if st != FV_OK:
            raise FvError(st, "fv_batch_init failed: " + self.lib.fv_status_string(st).decode())
        self.b = h
        self.n = n

    def _check(self, st):
        if st != FV_OK:
            raise FvError(st, self.lib.fv_batch_last_error(self.b).decode() or
                          self.lib.fv_status_string(st).decode())

    def close(self):
        if getattr(self, "b", None):
            self.lib.fv_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_state(self, k: int, src, primitive: bool = False, check: bool = True) -> int:
        p, dev = _ptr(src)
        st = self.lib.fv_batch_set_state(self.b, int(k), p, dev, _dtype_code(src), 1 if primitive else 0)
        if check:
            self._check(st)
        return st

    def run(self, nsteps: int, check: bool = True) -> int:
        st = self.lib.fv_batch_run(self.b, int(nsteps))
        if check:
            self._check(st)
        return st

    def get_state(self, k: int, dst):
        p, dev = _ptr(dst)
        self._check(self.lib.fv_batch_get_state(self.b, int(k), p, dev, _dtype_code(dst)))
        return dst

    def state(self, k: int, dtype="float64"):
        import numpy as np
        out = np.empty(self.shapes[k], dtype=dtype)
        return self.get_state(k, out)

    def time(self, k: int):
        t = ctypes.c_double(0)
        s = ctypes.c_longlong(0)
        self._check(self.lib.fv_batch_time(self.b, int(k), ctypes.byref(t), ctypes.byref(s)))
        return t.value, s.value

    def kernel_choice(self) -> str:
        h = ctypes.c_char_p()
        self._check(self.lib.fv_batch_kernel_choice(self.b, ctypes.byref(h)))
        return h.value.decode()

    def kernel_info(self):
        v = ctypes.c_int(0)
        d = ctypes.c_char_p()
        self._check(self.lib.fv_batch_kernel_info(self.b, ctypes.byref(v), ctypes.byref(d)))
        return v.value, d.value.decode()

    def set_dataflow(self, on: bool = True):
        """Fixed-dt dataflow mode: neighbour dependencies instead of one
        barrier per step (same results as the default mode)."""
        self._check(self.lib.fv_batch_set_dataflow(self.b, 1 if on else 0))

    def set_wait_limit(self, seconds: float, never_release_instance: int = -1):
        self._check(self.lib.fv_batch_set_wait_limit(self.b, float(seconds), int(never_release_instance)))
