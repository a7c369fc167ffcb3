"""FP64 CPU oracle for the first-order finite-volume step of arXiv:1701.05431.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the product library never does.  The
arithmetic lives in ``fv_oracle.c`` (plain C99, FP64, OpenMP over rows); this
module only compiles it and marshals arguments through ctypes.  It shares no
code with the CUDA path and imports nothing from it.

Sections followed (see the C file's header for the readings taken):
  Sec. 2.2.1  Eq. (VF_scheme), Lax-Friedrichs flux, Eq. (CFL_cond)
  Sec. 2.2.2  Eq. (SourceTerm), split forward-Euler source step
  Sec. 3.2, 4.1-4.2  partition, uLoc/RHS/overlap strips and tasks
  Sec. 5      Eq. (Euler) system
  Sec. 6.1-6.2  spray moment system and maximum-entropy reconstruction

``riemann.py`` (exact Riemann solver for the 1D Euler equations) is also
oracle-side: it pins the Euler flux against an exact solution.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ADVECTION, EULER, SPRAY = 0, 1, 2
PERIODIC, TRANSMISSIVE, DIRICHLET = 0, 1, 2
E, N, W, S = 0, 1, 2, 3
OK, ERR_ARG, ERR_CFL, ERR_NONPHYSICAL = 0, 1, 4, 5
NVAR = {ADVECTION: 1, EULER: 4, SPRAY: 6}


def build(force: bool = False) -> str:
    """Compile fv_oracle.c into liboracle.so next to it (gcc, -O2, no FMA
    contraction so every expression rounds in the written order)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("npart_x", ctypes.c_int), ("npart_y", ctypes.c_int),
        ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
        ("ymin", ctypes.c_double), ("ymax", ctypes.c_double),
        ("system", ctypes.c_int),
        ("bc", ctypes.c_int * 4),
        ("bc_state", (ctypes.c_double * 8) * 4),
        ("cfl", ctypes.c_double), ("fixed_dt", ctypes.c_double),
        ("params", ctypes.c_double * 8),
    ]


@dataclass
class Problem:
    """Problem statement of Sec. 2.1-2.2 (see fv_oracle.c for params)."""
    nx: int
    ny: int
    system: int = EULER
    npart_x: int = 1
    npart_y: int = 1
    xmin: float = 0.0
    xmax: float = 1.0
    ymin: float = 0.0
    ymax: float = 1.0
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC, PERIODIC)
    bc_state: tuple = ()
    cfl: float = 0.4
    fixed_dt: float = 0.0
    params: tuple = (1.4,)

    @property
    def nvar(self) -> int:
        return NVAR[self.system]

    @property
    def dx(self) -> float:
        return (self.xmax - self.xmin) / self.nx

    @property
    def dy(self) -> float:
        return (self.ymax - self.ymin) / self.ny

    def c(self) -> _Problem:
        p = _Problem()
        p.nx, p.ny, p.npart_x, p.npart_y = self.nx, self.ny, self.npart_x, self.npart_y
        p.xmin, p.xmax, p.ymin, p.ymax = self.xmin, self.xmax, self.ymin, self.ymax
        p.system = self.system
        for k in range(4):
            p.bc[k] = int(self.bc[k])
        for s, st in enumerate(self.bc_state):
            for v, val in enumerate(st):
                p.bc_state[s][v] = float(val)
        p.cfl, p.fixed_dt = self.cfl, self.fixed_dt
        for k, val in enumerate(self.params):
            p.params[k] = float(val)
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        L.ofv_run.argtypes = [pp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                              dp, dp, ctypes.POINTER(ctypes.c_int)]
        L.ofv_run.restype = ctypes.c_int
        L.ofv_prim_to_cons.argtypes = [pp, dp, dp]
        L.ofv_totals.argtypes = [pp, dp, dp]
        L.ofv_lambda_max.argtypes = [pp, dp]
        L.ofv_lambda_max.restype = ctypes.c_double
        L.ofv_cell_lambda.argtypes = [pp, dp]
        L.ofv_cell_lambda.restype = ctypes.c_double
        L.ofv_lf_flux.argtypes = [pp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.ofv_phys_flux.argtypes = [pp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.ofv_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.ofv_maxent.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp, dp,
                                 ctypes.POINTER(ctypes.c_int)]
        L.ofv_realizable.argtypes = [dp]
        L.ofv_spray_source_cell.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.ofv_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class RunResult:
    W: np.ndarray
    t: float
    dts: np.ndarray
    steps: int
    status: int = OK
    extra: dict = field(default_factory=dict)


def prim_to_cons(P: Problem, prim: np.ndarray) -> np.ndarray:
    prim = np.ascontiguousarray(prim, dtype=np.float64).reshape(P.nvar, P.ny, P.nx)
    W = np.empty_like(prim)
    pc = P.c()
    lib().ofv_prim_to_cons(ctypes.byref(pc), _dp(prim), _dp(W))
    return W


def run(P: Problem, W0: np.ndarray, nsteps: int, t_end: float = 0.0, mode: str = "plain",
        nthreads: int = 0, t0: float = 0.0) -> RunResult:
    """Advance conserved state W0 (nvar, ny, nx) by nsteps steps."""
    W = np.array(W0, dtype=np.float64, copy=True, order="C").reshape(P.nvar, P.ny, P.nx)
    dts = np.zeros(max(nsteps, 1))
    t = ctypes.c_double(t0)
    done = ctypes.c_int(0)
    pc = P.c()
    st = lib().ofv_run(ctypes.byref(pc), _dp(W), int(nsteps), float(t_end),
                       0 if mode == "plain" else 1, int(nthreads), ctypes.byref(t), _dp(dts),
                       ctypes.byref(done))
    return RunResult(W=W, t=t.value, dts=dts[: done.value], steps=done.value, status=st)


def totals(P: Problem, W: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(P.nvar)
    pc = P.c()
    lib().ofv_totals(ctypes.byref(pc), _dp(W), _dp(out))
    return out


def lambda_max(P: Problem, W: np.ndarray) -> float:
    W = np.ascontiguousarray(W, dtype=np.float64)
    pc = P.c()
    return lib().ofv_lambda_max(ctypes.byref(pc), _dp(W))


def cell_lambda(P: Problem, w: np.ndarray) -> float:
    w = np.ascontiguousarray(w, dtype=np.float64)
    pc = P.c()
    return lib().ofv_cell_lambda(ctypes.byref(pc), _dp(w))


def lf_flux(P: Problem, wl, wr, normal) -> np.ndarray:
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    out = np.zeros(P.nvar)
    pc = P.c()
    lib().ofv_lf_flux(ctypes.byref(pc), _dp(wl), _dp(wr), float(normal[0]), float(normal[1]), _dp(out))
    return out


def phys_flux(P: Problem, w, normal):
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(P.nvar)
    s = ctypes.c_double(0)
    pc = P.c()
    lib().ofv_phys_flux(ctypes.byref(pc), _dp(w), float(normal[0]), float(normal[1]), _dp(out),
                        ctypes.byref(s))
    return out, s.value


def gauss_legendre(Q: int):
    x = np.zeros(Q)
    w = np.zeros(Q)
    st = lib().ofv_gauss_legendre(int(Q), _dp(x), _dp(w))
    if st != OK:
        raise ValueError("bad Q")
    return x, w


def maxent(m, Q: int = 32, tol: float = 1e-13):
    """Maximum-entropy reconstruction (Sec. 6.2).  Returns (status, lam, n(0),
    m_{-1/2}, iterations)."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    x, w = gauss_legendre(Q)
    lam = np.zeros(4)
    n0 = ctypes.c_double(0)
    mmh = ctypes.c_double(0)
    it = ctypes.c_int(0)
    st = lib().ofv_maxent(_dp(m), int(Q), _dp(x), _dp(w), float(tol), _dp(lam), ctypes.byref(n0),
                          ctypes.byref(mmh), ctypes.byref(it))
    return st, lam, n0.value, mmh.value, it.value


def realizable(c) -> bool:
    c = np.ascontiguousarray(c, dtype=np.float64)
    return bool(lib().ofv_realizable(_dp(c)))


def spray_source_cell(P: Problem, dt: float, x: float, y: float, w) -> tuple:
    w = np.array(w, dtype=np.float64)
    pc = P.c()
    st = lib().ofv_spray_source_cell(ctypes.byref(pc), float(dt), float(x), float(y), _dp(w))
    return st, w


def max_threads() -> int:
    return lib().ofv_max_threads()
