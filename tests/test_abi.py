"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/*.h declares, rejects bad configurations before any
CUDA call, and its host-side Gauss-Legendre rule matches numpy's."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1701_05431_gb300 import fvlib
import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fv_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = fvlib.load()
    names = declared_functions()
    assert "fv_init" in names and "fv_run" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    L = fvlib.load()
    for s in range(8):
        assert L.fv_status_string(s)
    assert L.fv_status_string(99) == b"unknown status"


@pytest.mark.parametrize("Q", [1, 3, 8, 32, 64])
def test_library_gauss_legendre_matches_numpy(Q):
    x, w = fvlib.gauss_legendre(Q)
    t, wt = np.polynomial.legendre.leggauss(Q)
    np.testing.assert_allclose(x, 0.5 * (t + 1.0), rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * wt, rtol=0, atol=2e-15)


def _init_status(d, over=None):
    L = fvlib.load()
    c = fvlib.make_config(d, "f64")
    for k, v in (over or {}).items():
        setattr(c, k, v)
    h = ctypes.c_void_p()
    st = L.fv_init(ctypes.byref(c), ctypes.byref(h))
    if st == fvlib.FV_OK:
        L.fv_destroy(h)
    return st, L.fv_last_error(None).decode()


@pytest.mark.parametrize("over,frag", [
    (dict(nx=0), "nx and ny"),
    (dict(ny=-3), "nx and ny"),
    (dict(npart_x=0), "npart"),
    (dict(npart_y=100), "npart"),
    (dict(system=7), "unknown system"),
    (dict(precision=5), "unknown precision"),
    (dict(cfl=0.0, fixed_dt=0.0), "cfl"),
    (dict(xmax=0.0), "empty domain"),
])
def test_init_rejects_bad_config(over, frag):
    _, d = wl.random_smooth_euler(16, seed=1)
    st, msg = _init_status(d, over)
    assert st == fvlib.FV_ERR_INVALID_ARG
    assert frag in msg


def test_init_rejects_unpaired_periodic():
    _, d = wl.random_smooth_euler(16, seed=1)
    d = dict(d, bc=("periodic", "periodic", "transmissive", "periodic"))
    st, msg = _init_status(d)
    assert st == fvlib.FV_ERR_INVALID_ARG and "periodic" in msg


def test_init_rejects_bad_gamma():
    _, d = wl.random_smooth_euler(16, seed=1)
    st, msg = _init_status(dict(d, params=(1.0,)))
    assert st == fvlib.FV_ERR_INVALID_ARG and "gamma" in msg


def test_null_arguments():
    L = fvlib.load()
    assert L.fv_init(None, None) == fvlib.FV_ERR_INVALID_ARG
    assert L.fv_run(None, 1, 0.0, None) == fvlib.FV_ERR_INVALID_ARG
    assert L.fv_set_state(None, None, 0, 0, 0) == fvlib.FV_ERR_INVALID_ARG
    L.fv_destroy(None)


def test_fma_peak_rejects_bad_arguments_before_any_cuda_call():
    L = fvlib.load()
    r = ctypes.c_double(0)
    assert L.fv_fma_peak(7, 0.05, ctypes.byref(r), None) == fvlib.FV_ERR_INVALID_ARG
    assert L.fv_fma_peak(0, 10.0, ctypes.byref(r), None) == fvlib.FV_ERR_INVALID_ARG
    assert L.fv_fma_peak(0, 0.05, None, None) == fvlib.FV_ERR_INVALID_ARG


def test_recorded_kernel_table_names_compiled_candidates():
    """Every two-buffer entry of the autotuner's table names a candidate the
    library has compiled (a stale table would silently fall back)."""
    path = os.path.join(ROOT, "paper_1701_05431_gb300", "tune_table.json")
    if not os.path.exists(path):
        pytest.skip("no autotune table recorded")
    import json
    from paper_1701_05431_gb300 import autotune
    for r in json.load(open(path)):
        assert r["size_class"] == autotune.size_class(r["cells"])
        if r["mode"] == "single":
            names = fvlib.kernel_candidates(r["system"], r["precision"])
            for kernel, _ in r["candidates"]:
                assert kernel in names, (r["name"], kernel)
