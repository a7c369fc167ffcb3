"""The paper's validation cases on the GPU path (Sec. 5.1: localized cosine
perturbation and isentropic vortex, mesh convergence of Fig. Convergence):
the L1 error of the density against the exact solution falls at first
order (the paper measures slopes near 0.95), in FP64 and in FP32-bulk, on
grids up to 1024^2 that the oracle would take minutes for."""
from __future__ import annotations

import math

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("case", ["vortex", "cosine"])
def test_gpu_mesh_convergence_first_order(case, precision):
    from paper_1701_05431_gb300 import fvlib
    T = 0.1
    errs = []
    ns = [128, 256, 512, 1024]
    for n in ns:
        if case == "vortex":
            prim, d = wl.isentropic_vortex(n)
            exact_rho = wl.isentropic_vortex(n, t=T)[0][0]
        else:
            prim, d = wl.localized_cosine(n, repaired=True)
            exact_rho = wl.localized_cosine_exact(n, T, repaired=True)
        with fvlib.Solver(d, precision) as s:
            s.set_state(prim, primitive=True)
            t = s.run(100000, t_end=T)
            assert abs(t - T) <= 1e-14
            rho = s.state()[0]
        errs.append(np.abs(rho - exact_rho).mean())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    print(case, precision, "L1 errors", errs, "orders", orders)
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:]))
    assert 0.85 <= orders[-1] <= 1.1, orders
