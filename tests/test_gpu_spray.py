"""GPU parity of the spray moment system (Sec. 6.1-6.2): transport by the
fused step, then the FP64 maximum-entropy source step, against the oracle.

Tolerances: FP64 <= 1e-12 relative L-infinity (both sides converge the Newton
solve to a relative moment residual <= 1e-13; the source is a small
correction, K dt n(0) per step); FP32 storage <= 1e-5 relative L1.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from tests.helpers import oracle_problem, rel_l1, rel_linf, transpose_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()


def fv():
    from paper_1701_05431_gb300 import fvlib
    return fvlib


def gpu_run(d, prim, nsteps, precision="f64", primitive=True):
    f = fv()
    with f.Solver(d, precision) as s:
        s.set_state(np.ascontiguousarray(prim), primitive=primitive)
        t = s.run(nsteps)
        return s.state(), t


def oracle_run(d, prim, nsteps):
    P = oracle_problem(d)
    r = oracle.run(P, oracle.prim_to_cons(P, prim), nsteps)
    assert r.status == oracle.OK
    return r


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_spray_parity(precision):
    prim, d = wl.spray_field(96)
    ref = oracle_run(d, prim, 30)
    out, t = gpu_run(d, prim, 30, precision)
    if precision == "f64":
        assert rel_linf(out, ref.W).max() <= 1e-12
        assert abs(t - ref.t) <= 1e-13 * ref.t
    else:
        assert rel_l1(out, ref.W).max() <= 1e-5


def test_spray_parity_ragged_drag_off():
    prim, d = wl.spray_field(73)
    d = dict(d, ny=73, params=(0.3, 0.0, 0.0, 24.0, 1e-13))
    ref = oracle_run(d, prim, 12)
    out, _ = gpu_run(d, prim, 12)
    assert rel_linf(out, ref.W).max() <= 1e-12


def test_spray_constant_density_evaporation():
    """n(S) = C: one step lowers m0..m3/2 by K C dt exactly (to rounding)."""
    n = 16
    C, K = 0.8, 0.3
    prim = np.empty((6, n, n))
    for k in range(4):
        prim[k] = C / (1 + k / 2)
    prim[4] = 0.0
    prim[5] = 0.0
    d = wl.problem("spray", n, n, fixed_dt=0.01, params=(K, 0.0, 0.0, 32.0, 1e-13))
    out, _ = gpu_run(d, prim, 1)
    for k in range(4):
        np.testing.assert_allclose(out[k], C / (1 + k / 2) - K * C * 0.01, rtol=0, atol=2e-14)
    assert np.all(out[4] == 0.0) and np.all(out[5] == 0.0)


def test_spray_transport_constant_state_bitwise():
    n = 24
    const = [1.0, 0.55, 0.4, 0.31, 0.4 * 0.3, 0.4 * -0.2]
    W0 = np.empty((6, n, n))
    for v, c in enumerate(const):
        W0[v] = c
    d = wl.problem("spray", n, n, params=(0.0, 0.0, 0.0, 32.0, 1e-13))
    out, _ = gpu_run(d, W0, 5, primitive=False)
    assert np.array_equal(out, W0)


def test_spray_transposition_bitwise_transport_only():
    prim, d = wl.spray_field(40)
    prim = prim[:, :, :32].copy()
    d = dict(d, nx=32, params=(0.0, 0.0, 0.0, 32.0, 1e-13))
    P = oracle_problem(d)
    W0 = oracle.prim_to_cons(P, prim)
    out, _ = gpu_run(d, W0, 10, primitive=False)
    dt_ = dict(d, nx=40, ny=32)
    outt, _ = gpu_run(dt_, transpose_state(W0, "spray"), 10, primitive=False)
    assert np.array_equal(transpose_state(outt, "spray"), out)


def test_spray_nonrealizable_state_rejected():
    prim, d = wl.spray_field(16)
    prim[3, 4, 4] = prim[2, 4, 4]  # m3/2 = m1: outside the moment space
    f = fv()
    with f.Solver(d, "f64") as s:
        assert s.set_state(prim, primitive=True, check=False) == f.FV_ERR_NONPHYSICAL
