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


def test_spray_evaporation_momentum_keeps_velocity():
    """Momentum row of Eq. (Essadki) without drag: a uniform field moving at
    (u, v) is untouched by transport, so one step lowers m1 u by K m0 u dt
    (closed form for n(S) = C: (C/2) u - K C u dt) and keeps u."""
    n, C, K, dt = 20, 0.8, 0.3, 0.01
    u, v = 0.3, -0.2
    prim = np.empty((6, n, n))
    for k in range(4):
        prim[k] = C / (1 + k / 2)
    prim[4], prim[5] = u, v
    d = wl.problem("spray", n, n, fixed_dt=dt, params=(K, 0.0, 0.0, 32.0, 1e-13))
    out, _ = gpu_run(d, prim, 1)
    np.testing.assert_allclose(out[4], C / 2 * u - K * C * u * dt, rtol=4e-15, atol=0)
    np.testing.assert_allclose(out[5], C / 2 * v - K * C * v * dt, rtol=4e-15, atol=0)
    np.testing.assert_allclose(out[4] / out[2], u, rtol=4e-15, atol=0)
    np.testing.assert_allclose(out[5] / out[2], v, rtol=4e-15, atol=0)


def test_spray_drag_toward_taylor_green_gas_field():
    """Drag with the Taylor-Green gas field on droplets at rest in a uniform
    field (K = 0): one step gives m1 u = dt m0 u_g(x_i, y_j) / theta, with u_g
    evaluated here at the cell centres of a non-square grid, and keeps every
    moment."""
    nx, ny = 40, 24
    theta, dt = 0.25, 0.003
    m = wl.canonical_to_moments(1.1, 0.6, 0.3, 0.55)
    prim = np.zeros((6, ny, nx))
    for k in range(4):
        prim[k] = m[k]
    d = wl.problem("spray", nx, ny, fixed_dt=dt, params=(0.0, theta, 1.0, 32.0, 1e-13))
    out, _ = gpu_run(d, prim, 1)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    ug = np.outer(np.cos(2 * np.pi * y), np.sin(2 * np.pi * x))
    vg = -np.outer(np.sin(2 * np.pi * y), np.cos(2 * np.pi * x))
    np.testing.assert_allclose(out[4], dt * m[0] * ug / theta, rtol=0, atol=1e-16)
    np.testing.assert_allclose(out[5], dt * m[0] * vg / theta, rtol=0, atol=1e-16)
    for k in range(4):
        assert np.all(out[k] == m[k])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_spray_parity_long_run_across_cache_refreshes(precision):
    """256^2, 130 steps: the per-cell exponentials are updated from their
    last solve and recomputed in full every 32 steps (steps 32, 64, 96 and
    128 fall inside the run), so this checks that the roundings of up to 31
    updates in a row stay inside the tolerance."""
    prim, d = wl.spray_field(256)
    ref = oracle_run(d, prim, 130)
    out, t = gpu_run(d, prim, 130, precision)
    if precision == "f64":
        assert rel_linf(out, ref.W).max() <= 1e-12, rel_linf(out, ref.W)
        assert abs(t - ref.t) <= 1e-13 * ref.t
    else:
        assert rel_l1(out, ref.W).max() <= 1e-5, rel_l1(out, ref.W)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_spray_parity_wide_moment_recipe(precision):
    """Moments spread over the moment space (canonical moments 0.25..0.75
    +- 0.2, densities far from a constant): the cold-start damped Newton runs
    its Armijo steps on every cell of the first step.  256^2, 100 steps (the
    oracle stays admissible for 400 steps at this resolution)."""
    prim, d = wl.spray_field_wide(256)
    ref = oracle_run(d, prim, 100)
    out, t = gpu_run(d, prim, 100, precision)
    if precision == "f64":
        assert rel_linf(out, ref.W).max() <= 1e-12, rel_linf(out, ref.W)
        assert abs(t - ref.t) <= 1e-13 * ref.t
    else:
        assert rel_l1(out, ref.W).max() <= 1e-5, rel_l1(out, ref.W)


def test_spray_wide_recipe_leaves_moment_space_at_the_oracles_step():
    """At 128^2 the CFL step is large enough that forward-Euler evaporation
    drives some cell of the wide recipe out of the moment space in the first
    step (reading G16): the oracle stops there with a non-physical status and
    the GPU must report the same error at the same step."""
    prim, d = wl.spray_field_wide(128)
    P = oracle_problem(d)
    r = oracle.run(P, oracle.prim_to_cons(P, prim), 10)
    assert r.status == oracle.ERR_NONPHYSICAL and r.steps == 0
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(np.ascontiguousarray(prim), primitive=True)
        st, _ = s.run(10, check=False)
        assert st == f.FV_ERR_NONPHYSICAL
        _, step = s.time()
        assert step <= 1, step   # the failing step is the first one
