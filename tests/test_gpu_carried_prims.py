"""FP64 Euler kernels that carry the primitives (u, v, p, c) of every cell
from step to step: their results are the batched kernel's (a separate code
path, which carries them too) on every boundary condition, and those of the
two-step kernel (which recomputes them) across switches between the modes,
bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fv():
    from paper_1701_05431_gb300 import fvlib
    return fvlib


BCS = {
    "periodic": dict(bc=("periodic",) * 4),
    "transmissive": dict(bc=("transmissive",) * 4),
    "dirichlet": dict(bc=("dirichlet",) * 4, bc_state=((1.05, 0.1, -0.05, 2.6),) * 4),
    "mixed": dict(bc=("transmissive", "periodic", "dirichlet", "periodic"),
                  bc_state=((0,) * 4, (0,) * 4, (1.05, 0.1, -0.05, 2.6), (0,) * 4)),
}


@pytest.mark.parametrize("bc", sorted(BCS))
def test_carried_primitives_match_the_batched_kernel(bc):
    prim, d = wl.random_smooth_euler(157, seed=61, ny=93)
    d = dict(d, **BCS[bc])
    f = fv()
    with f.Solver(d, "f64") as s:
        assert s.kernel_info()[1].split(",")[0].endswith(" pc")
        s.set_state(prim, primitive=True)
        s.run(40)
        W, t = s.state(), s.time()
    with f.Batch([d], "f64") as b:
        b.set_state(0, prim, primitive=True)
        b.run(40)
        Wb, tb = b.state(0), b.time(0)
    assert np.array_equal(W, Wb)
    assert t == tb


def test_in_place_round_trip_refreshes_the_primitives():
    prim, d = wl.random_smooth_euler(131, seed=62, ny=75)
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(prim, primitive=True)
        s.run(15)
        ref = s.state()
    with f.Solver(d, "f64") as s:
        s.set_state(prim, primitive=True)
        s.run(5)
        s.set_inplace(True)     # planes 0..3 only
        s.run(5)
        s.set_inplace(False)    # the carried planes are stale here
        s.run(5)
        got = s.state()
    assert np.array_equal(got, ref)


def test_two_step_passes_then_single_steps():
    prim, d = wl.random_smooth_euler(96, seed=63, ny=64)
    rho, u, v, p = prim
    lam0 = float(np.max(np.maximum(np.abs(u), np.abs(v)) + np.sqrt(1.4 * p / rho)))
    d = dict(d, fixed_dt=0.4 / 96 / lam0)
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(prim, primitive=True)
        s.run(9)
        ref = s.state()
    with f.Solver(d, "f64") as s:
        s.set_time_blocking(2)
        s.set_state(prim, primitive=True)
        s.run(9)                # four two-step passes, then one single step
        s.set_time_blocking(1)
        got = s.state()
    assert np.array_equal(got, ref)


def test_restart_from_a_checkpoint():
    prim, d = wl.random_smooth_euler(88, seed=64, ny=70)
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(prim, primitive=True)
        s.run(12)
        mid, (t, n) = s.state(), s.time()
        s.run(8)
        ref = s.state()
    with f.Solver(d, "f64") as s:
        s.set_state(mid)        # conserved variables of step 12
        s.set_time(t, n)
        s.run(8)
        got = s.state()
    assert np.array_equal(got, ref)
