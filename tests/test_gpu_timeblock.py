"""Two time steps per launch (fv_set_time_blocking): in the paper's fixed-dt
mode a pass reads and writes the state once per two steps, on periodic,
transmissive and Dirichlet sides alike.
It must give the bits, times, step counts and errors of one step per
launch: also when the intermediate state fails the paper's check
dt lmax <= min(dx, dy) (the pass is void and the steps are redone one at a
time), when the state becomes inadmissible, and for odd step counts."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as wl
from tests.helpers import with_fixed_dt

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fv():
    from paper_1701_05431_gb300 import fvlib
    return fvlib


def run(d, prim, steps, precision, passes, split=None):
    f = fv()
    with f.Solver(d, precision) as s:
        s.set_state(prim, primitive=True)
        if passes:
            s.set_time_blocking(2)
        st = f.FV_OK
        for n in (split or [steps]):
            st, _ = s.run(n, check=False)
            if st != f.FV_OK:
                break
        return st, s.state(), s.time()


@pytest.mark.parametrize("precision", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("shape", [(193, 141), (64, 64), (31, 5), (7, 3), (250, 40)])
@pytest.mark.parametrize("steps", [23, 24])
def test_two_steps_per_pass_equal_single_steps(precision, shape, steps):
    nx, ny = shape
    prim, d = wl.random_smooth_euler(nx, seed=3 + nx, ny=ny)
    d = with_fixed_dt(d, prim, 0.4)
    a = run(d, prim, steps, precision, False)
    b = run(d, prim, steps, precision, True)
    assert a[0] == b[0] == fv().FV_OK
    assert np.array_equal(b[1], a[1])
    assert b[2] == a[2] == (a[2][0], steps)


FAR = (1.0137, 0.1013 * 1.0137, -0.0521 * 1.0137, 2.5173)  # a Dirichlet state (conserved variables)
BC_MIXES = {
    "transmissive": dict(bc=("transmissive",) * 4),
    "dirichlet": dict(bc=("dirichlet",) * 4, bc_state=(FAR,) * 4),
    "mixed": dict(bc=("dirichlet", "transmissive", "transmissive", "dirichlet"), bc_state=(FAR,) * 4),
    "x-periodic": dict(bc=("periodic", "dirichlet", "periodic", "transmissive"), bc_state=(FAR,) * 4),
    "y-periodic": dict(bc=("transmissive", "periodic", "dirichlet", "periodic"), bc_state=(FAR,) * 4),
}


@pytest.mark.parametrize("precision", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("shape", [(193, 141), (60, 64), (31, 5), (7, 3), (250, 40), (1, 9), (122, 2)])
@pytest.mark.parametrize("bcs", sorted(BC_MIXES))
def test_two_steps_per_pass_equal_single_steps_non_periodic(precision, shape, bcs):
    """On a transmissive or Dirichlet side a pass gives the ghosts of the
    intermediate state W^{n+1} the boundary condition (a copy of the border
    cell as stored, or the prescribed state): the bits of one step per
    launch, for strips that end on, before and past the last column."""
    nx, ny = shape
    prim, d = wl.random_smooth_euler(nx, seed=5 + nx, ny=ny)
    d = with_fixed_dt(dict(d, **BC_MIXES[bcs]), prim, 0.4)
    a = run(d, prim, 21, precision, False)
    b = run(d, prim, 21, precision, True)
    assert a[0] == b[0] == fv().FV_OK
    assert np.array_equal(b[1], a[1])
    assert b[2] == a[2] == (a[2][0], 21)


def test_two_steps_per_pass_four_quadrant_transmissive():
    """The 2048^2 four-quadrant Riemann problem on transmissive sides (the
    setting of the 8 x 8-subdomain workload) in the paper's fixed-dt mode."""
    prim, d = wl.four_quadrant(512, npart=8)
    d = with_fixed_dt(d, prim, 0.4)
    a = run(d, prim, 40, "f32", False)
    b = run(d, prim, 40, "f32", True)
    assert a[0] == b[0] == fv().FV_OK
    assert np.array_equal(b[1], a[1]) and b[2] == a[2]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_two_steps_per_pass_advection_dirichlet_inflow(precision):
    """Scalar advection entering through a Dirichlet west side and leaving
    through a transmissive east side."""
    prim, d = wl.advection_bump(96)
    d = dict(d, fixed_dt=0.45 / 96, cfl=0.0, bc=("transmissive", "periodic", "dirichlet", "periodic"),
             bc_state=((0.0,), (0.0,), (1.3,), (0.0,)))
    a = run(d, prim, 37, precision, False)
    b = run(d, prim, 37, precision, True)
    assert a[0] == b[0] == fv().FV_OK
    assert np.array_equal(b[1], a[1]) and b[2] == a[2]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_two_steps_per_pass_advection(precision):
    prim, d = wl.advection_bump(128)
    d = dict(d, fixed_dt=0.5 / 128, cfl=0.0)
    a = run(d, prim, 51, precision, False)
    b = run(d, prim, 51, precision, True)
    assert a[0] == b[0] == fv().FV_OK
    assert np.array_equal(b[1], a[1]) and b[2] == a[2]


def blob(n=64):
    """A high-pressure bump in a periodic box: lmax grows in the first steps."""
    x = wl.centres(n)
    r2 = (x[None, :] - 0.5) ** 2 + (x[:, None] - 0.5) ** 2
    prim = np.empty((4, n, n))
    prim[0] = 1.0
    prim[1] = 0.3
    prim[2] = -0.2
    prim[3] = 1.0 + 9.0 * np.exp(-r2 / 0.005)
    lam0 = np.max(np.maximum(np.abs(prim[1]), np.abs(prim[2])) + np.sqrt(1.4 * prim[3] / prim[0]))
    return prim, wl.problem("euler", n, n, cfl=0.4), lam0


@pytest.mark.parametrize("factor, first_bad", [(0.999, 1), (0.99, 2), (0.97, None)])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_failing_check_and_inadmissible_states_match(factor, first_bad, precision):
    """dt = factor min(dx, dy) / lmax(W^0): with 0.999 the check fails at step
    1 (inside the first pass: the pass is void and redone step by step), with
    0.99 at step 2 (at the start of the second pass); with 0.97 the state
    turns inadmissible later on.  Status, state, time and step count are
    those of one step per launch."""
    prim, d, lam0 = blob()
    d = dict(d, fixed_dt=factor * (1.0 / 64) / lam0)
    a = run(d, prim, 40, precision, False)
    b = run(d, prim, 40, precision, True)
    assert a[0] == b[0] != fv().FV_OK
    if first_bad is not None:
        assert a[0] == fv().FV_ERR_CFL and a[2][1] == first_bad
    assert np.array_equal(b[1], a[1], equal_nan=True)
    assert b[2] == a[2]


def test_switching_and_split_runs():
    prim, d = wl.random_smooth_euler(150, seed=8, ny=90)
    d = with_fixed_dt(d, prim, 0.4)
    ref = run(d, prim, 30, "f32", False)
    f = fv()
    with f.Solver(d, "f32") as s:
        s.set_state(prim, primitive=True)
        s.run(5)
        assert s.two_step_kernel() is None
        s.set_time_blocking(2)
        assert "tb2" in s.two_step_kernel()
        s.run(7)
        s.run(10)
        snap = np.empty((4, 90, 150), dtype=np.float32)
        s.snapshot(snap)
        s.snapshot_wait()
        s.set_time_blocking(1)
        s.run(8)
        W, t = s.state(), s.time()
    assert np.array_equal(W, ref[1]) and t == ref[2]
    assert np.array_equal(snap.astype(np.float64), run(d, prim, 22, "f32", False)[1])


def test_time_blocking_preconditions():
    f = fv()
    prim, d = wl.random_smooth_euler(64, seed=2)
    with f.Solver(d, "f32") as s:                      # adaptive dt
        with pytest.raises(f.FvError) as e:
            s.set_time_blocking(2)
        assert e.value.status == f.FV_ERR_INVALID_ARG
    d2 = with_fixed_dt(dict(d, bc=("transmissive",) * 4), prim, 0.4)
    with f.Solver(d2, "f32") as s:                     # non-periodic sides are accepted
        s.set_time_blocking(2)
        assert "tb2" in s.two_step_kernel()
    d3 = with_fixed_dt(d, prim, 0.4)
    with f.Solver(d3, "f32") as s:
        s.set_time_blocking(2)
        with pytest.raises(f.FvError):
            s.set_inplace(True)                        # not both
        with pytest.raises(f.FvError):
            s.set_time_blocking(3)
