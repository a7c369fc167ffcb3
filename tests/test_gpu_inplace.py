"""In-place mode (fv_set_inplace): one state buffer updated in place, halos
from overlap strips written by the producing tasks.  It must give the bits
of the default two-buffer mode, for every precision, boundary condition and
ragged tiling, keep state, time and step across switches, and serve
fv_get_state / fv_totals / fv_snapshot / fv_set_time as before."""
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


def run(d, prim, steps, precision, inplace):
    f = fv()
    with f.Solver(d, precision) as s:
        if inplace:
            s.set_inplace(True)
        s.set_state(prim, primitive=True)
        s.run(steps)
        return s.state(), s.time(), s.kernel_info()[1]


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("bc", sorted(BCS))
@pytest.mark.parametrize("shape", [(193, 141), (64, 64), (31, 5), (121, 67), (250, 40)])
def test_inplace_equals_two_buffers_bitwise(precision, bc, shape):
    nx, ny = shape
    prim, d = wl.random_smooth_euler(nx, seed=7 + nx, ny=ny)
    d = dict(d, **BCS[bc])
    W0, t0, _ = run(d, prim, 23, precision, False)
    W1, t1, k1 = run(d, prim, 23, precision, True)
    assert "inplace" in k1
    assert np.array_equal(W1, W0), (precision, bc, shape)
    assert t1 == t0


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("bc", ["mixed", "dirichlet", "transmissive"])
def test_every_inplace_candidate_equals_two_buffers(precision, bc):
    """Every compiled in-place candidate (cells per lane, rows per task,
    blocks per SM, ring depth) gives the two-buffer mode's bits."""
    f = fv()
    prim, d = wl.random_smooth_euler(193, seed=11, ny=141)
    d = dict(d, **BCS[bc])
    W0, t0, _ = run(d, prim, 17, precision, False)
    names = []
    k = 0
    while True:
        try:
            s = f.Solver(d, precision, tune=2 + k)
        except f.FvError:
            break
        with s:
            try:
                s.set_inplace(True)
            except f.FvError:
                break
            s.set_state(prim, primitive=True)
            s.run(17)
            names.append(s.kernel_info()[1])
            assert np.array_equal(s.state(), W0), names[-1]
            assert s.time() == t0
        k += 1
    assert len(names) >= 2 and all("inplace" in n for n in names)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_inplace_advection_equals_two_buffers(precision):
    prim, d = wl.advection_bump(128)
    d = dict(d, nx=128, ny=97)
    prim = np.ascontiguousarray(prim[:, :97, :])
    W0, t0, _ = run(d, prim, 40, precision, False)
    W1, t1, _ = run(d, prim, 40, precision, True)
    assert np.array_equal(W1, W0) and t1 == t0


def test_switching_keeps_state_time_and_step():
    """10 steps in two buffers, 11 in place, 12 in two buffers again (odd
    counts, so the state changes buffer parity at every switch) equal 33
    steps in two buffers; snapshots, totals and set_time work in place."""
    prim, d = wl.random_smooth_euler(150, seed=3, ny=90)
    W_ref, t_ref, _ = run(d, prim, 33, "f32", False)
    f = fv()
    with f.Solver(d, "f32") as s:
        s.set_state(prim, primitive=True)
        s.run(11)
        s.set_inplace(True)
        s.run(11)
        snap = np.empty((4, 90, 150), dtype=np.float32)
        s.snapshot(snap)
        s.snapshot_wait()
        assert np.array_equal(snap, s.state("float32"))
        tot_in = s.totals()
        s.set_inplace(False)
        assert np.array_equal(s.totals(), tot_in)
        s.run(11)
        W, t = s.state(), s.time()
    assert np.array_equal(W, W_ref) and t == t_ref
    # set_time changes the step parity: the strips follow
    with f.Solver(d, "f64") as s:
        s.set_inplace(True)
        s.set_state(prim, primitive=True)
        s.set_time(0.0, 1)
        s.run(5)
        Wa = s.state()
    with f.Solver(d, "f64") as s:
        s.set_state(prim, primitive=True)
        s.set_time(0.0, 1)
        s.run(5)
        Wb = s.state()
    assert np.array_equal(Wa, Wb)


def test_inplace_frees_the_second_buffer():
    f = fv()
    prim, d = wl.random_smooth_euler(4096, seed=1)
    torch.cuda.synchronize()
    with f.Solver(d, "f32") as s:
        s.set_state(prim, primitive=True)
        free0, _ = torch.cuda.mem_get_info()
        s.set_inplace(True)
        free1, _ = torch.cuda.mem_get_info()
        # 256 MiB of state freed, about 28% of it taken back by the strips
        # (two parities of four border strips per warp task; the column
        # strips hold the four cells of a halo lane per row)
        assert free1 - free0 > 160 * 2 ** 20, (free0, free1)
        s.run(3)


def test_inplace_rejects_spray():
    f = fv()
    _, d = wl.spray_field(32)
    with f.Solver(d, "f64") as s:
        with pytest.raises(f.FvError) as e:
            s.set_inplace(True)
        assert e.value.status == f.FV_ERR_INVALID_ARG
