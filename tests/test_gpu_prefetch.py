"""Asynchronous input (fv_prefetch_state / fv_set_state_prefetched): a state
copied in from host memory while earlier steps run loads exactly as
fv_set_state loads it, and the run from it is the run from fv_set_state."""
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


def run_from(d, prim, precision, steps, primitive=True):
    with fv().Solver(d, precision) as s:
        s.set_state(prim, primitive=primitive)
        s.run(steps)
        return s.state()


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
def test_prefetch_overlaps_a_run_and_loads_like_set_state(precision):
    primA, d = wl.random_smooth_euler(131, seed=51, ny=77)
    primB, _ = wl.random_smooth_euler(131, seed=52, ny=77)
    hB = torch.from_numpy(np.ascontiguousarray(primB.astype(np.float32))).pin_memory()
    refB = run_from(d, hB.numpy(), precision, 15)
    with fv().Solver(d, precision) as s:
        s.set_state(primA, primitive=True)
        s.prefetch_state(hB, primitive=True)   # copied while the steps of A run
        s.run(20)
        s.set_state_prefetched()
        assert s.time() == (0.0, 0)
        s.run(15)
        got = s.state()
    assert np.array_equal(got, refB)


def test_prefetched_state_is_the_set_state_bit_for_bit():
    prim, d = wl.random_smooth_euler(96, seed=53, ny=64)
    W = np.ascontiguousarray(prim)                     # float64, pageable
    with fv().Solver(d, "f64") as a, fv().Solver(d, "f64") as b:
        a.set_state(W, primitive=True)
        b.prefetch_state(W, primitive=True)
        b.set_state_prefetched()
        assert np.array_equal(a.state(), b.state())
        assert a.totals().tolist() == b.totals().tolist()


def test_conserved_layout_and_last_prefetch_wins():
    primA, d = wl.random_smooth_euler(80, seed=54)
    primB, _ = wl.random_smooth_euler(80, seed=55)
    with fv().Solver(d, "f64") as s:
        s.set_state(primB, primitive=True)
        WB = s.state()                                 # conserved variables of B
        s.prefetch_state(np.ascontiguousarray(primA), primitive=True)
        s.prefetch_state(WB)                           # replaces the first prefetch
        s.set_state_prefetched()
        assert np.array_equal(s.state(), WB)


def test_prefetch_errors():
    prim, d = wl.random_smooth_euler(48, seed=56)
    with fv().Solver(d, "f32") as s:
        with pytest.raises(fv().FvError):
            s.set_state_prefetched()                   # nothing prefetched
        with pytest.raises(ValueError):
            s.prefetch_state(np.zeros((4, 48, 47)))   # wrong size
        with pytest.raises(ValueError):
            s.prefetch_state(torch.zeros((4, 48, 48), device="cuda"))  # not host memory
        s.prefetch_state(np.ascontiguousarray(prim), primitive=True)
        s.set_state_prefetched()
        with pytest.raises(fv().FvError):
            s.set_state_prefetched()                   # consumed


def test_prefetch_of_nonphysical_state_is_rejected():
    prim, d = wl.random_smooth_euler(40, seed=57)
    bad = np.ascontiguousarray(prim.copy())
    bad[0, 5, 7] = -1.0                                # negative density
    with fv().Solver(d, "f64") as s:
        s.prefetch_state(bad, primitive=True)
        assert s.set_state_prefetched(check=False) == fv().FV_ERR_NONPHYSICAL
        s.prefetch_state(np.ascontiguousarray(prim), primitive=True)
        s.set_state_prefetched()
        s.run(3)
