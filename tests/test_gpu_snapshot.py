"""Asynchronous snapshots (fv_snapshot / fv_snapshot_wait): the host copy
holds the state of the step at which it was taken, bit for bit, even while
later steps run, and taking snapshots changes nothing in the run."""
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


def reference_states(d, prim, precision, steps):
    out = {}
    with fv().Solver(d, precision) as s:
        s.set_state(prim, primitive=True)
        done = 0
        for n in sorted(steps):
            s.run(n - done)
            done = n
            out[n] = s.state()
    return out


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
def test_snapshots_overlap_later_steps_and_hold_their_step(precision):
    prim, d = wl.random_smooth_euler(157, seed=41, ny=97)
    ref = reference_states(d, prim, precision, [7, 19, 40])
    shape = (4, 97, 157)
    a = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    b = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    with fv().Solver(d, precision) as s:
        s.set_state(prim, primitive=True)
        s.run(7)
        s.snapshot(a)
        s.run(12)        # runs while the copy of step 7 may be in flight
        s.snapshot(b)    # waits on the device for the first copy, not on the host
        s.run(21)
        s.snapshot_wait()
        final = s.state()
    assert np.array_equal(a.numpy(), ref[7])
    assert np.array_equal(b.numpy(), ref[19])
    assert np.array_equal(final, ref[40])


def test_snapshot_float32_and_pageable_target():
    prim, d = wl.random_smooth_euler(64, seed=43)
    with fv().Solver(d, "f64") as s:
        s.set_state(prim, primitive=True)
        s.run(5)
        want = s.state()
        out = np.empty((4, 64, 64), dtype=np.float32)   # pageable: the copy completes in the call
        s.snapshot(out)
        s.snapshot_wait()
        s.snapshot_wait()                               # nothing pending: returns at once
    assert np.array_equal(out, want.astype(np.float32))


def test_snapshot_rejects_bad_arguments():
    f = fv()
    prim, d = wl.random_smooth_euler(16, seed=1)
    with f.Solver(d, "f64") as s:
        with pytest.raises(f.FvError) as e:
            s.snapshot(np.empty((4, 16, 16)))                 # no state yet
        assert e.value.status == f.FV_ERR_STATE
        s.set_state(prim, primitive=True)
        with pytest.raises(TypeError):
            s.snapshot(np.empty((4, 16, 16), dtype=np.float16))
        with pytest.raises(ValueError):
            s.snapshot(torch.empty((4, 16, 16), dtype=torch.float64, device="cuda"))
    L = f.load()
    assert L.fv_snapshot(None, None, 0) == f.FV_ERR_INVALID_ARG
    assert L.fv_snapshot_wait(None) == f.FV_ERR_INVALID_ARG
