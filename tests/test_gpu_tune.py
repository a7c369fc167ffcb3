"""The autotuner's recorded kernel table (csrc/fv_tune_table.inc, written by
python -m paper_1701_05431_gb300.autotune): a context created with tune = 0
runs the candidate the table names for its (system, precision, grid-size
class, mode) and says so; keys the table lacks fall back to the heuristic;
forcing and leaving in-place mode keep the choice consistent."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                     "paper_1701_05431_gb300", "tune_table.json")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fv():
    from paper_1701_05431_gb300 import fvlib
    return fvlib


def recorded():
    if not os.path.exists(TABLE):
        pytest.skip("no autotune table recorded")
    with open(TABLE) as f:
        return json.load(f)


def _problem(name):
    if name.startswith("c3"):
        return wl.problem("euler", 8192, 8192)
    if name.startswith("c2"):
        return wl.four_quadrant(2048, npart=8)[1]
    if name.startswith("c5"):
        return wl.problem("spray", 2048, 2048)
    return wl.problem("advection", 128, 128)


def test_single_instance_entries_are_used():
    f = fv()
    for r in recorded():
        if r["mode"] == "batch":
            continue
        best = max(r["candidates"], key=lambda kv: kv[1])[0]
        d = _problem(r["name"])
        if r["mode"] == "two-step":
            d = dict(d, fixed_dt=1e-6)
        with f.Solver(d, r["precision"]) as s:
            if r["mode"] == "inplace":
                s.set_inplace(True)
            if r["mode"] == "two-step":
                s.set_time_blocking(2)
                assert s.two_step_kernel() == best, (r["name"], s.two_step_kernel())
                assert s.kernel_choice(two_step=True).startswith("table:"), r["name"]
            else:
                assert s.kernel_info()[1].split(", ")[0] == best, (r["name"], s.kernel_info())
                assert s.kernel_choice().startswith("table:"), (r["name"], s.kernel_choice())


def test_batched_entry_is_used():
    f = fv()
    rows = [r for r in recorded() if r["mode"] == "batch"]
    if not rows:
        pytest.skip("no batched entry")
    best = max(rows[0]["candidates"], key=lambda kv: kv[1])[0]
    insts = wl.batched_quadrants(512)
    with f.Batch([d for _, _, d in insts], "f32") as b:
        assert b.kernel_info()[1] == best
        assert b.kernel_choice().startswith("table:")


def test_unlisted_key_takes_the_heuristic_and_forcing_is_reported():
    f = fv()
    d = wl.problem("euler", 300, 200)        # an Euler grid below 2^16 cells: no entry
    with f.Solver(d, "f32") as s:
        assert s.kernel_choice().startswith("heuristic")
    with f.Solver(d, "f32", tune=3) as s:
        assert s.kernel_choice() == "forced: candidate 1"
        assert s.kernel_info()[0] == 1


def test_leaving_inplace_mode_restores_the_two_buffer_kernel():
    f = fv()
    prim, d = wl.random_smooth_euler(96, seed=3, ny=64)
    with f.Solver(d, "f32", tune=4) as s:
        k0, c0 = s.kernel_info(), s.kernel_choice()
        s.set_state(prim, primitive=True)
        s.set_inplace(True)
        assert "inplace" in s.kernel_info()[1]
        s.run(3)
        s.set_inplace(False)
        assert s.kernel_info() == k0 and s.kernel_choice() == c0
        s.run(3)
        out = s.state()
    with f.Solver(d, "f32", tune=4) as s:
        s.set_state(prim, primitive=True)
        s.run(6)
        assert np.array_equal(s.state(), out)
