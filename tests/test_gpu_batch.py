"""Batched instances in one persistent launch (fv_batch_*): every instance
must give the same bits as when it runs alone through fv_run (same
arithmetic, its own dt and t), match the FP64 oracle, and a wait that cannot
complete must end the launch with FV_ERR_TIMEOUT (bounded device waits)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as wl
from tests.helpers import oracle_problem, rel_l1, rel_linf, with_fixed_dt

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


def small_batch(n=10, lo=17, hi=180, seed=5):
    return wl.batched_quadrants(n, seed=seed, lo=lo, hi=hi)


def run_batch(insts, steps, precision, tune=0):
    f = fv()
    with f.Batch([d for _, _, d in insts], precision, tune=tune) as b:
        for k, (_, prim, _) in enumerate(insts):
            b.set_state(k, prim, primitive=True)
        b.run(steps)
        return [b.state(k) for k in range(len(insts))], [b.time(k) for k in range(len(insts))]


def run_single(d, prim, steps, precision):
    f = fv()
    with f.Solver(d, precision) as s:
        s.set_state(prim, primitive=True)
        s.run(steps)
        return s.state(), s.time()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batch_equals_single_bitwise(precision):
    insts = small_batch()
    outs, times = run_batch(insts, 40, precision)
    for k, (_, prim, d) in enumerate(insts):
        W, tt = run_single(d, prim, 40, precision)
        assert np.array_equal(outs[k], W), k
        assert times[k] == tt, (k, times[k], tt)


def test_batch_fp64_matches_oracle():
    insts = small_batch(6, seed=8)
    outs, times = run_batch(insts, 30, "f64")
    for k, (_, prim, d) in enumerate(insts):
        P = oracle_problem(d)
        r = oracle.run(P, oracle.prim_to_cons(P, prim), 30)
        assert r.status == oracle.OK
        assert rel_linf(outs[k], r.W).max() <= 1e-12, k
        assert abs(times[k][0] - r.t) <= 1e-13 * r.t


def test_batch_instances_keep_their_own_dt():
    insts = small_batch(4, seed=9)
    _, times = run_batch(insts, 10, "f64")
    ts = [t for t, _ in times]
    assert len(set(ts)) == len(ts)  # different sizes and states, different dt
    assert all(n == 10 for _, n in times)


def test_batch_every_candidate_same_bits():
    insts = small_batch(5, seed=3)
    f = fv()
    outs = []
    k = 0
    while True:
        try:
            o, _ = run_batch(insts, 12, "f32", tune=2 + k)
        except f.FvError:
            break
        outs.append(o)
        k += 1
    assert len(outs) >= 2
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_batch_autotuner_keeps_state_time_and_bits():
    """tune = 1 times one step of every candidate on the batch's own state
    before the first run; the control blocks are put back, so the results,
    times and step counts equal those of the untuned run."""
    insts = small_batch(6, seed=13)
    base, tb = run_batch(insts, 15, "f32", tune=0)
    tuned, tt = run_batch(insts, 15, "f32", tune=1)
    for a, b in zip(tuned, base):
        assert np.array_equal(a, b)
    assert tt == tb


def test_batch_c4_distribution_fp32_vs_oracle():
    """64 instances drawn like the 512 of the batched workload (sizes 64..1024,
    random four-quadrant states), 200 steps in one launch; the three smallest
    are checked against the FP64 oracle (relative L1 <= 1e-5 is not
    meaningful across shocks, so the bound is 1e-4 relative L1 here)."""
    insts = wl.batched_quadrants(64)
    outs, times = run_batch(insts, 200, "f32")
    sizes = [d["nx"] * d["ny"] for _, _, d in insts]
    for k in np.argsort(sizes)[:3]:
        _, prim, d = insts[k]
        P = oracle_problem(d)
        r = oracle.run(P, oracle.prim_to_cons(P, prim), 200)
        assert r.status == oracle.OK
        assert rel_l1(outs[k], r.W).max() <= 1e-4, (k, rel_l1(outs[k], r.W))
        assert abs(times[k][0] - r.t) <= 1e-5 * r.t


def test_batch_wait_timeout_is_reported():
    """An instance whose steps are never released makes the next step's wait
    run out: the launch ends with FV_ERR_TIMEOUT after about the limit, and
    the device stays usable."""
    f = fv()
    insts = small_batch(4, seed=11)
    with f.Batch([d for _, _, d in insts], "f32") as b:
        for k, (_, prim, _) in enumerate(insts):
            b.set_state(k, prim, primitive=True)
        b.set_wait_limit(0.2, never_release_instance=2)
        st = b.run(5, check=False)
        assert st == f.FV_ERR_TIMEOUT
    # the GPU still works
    _, prim, d = insts[0]
    W, _ = run_single(d, prim, 3, "f64")
    assert np.all(np.isfinite(W))


# ------------------------------------------------------------------ dataflow
def run_batch_mode(insts, steps, precision, dataflow, check=True):
    f = fv()
    with f.Batch([d for _, _, d in insts], precision) as b:
        for k, (_, prim, _) in enumerate(insts):
            b.set_state(k, prim, primitive=True)
        if dataflow:
            b.set_dataflow(True)
        st = b.run(steps, check=check)
        return st, [b.state(k) for k in range(len(insts))], [b.time(k) for k in range(len(insts))]


def fixed_dt_batch(seed=21):
    """Transmissive four-quadrant instances and periodic smooth ones (whose
    halos wrap around, so their tasks depend on tasks across the boundary),
    all in the paper's fixed-dt mode at CFL 0.4."""
    insts = [(k, prim, with_fixed_dt(d, prim, 0.4)) for k, prim, d in small_batch(5, seed=seed)]
    for k, (n, m) in enumerate([(97, 61), (150, 33), (31, 200)]):
        prim, d = wl.random_smooth_euler(n, seed=seed + k, ny=m)
        insts.append((100 + k, prim, with_fixed_dt(d, prim, 0.4)))
    return insts


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_dataflow_equals_step_gated_bitwise(precision):
    """Neighbour dependencies instead of a barrier per step change nothing:
    states, times and step counts are identical to the step-gated run."""
    insts = fixed_dt_batch()
    st0, W0, t0 = run_batch_mode(insts, 37, precision, False)
    st1, W1, t1 = run_batch_mode(insts, 37, precision, True)
    assert st0 == st1 == fv().FV_OK
    for a, b in zip(W1, W0):
        assert np.array_equal(a, b)
    assert t1 == t0


def test_dataflow_flagged_instance_is_replayed_exactly():
    """An instance whose Dirichlet inflow has a negative density becomes
    inadmissible during the run: the dataflow run flags it, puts it back to
    its state at the start and replays it step-gated, so status, state and
    step count equal the step-gated run's; the other instances are untouched.
    A second instance violates the paper's check at its first step (fixed dt
    above min(dx, dy) / lmax) and never advances, in both modes."""
    insts = fixed_dt_batch(seed=33)
    k, prim, d = insts[2]
    bad = dict(d, bc=("transmissive", "transmissive", "dirichlet", "transmissive"),
               bc_state=((0,) * 4, (0,) * 4, (-1.0, 0.5, 0.0, 2.0), (0,) * 4))
    insts[2] = (k, prim, bad)
    k, prim, d = insts[4]
    insts[4] = (k, prim, dict(d, fixed_dt=d["fixed_dt"] * 3.0))
    st0, W0, t0 = run_batch_mode(insts, 25, "f32", False, check=False)
    st1, W1, t1 = run_batch_mode(insts, 25, "f32", True, check=False)
    assert st0 == st1 and st0 in (fv().FV_ERR_NONPHYSICAL, fv().FV_ERR_CFL)
    for a, b in zip(W1, W0):
        assert np.array_equal(a, b, equal_nan=True)
    assert t1 == t0
    assert t0[4][1] == 0 and t0[2][1] < 25 and t0[0][1] == 25


def test_dataflow_needs_fixed_dt():
    f = fv()
    insts = small_batch(3, seed=2)
    with f.Batch([d for _, _, d in insts], "f32") as b:
        with pytest.raises(f.FvError) as e:
            b.set_dataflow(True)
        assert e.value.status == f.FV_ERR_INVALID_ARG


def test_dataflow_wait_timeout_is_reported():
    """In dataflow mode too, a dependency that is never released ends the
    launch with FV_ERR_TIMEOUT after about the limit, and the device stays
    usable."""
    f = fv()
    insts = fixed_dt_batch(seed=44)
    with f.Batch([d for _, _, d in insts], "f32") as b:
        for k, (_, prim, _) in enumerate(insts):
            b.set_state(k, prim, primitive=True)
        b.set_dataflow(True)
        b.set_wait_limit(0.2, never_release_instance=1)
        assert b.run(5, check=False) == f.FV_ERR_TIMEOUT
    _, prim, d = insts[0]
    W, _ = run_single(d, prim, 3, "f64")
    assert np.all(np.isfinite(W))
