"""Full-size parity in the benchmarked launch configuration, against sampled
FP64-oracle outputs written by tests/golden/make_oracle_samples.py (the
oracle needs minutes for these sizes, so it is not rerun here).

  C2: Euler 2048^2, four-quadrant Riemann data, 8 x 8 subdomains,
      transmissive, CFL 0.4, 500 steps, FP64.
  C3: Euler 8192^2, smooth periodic data, CFL 0.4, 100 steps, FP64 and FP32.
  C5: spray moments 2048^2, periodic, CFL 0.4, 40 steps (the first full
      recomputation of every cell's cached exponentials is at step 32),
      FP64 and FP32 storage.

FP64 <= 1e-12 relative L-infinity per variable over the samples; FP32
<= 1e-5 relative L1 over the samples (smooth data).  Also in the bench's
launch configurations: C3 in place and with two steps per launch (the
paper's fixed dt) against the default mode, bit for bit, and the C4 batch
of 512 instances against oracle runs of four of them.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import workloads as wl
from tests.helpers import transpose_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fv():
    from paper_1701_05431_gb300 import fvlib
    return fvlib


def golden(name):
    return np.load(os.path.join(GOLDEN, f"{name}_oracle_samples.npz"))


def run_full(d, prim, steps, precision, tune=0):
    f = fv()
    with f.Solver(d, precision, stream=torch.cuda.current_stream().cuda_stream, tune=tune) as s:
        s.set_state(torch.from_numpy(prim).cuda(), primitive=True)
        t = s.run(steps)
        return s.state(), t, s


def sampled(W, idx):
    return W.reshape(W.shape[0], -1)[:, idx]


def test_c2_four_quadrant_2048_fp64():
    g = golden("c2")
    prim, d = wl.four_quadrant(2048, npart=8)
    W, t, _ = run_full(d, prim, int(g["steps"]), "f64")
    got = sampled(W, g["flat_index"])
    ref = g["W"]
    err = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert err.max() <= 1e-12, err
    assert abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
    # the four-quadrant problem is symmetric under x <-> y, u <-> v
    assert np.array_equal(transpose_state(W, "euler"), W)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_c3_smooth_8192(precision):
    g = golden("c3")
    prim, d = wl.smooth_periodic(8192)
    W, t, _ = run_full(d, prim, int(g["steps"]), precision)
    got = sampled(W, g["flat_index"])
    ref = g["W"]
    if precision == "f64":
        err = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
        assert err.max() <= 1e-12, err
        assert abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
    else:
        l1 = np.abs(got - ref).sum(axis=1) / np.abs(ref).sum(axis=1)
        assert l1.max() <= 1e-5, l1
        assert abs(t - float(g["t"])) <= 1e-5 * float(g["t"])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_c5_spray_2048(precision):
    g = golden("c5")
    prim, d = wl.spray_field(2048)
    W, t, _ = run_full(d, prim, int(g["steps"]), precision)
    got = sampled(W, g["flat_index"])
    ref = g["W"]
    if precision == "f64":
        err = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
        assert err.max() <= 1e-12, err
        assert abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
    else:
        l1 = np.abs(got - ref).sum(axis=1) / np.abs(ref).sum(axis=1)
        assert l1.max() <= 1e-5, l1


def test_c3_conservation_fp64_full():
    prim, d = wl.smooth_periodic(8192)
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(torch.from_numpy(prim).cuda(), primitive=True)
        t0 = s.totals()
        W = s.state()
        s.run(100)
        t1 = s.totals()
    mass = np.abs(W).sum(axis=(1, 2)) / 8192 ** 2
    assert np.all(np.abs(t1 - t0) / mass <= 1e-13), np.abs(t1 - t0) / mass


def test_c3_inplace_8192_fp32():
    """The in-place mode as the bench times it (the kernel table's in-place
    entry, one state buffer and overlap strips, 100 steps of 8192^2): the
    oracle samples within the FP32 bound, and the bits of the two-buffer run
    at every sampled cell."""
    g = golden("c3")
    prim, d = wl.smooth_periodic(8192)
    f = fv()
    idx = g["flat_index"]
    with f.Solver(d, "f32", stream=torch.cuda.current_stream().cuda_stream) as s:
        s.set_inplace(True)
        assert "inplace" in s.kernel_info()[1]
        s.set_state(torch.from_numpy(prim).cuda(), primitive=True)
        t_in = s.run(int(g["steps"]))
        got = sampled(s.state("float32"), idx)
    W2, t2, _ = run_full(d, prim, int(g["steps"]), "f32")
    assert np.array_equal(got, sampled(W2, idx).astype(np.float32)) and t_in == t2
    ref = g["W"]
    l1 = np.abs(got - ref).sum(axis=1) / np.abs(ref).sum(axis=1)
    assert l1.max() <= 1e-5, l1


def test_c3_two_steps_per_launch_8192_fp32_equals_one_step():
    """The paper's fixed dt on 8192^2 (dt = 0.4 h / lmax(W^0)), two steps per
    launch as the bench times it (the table's two-step kernel) against one
    step per launch: every cell bit for bit after 20 steps."""
    prim, d = wl.smooth_periodic(8192)
    rho, u, v, p = prim
    lam = float(np.max(np.maximum(np.abs(u), np.abs(v)) + np.sqrt(1.4 * p / rho)))
    d = dict(d, fixed_dt=0.4 * (1.0 / 8192) / lam)
    f = fv()
    outs = []
    for two in (False, True):
        with f.Solver(d, "f32", stream=torch.cuda.current_stream().cuda_stream) as s:
            if two:
                s.set_time_blocking(2)
            s.set_state(torch.from_numpy(prim).cuda(), primitive=True)
            t = s.run(20)
            out = torch.empty((4, 8192, 8192), dtype=torch.float32, device="cuda")
            s.get_state(out)
            outs.append((out, t))
    assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_c4_batched_512_against_oracle():
    """The 512-instance batch as the bench times it (FP32, one persistent
    launch for 200 steps) against the FP64 oracle on the three smallest
    instances and the largest, every cell; the FP64 batched kernel on the
    same instances within 1e-12."""
    import oracle
    from tests.helpers import oracle_problem
    f = fv()
    insts = wl.batched_quadrants(512)
    sizes = [d["nx"] * d["ny"] for _, _, d in insts]
    order = sorted(range(len(insts)), key=lambda k: sizes[k])
    pick = order[:3] + [order[-1]]
    with f.Batch([d for _, _, d in insts], "f32", stream=torch.cuda.current_stream().cuda_stream) as b:
        for i, (_, prim, _) in enumerate(insts):
            b.set_state(i, prim, primitive=True)
        b.run(200)
        got32 = [b.state(k) for k in pick]
    with f.Batch([insts[k][2] for k in pick], "f64") as b64:
        for q, k in enumerate(pick):
            b64.set_state(q, insts[k][1], primitive=True)
        b64.run(200)
        got64 = [b64.state(q) for q in range(len(pick))]
    for q, k in enumerate(pick):
        _, prim, d = insts[k]
        P = oracle_problem(d)
        r = oracle.run(P, oracle.prim_to_cons(P, prim), 200)
        assert r.status == oracle.OK
        ref = r.W.reshape(r.W.shape[0], -1)
        g32 = got32[q].reshape(ref.shape)
        g64 = got64[q].reshape(ref.shape)
        l1 = np.abs(g32 - ref).sum(axis=1) / np.abs(ref).sum(axis=1)
        assert l1.max() <= 1e-5, (k, l1)
        linf = np.abs(g64 - ref).max(axis=1) / np.abs(ref).max(axis=1)
        assert linf.max() <= 1e-12, (k, linf)
