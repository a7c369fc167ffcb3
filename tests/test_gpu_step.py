"""GPU parity of the fused step against the FP64 oracle, and the invariants
the method fixes, checked on the CUDA path through the C ABI.

Tolerances: FP64 <= 1e-12 relative L-infinity per variable (the oracle and
the kernel round differently only through FMA contraction and the order of
a few products, ~1e-16 per operation); FP32 storage and arithmetic <= 1e-5
relative L1 on smooth data (a few FP32 roundings per step, ~1e-7, growing
like the square root of the step count).
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
    from paper_1701_05431_gb300 import fvlib
    fvlib.load()
    oracle.build()


def fv():
    from paper_1701_05431_gb300 import fvlib
    return fvlib


def n_variants(system, precision):
    """Number of kernel candidates built for (system, precision)."""
    f = fv()
    k = 0
    prim, d = wl.random_smooth_euler(8, seed=0)
    if system == "advection":
        d = wl.problem("advection", 8, 8)
    while True:
        try:
            with f.Solver(d, precision, tune=2 + k):
                k += 1
        except f.FvError:
            return k


def gpu_run(d, prim, nsteps, precision="f64", tune=0, primitive=True, t_end=0.0):
    f = fv()
    with f.Solver(d, precision, stream=torch.cuda.current_stream().cuda_stream, tune=tune) as s:
        s.set_state(torch.from_numpy(np.ascontiguousarray(prim)).cuda(), primitive=primitive)
        t = s.run(nsteps, t_end=t_end)
        return s.state(), t, s.time()[1]


def oracle_run(d, prim, nsteps, mode="plain", t_end=0.0):
    P = oracle_problem(d)
    r = oracle.run(P, oracle.prim_to_cons(P, prim), nsteps, mode=mode, t_end=t_end)
    assert r.status == oracle.OK
    return r


# ------------------------------------------------------------------ parity
def test_c1_advection_128_parity():
    """Scalar advection, a = (1, 0.5), 128^2, CFL 0.5, 100 steps (full size)."""
    prim, d = wl.advection_bump(128)
    ref = oracle_run(d, prim, 100)
    out, t, steps = gpu_run(d, prim, 100)
    assert steps == 100 and t == ref.t
    assert rel_linf(out, ref.W).max() <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "transmissive", "dirichlet", "mixed"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_euler_parity_ragged(bc, precision):
    """Several tiles in x and y with ragged tails (193 x 141)."""
    prim, d = wl.random_smooth_euler(193, seed=23, ny=141)
    if bc == "mixed":
        d = dict(d, bc=("transmissive", "periodic", "dirichlet", "periodic"),
                 bc_state=((0,) * 4, (0,) * 4, (1.05, 0.1, -0.05, 2.6), (0,) * 4))
    else:
        d = dict(d, bc=(bc,) * 4, bc_state=((1.05, 0.1, -0.05, 2.6),) * 4)
    ref = oracle_run(d, prim, 60)
    out, t, _ = gpu_run(d, prim, 60, precision)
    if precision == "f64":
        assert rel_linf(out, ref.W).max() <= 1e-12
        assert abs(t - ref.t) <= 1e-13 * ref.t
    else:
        assert rel_l1(out, ref.W).max() <= 1e-5
        assert abs(t - ref.t) <= 1e-5 * ref.t


def test_bf16_storage_error_bound():
    """bfloat16 storage, FP32 arithmetic: every stored value is rounded to
    8 significant bits (unit roundoff u = 2^-9 = 2.0e-3) after every step,
    while one step changes a cell by only ~CFL x (its relative variation over
    a cell) ~ 0.4%.  The roundings accumulate like a random walk, ~sqrt(N) u
    relative to |W| after N steps (1.5% for N = 60), more on the momenta whose
    L1 mass is small compared with their magnitude.  Bound: 5% relative L1
    per variable after 60 steps (measured 1.6% / 3.4% / 2.5% / 1.2%).

    The conserved totals are not conserved exactly: the FP32 update is
    conservative to ~1e-7, but each stored value is then rounded by up to
    u |W|, so after N steps the totals can move by at most N u sum|W| dx dy
    (all roundings of one sign).  Updates smaller than half an ulp round away
    in the same direction step after step, so the drift sits well above a
    random walk (measured 1.9e-3 of the energy mass after 60 steps); the test
    checks the worst-case bound N u."""
    prim, d = wl.random_smooth_euler(193, seed=23, ny=141)
    N = 60
    ref = oracle_run(d, prim, N)
    out, t, _ = gpu_run(d, prim, N, "bf16")
    l1 = rel_l1(out, ref.W)
    print("bf16 rel L1 per variable", l1, "rel Linf", rel_linf(out, ref.W))
    assert l1.max() <= 5e-2, l1
    assert abs(t - ref.t) <= 1e-2 * ref.t
    P = oracle_problem(d)
    t0 = oracle.totals(P, oracle.prim_to_cons(P, prim))
    t1 = oracle.totals(P, out)
    mass = np.abs(ref.W).sum(axis=(1, 2)) * P.dx * P.dy
    drift = np.abs(t1 - t0) / mass
    print("bf16 totals drift / mass", drift)
    assert np.all(drift <= N * 2.0 ** -9), drift


def test_bf16_one_step_is_the_rounded_oracle_step():
    """One bfloat16 step from a state whose values are bfloat16 numbers is the
    FP64 oracle step rounded to bfloat16: the FP32 arithmetic errs by ~1e-6
    relative, far below the bfloat16 spacing 2^-8 relative, so the rounded
    results agree except where the exact value lies within that error of a
    rounding boundary (expected fraction ~1e-3 or less), and there they differ
    by one bfloat16 spacing."""
    prim, d = wl.random_smooth_euler(193, seed=31, ny=141)
    P = oracle_problem(d)
    W0 = to_bf16(oracle.prim_to_cons(P, prim))
    r = oracle.run(P, W0, 1, mode="plain")
    assert r.status == oracle.OK
    out, t, _ = gpu_run(d, W0, 1, "bf16", primitive=False)
    want = to_bf16(r.W)
    assert abs(t - r.t) <= 1e-6 * r.t
    spacing = 2.0 ** (np.floor(np.log2(np.maximum(np.abs(r.W), 1e-30))) - 7)
    off = out != want
    print("bf16 one step: values off the rounded oracle", off.mean())
    assert np.all(np.abs(out - r.W) <= spacing)
    assert off.mean() <= 1e-2


def test_four_quadrant_512_parity_and_symmetry():
    """The four-quadrant Riemann problem (transmissive, 8 x 8 subdomains) at
    512^2 for 500 steps; the exact solution is transpose symmetric and so is
    the GPU result, bit for bit."""
    prim, d = wl.four_quadrant(512, npart=8)
    ref = oracle_run(d, prim, 500)
    out, t, _ = gpu_run(d, prim, 500)
    assert rel_linf(out, ref.W).max() <= 1e-12
    assert np.array_equal(transpose_state(out, "euler"), out)


def to_bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("bcs", ["transmissive-periodic", "dirichlet-mix"])
@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
def test_every_kernel_variant_gives_the_same_bits(precision, bcs):
    """Tile shape, cells per lane, warps per block and row staging change only
    the work decomposition: every candidate returns identical bits (with
    Dirichlet sides whose states bfloat16 cannot hold exactly, ghost rows and
    ghost columns take the same stored value)."""
    prim, d = wl.random_smooth_euler(157, seed=31, ny=97)
    if bcs == "transmissive-periodic":
        d = dict(d, bc=("transmissive", "periodic", "transmissive", "periodic"))
    else:
        far = (1.0137, 0.1013 * 1.0137, -0.0521 * 1.0137, 2.5173)
        d = dict(d, bc=("dirichlet", "dirichlet", "transmissive", "dirichlet"), bc_state=(far,) * 4)
    outs = [gpu_run(d, prim, 25, precision, tune=2 + k)[0] for k in range(n_variants("euler", precision))]
    assert len(outs) >= 2
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (2, 3), (31, 5), (61, 2), (121, 67)])
def test_degenerate_and_odd_grids(shape):
    nx, ny = shape
    prim, d = wl.random_smooth_euler(nx, seed=3, ny=ny)
    d = dict(d, bc=("transmissive", "periodic", "transmissive", "periodic"))
    ref = oracle_run(d, prim, 9)
    for precision in ("f64", "f32", "bf16"):
        for k in range(n_variants("euler", precision)):
            out, _, _ = gpu_run(d, prim, 9, precision, tune=2 + k)
            if precision == "f64":
                assert rel_linf(out, ref.W).max() <= 1e-12, (shape, k)
            elif precision == "f32":
                assert rel_linf(out, ref.W).max() <= 1e-5, (shape, k)
            else:
                assert rel_linf(out, ref.W).max() <= 5e-2, (shape, k)


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("bc", ["periodic", "transmissive", "dirichlet"])
def test_constant_state_bitwise(precision, bc):
    const = np.array([1.3, 0.4 * 1.3, -0.25 * 1.3, 2.5])
    if precision == "f32":
        const = const.astype(np.float32).astype(np.float64)
    if precision == "bf16":
        const = to_bf16(const)
    W0 = np.empty((4, 37, 45))
    for v in range(4):
        W0[v] = const[v]
    d = wl.problem("euler", 45, 37, bc=(bc,) * 4, bc_state=(tuple(const),) * 4)
    out, _, _ = gpu_run(d, W0, 13, precision, primitive=False)
    assert np.array_equal(out, W0)


def rows_per_task(info: str) -> int:
    """Rows per warp task of a kernel description: the balanced count when
    the host reports one (", N-row tasks"), else the candidate's TY."""
    import re
    m = re.search(r", (\d+)-row tasks", info)
    return int(m.group(1)) if m else int(re.search(r" ty(\d+)", info).group(1))


def test_default_kernel_fills_the_gpu_on_small_grids():
    """Without tuning, a large grid gets the first candidate; a grid whose
    warp tasks cannot fill the GPU with it gets shorter tasks: another
    candidate, its rows per task balanced over the GPU where the host does
    that."""
    f = fv()
    for precision in ("f32", "f64", "bf16"):
        first = f.kernel_candidates("euler", precision)[0]
        big = wl.problem("euler", 8192, 8192)
        small = wl.problem("euler", 256, 256)
        with f.Solver(big, precision) as s:
            # FP64 kernels may report rows per task balanced over the GPU
            assert s.kernel_info()[1].split(",")[0] == first
        with f.Solver(small, precision) as s:
            info = s.kernel_info()[1]
        got = info.split(",")[0]
        assert got != first and rows_per_task(info) < rows_per_task(first), (precision, info)


def test_periodic_conservation_fp64_and_fp32_drift():
    prim, d = wl.random_smooth_euler(256, seed=41, ny=192)
    f = fv()
    for precision, bound in (("f64", 1e-13), ("f32", 2e-6)):
        with f.Solver(d, precision) as s:
            s.set_state(prim, primitive=True)
            t0 = s.totals()
            s.run(200)
            t1 = s.totals()
            W = s.state()
        mass = np.abs(W).sum(axis=(1, 2)) * (1 / 256) * (1 / 192)
        drift = np.abs(t1 - t0) / mass
        assert np.all(drift <= bound), (precision, drift)


def test_totals_match_compensated_sum():
    prim, d = wl.random_smooth_euler(300, seed=5, ny=211)
    P = oracle_problem(d)
    W = oracle.prim_to_cons(P, prim)
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(W)
        tot = s.totals()
    ref = oracle.totals(P, W)
    assert np.all(np.abs(tot - ref) <= 1e-15 * np.abs(W).sum(axis=(1, 2)) * P.dx * P.dy)


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
def test_transposition_bitwise(precision):
    prim, d = wl.random_smooth_euler(83, seed=7, ny=54)
    d = dict(d, bc=("transmissive", "periodic", "transmissive", "periodic"))
    P = oracle_problem(d)
    W0 = oracle.prim_to_cons(P, prim)
    if precision == "f32":
        W0 = W0.astype(np.float32).astype(np.float64)
    if precision == "bf16":
        W0 = to_bf16(W0)
    out, _, _ = gpu_run(d, W0, 30, precision, primitive=False)
    dt_ = dict(d, nx=54, ny=83, bc=("periodic", "transmissive", "periodic", "transmissive"))
    outt, _, _ = gpu_run(dt_, transpose_state(W0, "euler"), 30, precision, primitive=False)
    assert np.array_equal(transpose_state(outt, "euler"), out)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_exact_shift_cfl1_bitwise(axis):
    n = 96
    x = wl.centres(n)
    u = 1.0 + 0.9 * np.exp(-((x[None, :] - 0.4) ** 2 + (x[:, None] - 0.55) ** 2) / 0.02)
    W0 = (np.round(u * 2.0 ** 40) / 2.0 ** 40)[None]
    a = (1.0, 0.0) if axis == "x" else (0.0, 1.0)
    d = wl.problem("advection", n, n, cfl=1.0, params=a)
    out, _, _ = gpu_run(d, W0, 37, primitive=False)
    assert np.array_equal(out, np.roll(W0, 37, axis=2 if axis == "x" else 1))


def test_partition_does_not_change_results():
    prim, d = wl.random_smooth_euler(120, seed=9, ny=90)
    a = gpu_run(dict(d, npart_x=1, npart_y=1), prim, 20)[0]
    b = gpu_run(dict(d, npart_x=7, npart_y=5), prim, 20)[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_resume_bitwise(precision):
    """run(2N) == run(N) -> get_state -> set_state -> set_time -> run(N)."""
    prim, d = wl.random_smooth_euler(100, seed=12, ny=77)
    f = fv()
    with f.Solver(d, precision) as s:
        s.set_state(prim, primitive=True)
        s.run(30)
        full = s.state("float64" if precision == "f64" else "float32")
        tfull = s.time()
    with f.Solver(d, precision) as s:
        s.set_state(prim, primitive=True)
        s.run(15)
        half = s.state("float64" if precision == "f64" else "float32")
        t, n = s.time()
    with f.Solver(d, precision) as s:
        s.set_state(half)
        s.set_time(t, n)
        s.run(15)
        again = s.state("float64" if precision == "f64" else "float32")
        assert s.time() == tfull
    assert np.array_equal(again, full)


def test_step_by_step_equals_run():
    prim, d = wl.random_smooth_euler(64, seed=2, ny=48)
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(prim, primitive=True)
        dts = [s.step() for _ in range(10)]
        a = s.state()
    ref = oracle_run(d, prim, 10)
    np.testing.assert_allclose(dts, ref.dts, rtol=1e-13)
    b = gpu_run(d, prim, 10)[0]
    assert np.array_equal(a, b)


def test_sod_rows_identical_and_parity():
    prim, d = wl.sod_x(400, ny=6)
    ref = oracle_run(d, prim, 10000, t_end=0.2)
    out, t, _ = gpu_run(d, prim, 10000, t_end=0.2)
    assert abs(t - 0.2) < 1e-14
    for j in range(1, 6):
        assert np.array_equal(out[:, j], out[:, 0])
    assert rel_linf(out, ref.W).max() <= 1e-12


# ------------------------------------------------------------------ errors
def test_fixed_dt_cfl_violation_keeps_state():
    prim, d = wl.random_smooth_euler(40, seed=4)
    P = oracle_problem(d)
    lmax = oracle.lambda_max(P, oracle.prim_to_cons(P, prim))
    f = fv()
    good = dict(d, fixed_dt=0.9 * P.dx / lmax)
    with f.Solver(good, "f64") as s:
        s.set_state(prim, primitive=True)
        assert abs(s.lambda_max() - lmax) <= 1e-14 * lmax
        s.run(1)
    bad = dict(d, fixed_dt=1.1 * P.dx / lmax)
    with f.Solver(bad, "f64") as s:
        s.set_state(prim, primitive=True)
        W0 = s.state()
        st, _ = s.run(3, check=False)
        assert st == f.FV_ERR_CFL
        assert s.time() == (0.0, 0)
        assert np.array_equal(s.state(), W0)


def test_nonphysical_state_rejected():
    prim, d = wl.random_smooth_euler(32, seed=4)
    prim[3, 10, 11] = -0.5  # negative pressure
    f = fv()
    with f.Solver(d, "f64") as s:
        st = s.set_state(prim, primitive=True, check=False)
        assert st == f.FV_ERR_NONPHYSICAL
        st, _ = s.run(1, check=False)
        assert st == f.FV_ERR_STATE


def test_zero_wave_speed_rejected():
    d = wl.problem("advection", 16, 16, params=(0.0, 0.0))
    f = fv()
    with f.Solver(d, "f64") as s:
        s.set_state(np.ones((1, 16, 16)))
        st, _ = s.run(1, check=False)
        assert st == f.FV_ERR_INVALID_ARG


def test_t_end_clips_last_step():
    prim, d = wl.random_smooth_euler(48, seed=6)
    ref = oracle_run(d, prim, 1000, t_end=0.013)
    out, t, steps = gpu_run(d, prim, 1000, t_end=0.013)
    assert steps == ref.steps and abs(t - 0.013) <= 1e-15
    assert rel_linf(out, ref.W).max() <= 1e-12


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0, 1.1])
def test_primitive_load_is_the_fp64_definition_bit_for_bit(gamma):
    """rho E = p/(gamma - 1) + rho (u u + v v)/2 per cell, each operation
    rounded once in FP64 (numpy's float64 arithmetic): the load divides by
    gamma - 1 through a correction of the product with its reciprocal, which
    must give the quotient itself."""
    rng = np.random.default_rng(91)
    ny, nx = 211, 173
    prim = np.empty((4, ny, nx))
    # wide magnitudes, kept admissible: p stays far above the rounding of
    # rho E - rho (u u + v v)/2, so the load's check accepts every cell
    prim[0] = rng.lognormal(0.0, 1.5, (ny, nx))
    prim[1] = rng.normal(0.0, 1.0, (ny, nx))
    prim[2] = rng.normal(0.0, 1.0, (ny, nx))
    prim[3] = rng.lognormal(1.0, 1.0, (ny, nx)) + 0.1
    d = wl.problem("euler", nx, ny, params=(gamma,))
    rho, u, v, p = prim
    q = u * u + v * v
    want = np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + (rho * q) * 0.5])
    with fv().Solver(d, "f64") as s:
        s.set_state(np.ascontiguousarray(prim), primitive=True)
        got = s.state()
    assert np.array_equal(got, want)
    # FP32 input and storage: the FP64 value rounded once to FP32
    p32 = prim.astype(np.float32)
    rho, u, v, p = (x.astype(np.float64) for x in p32)
    want32 = np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + (rho * (u * u + v * v)) * 0.5]).astype(np.float32)
    with fv().Solver(d, "f32") as s:
        s.set_state(np.ascontiguousarray(p32), primitive=True)
        got32 = s.state("float32")
    assert np.array_equal(got32, want32)
