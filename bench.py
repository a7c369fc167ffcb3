"""Benchmark of the fused finite-volume step on one GB300 (or N replicas).

Workload (default): 2D Euler, gamma = 1.4, 8192 x 8192 cells, periodic,
seeded smooth sinusoidal data, CFL 0.4; one bench step = one job of 100
time steps advanced by fv_run from a state resident in HBM.  The headline
`value` is FP32-bulk cell-updates/s; the FP64-plain figure of the same job is
reported beside it under "fp64".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c3|c2|c1|c4|c5] [--no-cpu-baseline] [--no-e2e]

Under torchrun (N > 1) every rank runs an independent replica (the grid is
not sharded across GPUs): value = all ranks' cell-updates / max rank time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the oracle is the only reference there is).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0   # NVIDIA's HBM3e figure for GB300, for context beside the measured copy rate


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


WORKLOADS = {
    # name: (builder, steps per job, description)
    "c3": (lambda: wl.smooth_periodic(8192), 100,
           "euler 8192x8192 periodic smooth sinusoids, CFL 0.4, 100 steps"),
    "c3s": (lambda: wl.smooth_periodic(4096), 100,
            "euler 4096x4096 periodic smooth sinusoids, CFL 0.4, 100 steps (profiling size)"),
    "c2": (lambda: wl.four_quadrant(2048, npart=8), 500,
           "euler 2048x2048 four-quadrant Riemann, 8x8 subdomains, transmissive, CFL 0.4, 500 steps"),
    "c1": (lambda: wl.advection_bump(128), 100,
           "advection 128x128 a=(1,0.5) periodic, CFL 0.5, 100 steps"),
}

# the bench's metric, the same string on both arms
METRIC = "cell-updates/s (FP32-bulk; FP64 plain beside it) and HBM GB/s"

BYTES_PER_CELL = {"advection": 1, "euler": 4, "spray": 6}  # nvar
# names of the per-configuration entries of accuracy_vs_oracle
WORKLOAD_KEYS = {"c3": "c3_euler_8192", "c2": "c2_four_quadrant_2048", "c1": "c1_advection_128",
                 "c3s": "c3_euler_4096"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        # the raw samples go to FV_CLOCKS_DIR (default: the system's temporary directory)
        d = os.environ.get("FV_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"fv_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def measured_traffic_per_cell(kernel_desc: str):
    """DRAM bytes per cell-update of a kernel, from the ncu capture recorded
    next to the profile summaries (None when that kernel was not captured)."""
    try:
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if line.startswith("#") or "|" not in line:
                    continue
                desc, val = (x.strip() for x in line.split("|", 1))
                if desc == kernel_desc:
                    return float(val)
    except OSError:
        pass
    return None


FP64_OPS_FILE = os.path.join(ROOT, "profiles", "fp64_ops.txt")


def measured_fp64_ops_per_cell(kernel_desc: str):
    """FP64 work per cell-update of a kernel from the ncu capture recorded next
    to the profile summaries: {"dfma", "dmul", "dadd", "pipe"} thread-level
    instructions per cell-update (pipe: every instruction the FP64 pipe
    executed), or None when that kernel was not captured."""
    try:
        with open(FP64_OPS_FILE) as f:
            for line in f:
                if line.startswith("#") or "|" not in line:
                    continue
                parts = [x.strip() for x in line.split("|")]
                if parts[0] == kernel_desc and len(parts) >= 5:
                    return dict(zip(("dfma", "dmul", "dadd", "pipe"), map(float, parts[1:5])))
    except (OSError, ValueError):
        pass
    return None


def fp64_roofline(kernel_desc: str, cell_updates_per_s: float, dfma_peak: float):
    """Arithmetic roofline of an FP64-pipe-bound kernel: FP64 FLOP/s retired
    (2 per DFMA, 1 per DMUL or DADD, counted per cell-update by ncu) against
    twice the measured DFMA rate, and the FP64 pipe's instruction rate against
    the measured DFMA rate (every FP64-pipe instruction takes the pipe as long
    as a DFMA)."""
    # the rows per warp task (", N-row tasks") change the halo share by a few
    # per cent only; the capture is keyed by the kernel itself
    ops = measured_fp64_ops_per_cell(kernel_desc.split(", ")[0])
    out = {"bound": "alu", "unit": "TFLOP/s", "peak": 2 * dfma_peak / 1e12,
           "peak_source": "measured: fv_fma_peak (DFMA chains on every SM, CUDA events) x 2 FLOP",
           "peak_nominal": 1.25, "ops_per_cell_update": ops}
    if ops is None or not dfma_peak:
        out.update(achieved=None, frac=None, pipe_frac=None)
        return out
    flops = (2 * ops["dfma"] + ops["dmul"] + ops["dadd"]) * cell_updates_per_s
    out.update(achieved=flops / 1e12, frac=flops / (2 * dfma_peak), frac_nominal=flops / 1.25e12,
               pipe_frac=ops["pipe"] * cell_updates_per_s / dfma_peak,
               ops_source="ncu sm__sass_thread_inst_executed_op_{dfma,dmul,dadd}_pred_on.sum and "
                          "sm__thread_inst_executed_pipe_fp64_pred_on.sum of one launch (profiles/fp64_ops.txt)")
    return out


def max_over_ranks(value: float, device: str = "cpu") -> float:
    """Largest value over all ranks (the slowest rank's time); identity on one
    process.  device: where the reduction tensor lives ("cuda:k" for NCCL,
    "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(cells: int, steps_per_job: int, jobs: int, world_size: int, max_ms: float) -> float:
    """Cell-updates/s of the whole job: every rank advances its own replica of
    `cells` cells by jobs * steps_per_job steps, timed by the slowest rank."""
    return cells * steps_per_job * jobs * world_size / (max_ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_model() -> str:
    """The host CPU as lscpu names it (model name and core count)."""
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        info = dict(l.split(":", 1) for l in txt.splitlines() if ":" in l)
        name = (info.get("Model name") or info.get("Vendor ID") or "").strip()
        return f"{name}, {os.cpu_count()} logical CPUs".strip(", ")
    except Exception:
        return f"{os.cpu_count()} logical CPUs"


def cpu_baseline_run(name, d, prim, sample_steps=None, seconds_target=15.0):
    """Time the FP64 oracle, as it stands, on the host cores on a bounded
    sample of the workload (a few steps on the full grid)."""
    import oracle
    from tests.helpers import oracle_problem
    oracle.build()
    P = oracle_problem(d)
    W0 = oracle.prim_to_cons(P, prim)
    threads = oracle.max_threads()
    ncell = d["nx"] * d["ny"]
    # one probe step to size the sample
    t = time.perf_counter()
    r = oracle.run(P, W0, 1)
    one = time.perf_counter() - t
    steps = sample_steps or max(1, min(50, int(seconds_target / max(one, 1e-6))))
    t = time.perf_counter()
    r = oracle.run(P, r.W, steps)
    el = time.perf_counter() - t
    out = {"value": ncell * steps / el, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
           "cpu": cpu_model(),
           "sample": f"{name}: full {d['nx']}x{d['ny']} grid, {steps} FP64 steps (plain mode) after one "
                     f"warm-up step, {el:.1f} s"}
    # the same oracle on one thread, one step of a 4096^2 grid of the same data recipe
    if ncell > 4096 * 4096:
        prim1, d1 = wl.smooth_periodic(4096)
        P1 = oracle_problem(d1)
        W1 = oracle.prim_to_cons(P1, prim1)
        t = time.perf_counter()
        oracle.run(P1, W1, 1, nthreads=1)
        el1 = time.perf_counter() - t
        out["single_thread"] = {"value": 4096 * 4096 / el1, "unit": "cell-updates/s", "cores": 1,
                                "sample": f"one FP64 step of a 4096x4096 grid of the same recipe, {el1:.1f} s"}
    return out


def oracle_sample(d, prim, steps, what):
    """Oracle cell-updates/s on the host cores for `steps` steps of one
    configuration (input prepared outside the timed region)."""
    import oracle
    from tests.helpers import oracle_problem
    oracle.build()
    P = oracle_problem(d)
    W = oracle.prim_to_cons(P, prim)
    t = time.perf_counter()
    r = oracle.run(P, W, steps)
    el = time.perf_counter() - t
    return {"value": d["nx"] * d["ny"] * steps / el, "unit": "cell-updates/s", "cores": oracle.max_threads(),
            "status": int(r.status), "sample": f"{what}: {steps} FP64 steps of {d['nx']}x{d['ny']}, {el:.2f} s"}


def job_config(desc, ncell, nsteps_job, ws):
    """The workload both arms report (the kernel that ran is a key of its own)."""
    f32_bytes = 4 * 4 * ncell  # one FP32 Euler state buffer
    l2 = (f"inputs larger than L2 (state buffers {f32_bytes / 2**30:.3g} GiB f32 / {2 * f32_bytes / 2**30:.3g} GiB f64)"
          if f32_bytes > 129e6 else "state within L2 (a small workload: no flush between steps)")
    return {"workload": desc, "cells": ncell, "time_steps_per_bench_step": nsteps_job, "l2": l2,
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    build, nsteps_job, desc = WORKLOADS[args.workload]
    prim, d = build()
    import oracle
    from tests.helpers import oracle_problem
    oracle.build()
    P = oracle_problem(d)
    W = oracle.prim_to_cons(P, prim)
    ncell = d["nx"] * d["ny"]
    # each step: a bounded sample of the job (a few FV steps of the full grid)
    t = time.perf_counter()
    oracle.run(P, W, 1)
    one = time.perf_counter() - t
    per = max(1, int(8.0 / max(one, 1e-6)))
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle.run(P, W, 1)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        r = oracle.run(P, W, per)
        times.append(time.perf_counter() - t)
        W = r.W
    el = sum(times)
    value = ncell * per * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": job_config(desc, ncell, nsteps_job, ws),
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": oracle.max_threads(), "cpu": cpu_model(),
                             "kind": "oracle",
                             "sample": f"{per} FV steps of the full {d['nx']}x{d['ny']} grid per bench step"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def errors_vs(got, ref):
    """Per-variable relative L1 (sum|a-b| / sum|b|) and relative L-infinity
    (max|a-b| / max|b|) of `got` against the oracle's `ref` (nvar x cells)."""
    got = np.asarray(got, dtype=np.float64).reshape(ref.shape[0], -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(ref.shape[0], -1)
    l1 = (np.abs(got - ref).sum(axis=1) / np.abs(ref).sum(axis=1)).tolist()
    linf = (np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).tolist()
    return {"rel_l1": l1, "rel_linf": linf}


def c4_accuracy(fvlib, b, insts, pick, sptr):
    """FP32 batched states of the picked instances after 200 steps against the
    FP64 oracle run of each instance (and the FP64 batched kernel on the same
    instances)."""
    import oracle
    from tests.helpers import oracle_problem
    oracle.build()
    res = {"instances": [], "steps": 200,
           "against": "oracle.run of each instance, 200 FP64 steps, every cell"}
    refs = []
    for k in pick:
        _, pr, dd = insts[k]
        P = oracle_problem(dd)
        r = oracle.run(P, oracle.prim_to_cons(P, pr), 200)
        refs.append(r.W)
        e = errors_vs(b.state(k), r.W)
        res["instances"].append({"index": k, "nx": dd["nx"], "ny": dd["ny"], "oracle_status": int(r.status),
                                 "f32": e})
    with fvlib.Batch([insts[k][2] for k in pick], "f64", stream=sptr) as b64:
        for q, k in enumerate(pick):
            b64.set_state(q, insts[k][1], primitive=True)
        b64.run(200)
        for q in range(len(pick)):
            res["instances"][q]["f64"] = errors_vs(b64.state(q), refs[q])
    for prec in ("f32", "f64"):
        res[prec] = {"rel_l1": np.max([x[prec]["rel_l1"] for x in res["instances"]], axis=0).tolist(),
                     "rel_linf": np.max([x[prec]["rel_linf"] for x in res["instances"]], axis=0).tolist()}
    return res


def golden_samples(name):
    path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle_samples.npz")
    return np.load(path) if os.path.exists(path) else None


def secondary_workloads(fvlib, torch, sptr, local, hbm, oracle_too=False, accuracy=None, dfma_peak=None):
    """The other configurations of the hot path, one or two timed jobs each
    (device-resident inputs, CUDA events around the run calls)."""
    out = {}
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()  # warm-up (also builds the graph)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    # C1: scalar advection 128^2, FP64, 100 steps (latency-bound: 16 K cells)
    prim, d = wl.advection_bump(128)
    with fvlib.Solver(d, "f64", stream=sptr) as s:
        s.set_state(torch.from_numpy(prim).to(f"cuda:{local}"), primitive=True)
        sec = timed(lambda: s.run(100), 5)
        out["c1_advection_128_f64"] = {"cell_updates_per_s": 128 * 128 * 100 / sec, "ms_per_job": sec * 1e3,
                                       "kernel": s.kernel_info()[1], "kernel_choice": s.kernel_choice()}
        if accuracy is not None:
            import oracle
            from tests.helpers import oracle_problem
            oracle.build()
            P = oracle_problem(d)
            ref = oracle.run(P, oracle.prim_to_cons(P, prim), 100)
            s.set_state(torch.from_numpy(prim).to(f"cuda:{local}"), primitive=True)
            s.run(100)
            accuracy["c1_advection_128"] = {"f64": errors_vs(s.state(), ref.W), "samples": 128 * 128,
                                            "steps": 100, "against": "oracle.run of the whole job, every cell"}
    if oracle_too:
        out["c1_advection_128_f64"]["oracle"] = oracle_sample(d, prim, 100, "the whole job")
    # C2: four-quadrant Euler 2048^2, 8x8 subdomains, FP64, 500 steps (and FP32)
    prim, d = wl.four_quadrant(2048, npart=8)
    pd = torch.from_numpy(prim).to(f"cuda:{local}")
    g2 = golden_samples("c2")
    acc2 = {}
    for precision in ("f64", "f32"):
        with fvlib.Solver(d, precision, stream=sptr) as s:
            def job():
                s.set_state(pd, primitive=True)
                s.run(500)
            sec = timed(job, 1)
            if g2 is not None and accuracy is not None:
                # the state after the last timed job is the 500-step result
                acc2[precision] = errors_vs(s.state().reshape(4, -1)[:, g2["flat_index"]], g2["W"])
            nb = 2 * 4 * (8 if precision == "f64" else 4) * 2048 * 2048 * 500
            out[f"c2_four_quadrant_2048_{precision}"] = {
                "cell_updates_per_s": 2048 * 2048 * 500 / sec, "ms_per_job": sec * 1e3,
                "hbm_gbs_algorithmic": nb / sec / 1e9, "kernel": s.kernel_info()[1],
                "kernel_choice": s.kernel_choice(),
                "note": "job = set_state from device + 500 steps; 134 MB/268 MB state, close to L2 size"}
    # the same grid in the paper's fixed-dt mode, dt = 0.4 min(dx, dy) / lmax(W^0):
    # one step per launch, and two steps per launch (transmissive ghosts of the
    # intermediate state inside the pass)
    lam0 = float(np.max(np.maximum(np.abs(prim[1]), np.abs(prim[2])) + np.sqrt(1.4 * prim[3] / prim[0])))
    dfix2 = dict(d, fixed_dt=0.4 * min(1.0 / d["nx"], 1.0 / d["ny"]) / lam0)
    for passes in (1, 2):
        with fvlib.Solver(dfix2, "f32", stream=sptr) as s:
            if passes == 2:
                s.set_time_blocking(2)

            def job():
                s.set_state(pd, primitive=True)
                s.run(500)
            sec = timed(job, 1)
            name = "two_steps_per_launch" if passes == 2 else "per_step_launches"
            out[f"c2_fixed_dt_{name}_f32"] = {
                "cell_updates_per_s": 2048 * 2048 * 500 / sec, "ms_per_job": sec * 1e3,
                "kernel": s.two_step_kernel() if passes == 2 else s.kernel_info()[1],
                "kernel_choice": s.kernel_choice(two_step=(passes == 2)),
                "note": "four-quadrant 2048^2, transmissive, fixed dt; job = set_state from device + 500 steps"}
    if acc2:
        accuracy["c2_four_quadrant_2048"] = dict(acc2, samples=int(len(g2["flat_index"])), steps=500,
                                                 against="stored oracle samples (tests/golden/c2_oracle_samples.npz)")
    if oracle_too:
        out["c2_four_quadrant_2048_f64"]["oracle"] = oracle_sample(d, prim, 5, "a sample")
    del pd
    # C4: 512 batched four-quadrant instances, FP32, 200 steps in one persistent launch
    insts = wl.batched_quadrants(512)
    ncells = sum(dd["nx"] * dd["ny"] for _, _, dd in insts)
    c4_oracle = None
    if oracle_too:
        # eight of the instances, 20 steps each
        vals, cells, secs = [], 0, 0.0
        for _, pr, dd in insts[:8]:
            o = oracle_sample(dd, pr, 20, "instance")
            cells += dd["nx"] * dd["ny"] * 20
            secs += dd["nx"] * dd["ny"] * 20 / o["value"]
        c4_oracle = {"value": cells / secs, "unit": "cell-updates/s", "cores": o["cores"],
                     "sample": f"the first 8 of the 512 instances, 20 FP64 steps each, {secs:.2f} s"}
    with fvlib.Batch([dd for _, _, dd in insts], "f32", stream=sptr) as b:
        for k, (_, pr, _) in enumerate(insts):
            b.set_state(k, pr, primitive=True)
        sec = timed(lambda: b.run(200), 2)
        if accuracy is not None:
            # outside the timed region: every instance restarted and advanced
            # 200 steps by the same batched launch, then the three smallest
            # instances and the largest compared with the oracle
            for k, (_, pr, _) in enumerate(insts):
                b.set_state(k, pr, primitive=True)
            b.run(200)
            sizes = [dd["nx"] * dd["ny"] for _, _, dd in insts]
            order = sorted(range(len(insts)), key=lambda k: sizes[k])
            pick = order[:3] + order[-1:]
            accuracy["c4_batched_512"] = c4_accuracy(fvlib, b, insts, pick, sptr)
        del insts
        nb = 2 * 4 * 4 * ncells * 200
        out["c4_batched_512_f32"] = {"cell_updates_per_s": ncells * 200 / sec, "ms_per_job": sec * 1e3,
                                     "cells": ncells, "hbm_gbs_algorithmic": nb / sec / 1e9,
                                     "hbm_frac": nb / sec / 1e9 / hbm, "kernel": b.kernel_info()[1],
                                     "kernel_choice": b.kernel_choice(),
                                     "launches_per_job": 1}
        if c4_oracle:
            out["c4_batched_512_f32"]["oracle"] = c4_oracle
    # The paper's fixed dt (per instance: 0.4 min(dx, dy) / lmax(W^0)) on the
    # same 512 instances, step-gated and with device dataflow (neighbour
    # dependencies, no barrier per step); and one 8192^2 grid as a batch of one
    # against the per-step launches of fv_run.
    def lmax0(prim, gamma=1.4):
        rho, u, v, p = prim
        return float(np.max(np.maximum(np.abs(u), np.abs(v)) + np.sqrt(gamma * p / rho)))

    def fixed(prim, dd):
        return dict(dd, fixed_dt=0.4 * min(1.0 / dd["nx"], 1.0 / dd["ny"]) / lmax0(prim))

    insts = wl.batched_quadrants(512)
    cfgs = [fixed(pr, dd) for _, pr, dd in insts]
    for mode in ("gated", "dataflow"):
        with fvlib.Batch(cfgs, "f32", stream=sptr) as b:
            for k, (_, pr, _) in enumerate(insts):
                b.set_state(k, pr, primitive=True)
            b.set_dataflow(mode == "dataflow")
            sec = timed(lambda: b.run(200), 1)
            out[f"c4_fixed_dt_{mode}_f32"] = {
                "cell_updates_per_s": ncells * 200 / sec, "ms_per_job": sec * 1e3,
                "hbm_frac": 2 * 4 * 4 * ncells * 200 / sec / 1e9 / hbm, "kernel": b.kernel_info()[1],
                "kernel_choice": b.kernel_choice()}
    del insts, cfgs
    prim, d = wl.smooth_periodic(8192, dtype=np.float32)
    dfix = fixed(prim, d)
    pd = torch.from_numpy(prim).to(f"cuda:{local}")
    with fvlib.Solver(dfix, "f32", stream=sptr) as s:
        def job():
            s.set_state(pd, primitive=True)
            s.run(100)
        sec = timed(job, 1)
        out["c3_fixed_dt_per_step_launches_f32"] = {"cell_updates_per_s": 8192 * 8192 * 100 / sec,
                                                    "ms_per_job": sec * 1e3, "kernel": s.kernel_info()[1],
                                                    "note": "job = set_state from device + 100 steps"}
    for precision in ("f32", "bf16"):
        with fvlib.Solver(dfix, precision, stream=sptr) as s:
            s.set_time_blocking(2)

            def job():
                s.set_state(pd, primitive=True)
                s.run(100)
            sec = timed(job, 1)
            out[f"c3_fixed_dt_two_steps_per_launch_{precision}"] = {
                "cell_updates_per_s": 8192 * 8192 * 100 / sec, "ms_per_job": sec * 1e3,
                "algorithmic_bytes_per_cell_update": (16 if precision == "f32" else 8),
                "kernel": s.two_step_kernel(), "kernel_choice": s.kernel_choice(two_step=True),
                "note": "job = set_state from device + 100 steps = 50 launches"}
    for mode in ("gated", "dataflow"):
        # one large instance: the batched table entry is keyed by total cells
        # and measured on 512 small instances, so these time their candidates
        with fvlib.Batch([dfix], "f32", stream=sptr, tune=1) as b:
            b.set_dataflow(mode == "dataflow")

            def job():
                b.set_state(0, pd, primitive=True)
                b.run(100)
            sec = timed(job, 1)
            out[f"c3_fixed_dt_batch_of_one_{mode}_f32"] = {
                "cell_updates_per_s": 8192 * 8192 * 100 / sec, "ms_per_job": sec * 1e3,
                "kernel": b.kernel_info()[1], "kernel_choice": b.kernel_choice(),
                "note": "job = set_state from device + 100 steps, one launch"}
    del pd
    # f2: the headline job with one state buffer updated in place (halos from
    # overlap strips) instead of two
    prim, d = wl.smooth_periodic(8192, dtype=np.float32)
    pd = torch.from_numpy(prim).to(f"cuda:{local}")
    for precision in ("f32", "f64"):
        with fvlib.Solver(d, precision, stream=sptr) as s:
            s.set_inplace(True)

            def job():
                s.set_state(pd, primitive=True)
                s.run(100 if precision == "f32" else 10)
            sec = timed(job, 1)
            nsteps = 100 if precision == "f32" else 10
            out[f"c3_inplace_{precision}"] = {
                "cell_updates_per_s": 8192 * 8192 * nsteps / sec, "ms_per_job": sec * 1e3,
                "kernel": s.kernel_info()[1], "kernel_choice": s.kernel_choice(),
                "note": f"job = set_state from device + {nsteps} steps; one state buffer + overlap strips"}
    del pd
    # C5: spray moments 2048^2, periodic, 200 steps; FP64 plain and FP32-bulk
    prim, d = wl.spray_field(2048)
    pd = torch.from_numpy(prim).to(f"cuda:{local}")
    g5 = golden_samples("c5")
    acc5 = {}
    for precision in ("f64", "f32"):
        with fvlib.Solver(d, precision, stream=sptr) as s:
            s.set_state(pd, primitive=True)
            s.run(2)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.run(200)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            out[f"c5_spray_2048_{precision}"] = {
                "cell_updates_per_s": 2048 * 2048 * 200 / sec, "ms_per_job": sec * 1e3,
                "kernel": s.kernel_info()[1], "kernel_choice": s.kernel_choice(),
                "bound": "fp64 pipe (maximum-entropy Newton in FP64 in both precisions)"}
            if dfma_peak:
                out[f"c5_spray_2048_{precision}"]["roofline"] = fp64_roofline(
                    f"spray step {precision}", 2048 * 2048 * 200 / sec, dfma_peak)
            if g5 is not None and accuracy is not None:
                s.set_state(pd, primitive=True)
                s.run(int(g5["steps"]))
                acc5[precision] = errors_vs(s.state().reshape(6, -1)[:, g5["flat_index"]], g5["W"])
    if acc5:
        accuracy["c5_spray_2048"] = dict(acc5, samples=int(len(g5["flat_index"])), steps=int(g5["steps"]),
                                         against="stored oracle samples (tests/golden/c5_oracle_samples.npz)")
    if oracle_too:
        out["c5_spray_2048_f64"]["oracle"] = oracle_sample(d, prim, 2, "a sample (cold Newton starts)")
    del pd
    return out



def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other configurations")
    ap.add_argument("--tune", type=int, default=0)
    ap.add_argument("--only", choices=["f32", "f64"], default=None,
                    help="time one precision only (profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1701_05431_gb300 import fvlib

    build, nsteps_job, desc = WORKLOADS[args.workload]
    prim, d = build()
    system = d["system"]
    nvar = BYTES_PER_CELL[system]
    ncell = d["nx"] * d["ny"]
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    prim_dev = torch.from_numpy(prim).to(f"cuda:{local}")

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    choices = {}

    def time_jobs(precision, steps, warmup, clocks=False):
        s = fvlib.Solver(d, precision, stream=sptr, tune=args.tune)
        s.set_state(prim_dev, primitive=True)
        for _ in range(warmup):
            s.run(nsteps_job)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ck = Clocks(local) if clocks else None
        barrier()
        if ck:
            ck.start()
        ev0.record(stream)
        for _ in range(steps):
            s.run(nsteps_job)
        ev1.record(stream)
        barrier()
        ck_res = ck.stop() if ck else None
        ms = max_over_ranks(ev0.elapsed_time(ev1), f"cuda:{local}")
        info = s.kernel_info()[1]
        choices[precision] = s.kernel_choice()
        s.close()
        return ms, ck_res, info

    if args.only == "f64":
        ms, _, kinfo = time_jobs("f64", args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"profile_only": "f64", "kernel": kinfo, "ms_per_step": ms / args.steps,
                              "value": ncell * nsteps_job * args.steps / (ms / 1e3)}))
        return 0

    # ---- FP32-bulk headline
    ms32, clk, kinfo32 = time_jobs("f32", args.steps, args.warmup, clocks=(rank == 0))
    # the step kernels of the region, and per job the one-warp read-back of
    # the control block that fv_run ends with
    launches = args.steps * nsteps_job
    value32 = whole_job_throughput(ncell, nsteps_job, args.steps, ws, ms32)
    hbm, peak_kind = peaks()
    algo_bytes_32 = 2 * nvar * 4 * ncell          # one read + one write per cell
    avg_launch_s = ms32 / 1e3 / launches
    achieved32 = algo_bytes_32 / avg_launch_s / 1e9

    out = {"metric": METRIC,
           "value": value32, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": job_config(desc, ncell, nsteps_job, ws),
           "kernel": kinfo32, "kernel_choice": choices.get("f32"),
           "roofline": {"bound": "hbm", "achieved": achieved32, "peak": hbm, "unit": "GB/s",
                        "frac": achieved32 / hbm, "frac_nominal": achieved32 / NOMINAL_HBM_GBS,
                        "traffic": (None if measured_traffic_per_cell(kinfo32) is None
                                    else measured_traffic_per_cell(kinfo32) * ncell),
                        "traffic_source": "ncu dram__bytes_read+write of one launch of this kernel on the 8192^2 workload",
                        "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                        "algorithmic_bytes_per_launch": algo_bytes_32,
                        "avg_launch_us": avg_launch_s * 1e6},
           "gpu_launches": launches + args.steps}
    if clk:
        out["clocks"] = clk

    # ---- FP64 plain beside it
    if args.only == "f32":
        args.no_fp64 = args.no_e2e = args.no_cpu_baseline = args.no_extra = True
    dfma_peak = None
    if not args.no_fp64:
        dfma_peak = fvlib.fma_peak("f64", 0.05, sptr)
        out["fp64_pipe_peak"] = {"dfma_per_s": dfma_peak, "tflops": 2 * dfma_peak / 1e12,
                                 "ffma_per_s": fvlib.fma_peak("f32", 0.05, sptr),
                                 "how": "fv_fma_peak: 8 blocks of 256 threads per SM, 8 independent FMA chains "
                                        "per thread, best of 3 launches of ~50 ms, CUDA events"}
        k64 = max(1, min(args.steps, 2))
        ms64, _, kinfo64 = time_jobs("f64", k64, 1)
        value64 = whole_job_throughput(ncell, nsteps_job, k64, ws, ms64)
        algo64 = 2 * nvar * 8 * ncell
        avg64 = ms64 / 1e3 / (k64 * nsteps_job)
        moved64 = (2 * 8 * 8 * ncell) if " pc" in kinfo64 else algo64
        out["fp64"] = {"value": value64, "unit": "cell-updates/s", "ms_per_step": ms64 / k64,
                       "steps": k64, "kernel": kinfo64,
                       "hbm_gbs_achieved": algo64 / avg64 / 1e9, "hbm_frac": algo64 / avg64 / 1e9 / hbm,
                       "roofline": fp64_roofline(kinfo64, value64 / ws, dfma_peak),
                       "traffic": {"algorithmic_bytes_per_cell_update": 2 * nvar * 8,
                                   "moved_bytes_per_cell_update": moved64 // ncell,
                                   "note": "the carried-primitive kernel (pc) stores u, v, p, c as four more "
                                           "planes: 128 B moved per cell-update against the method's 64"},
                       "note": "FP64 arithmetic is bound by the FP64 pipe, not HBM"}
        out["fp32_speedup_vs_fp64"] = value32 / value64
        out["fp64"]["gpu_launches"] = k64 * (nsteps_job + 1)
        out["fp64"]["kernel_choice"] = choices.get("f64")

    # ---- bfloat16 storage (FP32 arithmetic), 16 B per cell-update
    if not args.no_fp64:
        kb = max(1, min(args.steps, 3))
        msb, _, kinfob = time_jobs("bf16", kb, 2)
        valueb = whole_job_throughput(ncell, nsteps_job, kb, ws, msb)
        algob = 2 * nvar * 2 * ncell
        avgb = msb / 1e3 / (kb * nsteps_job)
        out["bf16_storage"] = {"value": valueb, "unit": "cell-updates/s", "ms_per_step": msb / kb, "steps": kb,
                               "kernel": kinfob, "hbm_gbs_achieved": algob / avgb / 1e9,
                               "hbm_frac": algob / avgb / 1e9 / hbm,
                               "kernel_choice": choices.get("bf16"),
                               "note": "bfloat16 state, FP32 arithmetic, FP64 dt/t/totals; accuracy below"}

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e:
        s = fvlib.Solver(d, "f32", stream=sptr, tune=args.tune)
        P0 = np.ascontiguousarray(prim.astype(np.float32))
        h_in = torch.from_numpy(P0).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        # one untimed job through the same calls (allocates the side buffers)
        s.prefetch_state(h_in, primitive=True)
        s.set_state_prefetched()
        s.run(nsteps_job)
        s.snapshot(h_out)
        s.snapshot_wait()
        k = max(20, args.steps)
        # each job: its input copied in from pinned host memory, nsteps_job
        # steps, its result copied out to pinned host memory.  The copy in of
        # job j+1 (fv_prefetch_state) and the copy out of job j (fv_snapshot)
        # run on side streams while job j+1's steps run; the first copy in and
        # the last copy out are inside the region and overlap nothing.
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.prefetch_state(h_in, primitive=True)
        for j in range(k):
            s.set_state_prefetched()
            if j + 1 < k:
                s.prefetch_state(h_in, primitive=True)
            s.run(nsteps_job)
            s.snapshot(h_out)
        s.snapshot_wait()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        wall = max_over_ranks(wall, f"cuda:{local}")
        s.close()
        out["e2e"] = {"value": ncell * nsteps_job * k * ws / wall, "unit": "cell-updates/s",
                      "h2d_bytes_per_step": int(h_in.numel() * 4), "d2h_bytes_per_step": int(h_out.numel() * 4),
                      "wall_s": wall, "steps": k,
                      "path": "fv_prefetch_state(pinned host f32 primitive, asynchronous, overlapping the previous "
                              "job) + fv_set_state_prefetched + fv_run + fv_snapshot(pinned host f32, "
                              "asynchronous, overlapping the next job) + fv_snapshot_wait; host wall clock"}
        # per job: load, wave-speed seed and control read-back (set_state_prefetched),
        # the steps and a read-back (fv_run), a read-back and the staging copy (fv_snapshot)
        out["e2e"]["gpu_launches"] = k * (nsteps_job + 6)

    # ---- accuracy of the timed configuration against stored oracle samples
    accuracy = {}
    g = golden_samples(args.workload)
    if g is not None:
        acc = {}
        for precision in ("f32", "f64", "bf16"):
            s = fvlib.Solver(d, precision, stream=sptr)
            s.set_state(prim_dev, primitive=True)
            s.run(int(g["steps"]))
            W = s.state()
            s.close()
            acc[precision] = errors_vs(W.reshape(W.shape[0], -1)[:, g["flat_index"]], g["W"])
        accuracy[WORKLOAD_KEYS.get(args.workload, args.workload)] = dict(
            acc, samples=int(len(g["flat_index"])), steps=int(g["steps"]),
            against=f"stored oracle samples (tests/golden/{args.workload}_oracle_samples.npz)")

    if not args.no_extra and args.workload == "c3":
        out["other_workloads"] = secondary_workloads(fvlib, torch, sptr, local, hbm,
                                                     oracle_too=(rank == 0 and not args.no_cpu_baseline and ws == 1),
                                                     accuracy=accuracy, dfma_peak=dfma_peak)
    if accuracy:
        out["accuracy_vs_oracle"] = dict(accuracy, norms="per variable: rel_l1 = sum|gpu-oracle| / sum|oracle|, "
                                                          "rel_linf = max|gpu-oracle| / max|oracle|")

    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline_run(args.workload, d, prim)

    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
