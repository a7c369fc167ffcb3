"""Autotuner: time every compiled kernel candidate on each configuration and
record the fastest per (system, precision, grid-size class, mode).

  python -m paper_1701_05431_gb300.autotune [--out-dir DIR] [--only NAME ...] [--merge TABLE.json]

For each configuration below it builds the seeded synthetic input, and for
every candidate of the configuration's mode (two state buffers, in place, two
time steps per launch, batched) it loads the state through the C ABI, runs a
few untimed warm-up steps and times `steps` steps three times with CUDA
events on the launching stream; the median is the candidate's rate.  It
writes

  DIR/fv_tune_table.inc   the fastest candidate per key, compiled into the
                          library (csrc/fv_tune_table.inc) and read by every
                          context created with fv_config.tune = 0;
  DIR/tune_table.json     every candidate's measured rate per configuration.

DIR defaults to the package's csrc/ (the .inc) and the package directory (the
.json); the library must be rebuilt afterwards to use a new table.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SYS_ID = {"advection": 0, "euler": 1, "spray": 2}
PREC_ID = {"f64": 0, "f32": 1, "bf16": 2}
MODE_ID = {"single": 0, "inplace": 1, "two-step": 2, "batch": 3}


def size_class(cells: int) -> int:
    """Grid-size class of a cell count, as the library computes it:
    0 below 2^16 cells, 1 below 2^20, 2 below 2^24, 3 from 2^24 on."""
    if cells < 1 << 16:
        return 0
    if cells < 1 << 20:
        return 1
    if cells < 1 << 24:
        return 2
    return 3


def _fixed_dt(prim, d, cfl=0.4, gamma=1.4):
    import numpy as np
    rho, u, v, p = (np.asarray(q, dtype=np.float64) for q in prim)
    lam = float(np.max(np.maximum(np.abs(u), np.abs(v)) + np.sqrt(gamma * p / rho)))
    return dict(d, fixed_dt=cfl * min(1.0 / d["nx"], 1.0 / d["ny"]) / lam)


def configurations():
    """(name, workload description, system, precision, mode, builder, steps, warm-up steps)."""
    import numpy as np
    import workloads as wl
    c3 = lambda: wl.smooth_periodic(8192, dtype=np.float32)  # noqa: E731
    c3f = lambda: (lambda pr, d: (pr, _fixed_dt(pr, d)))(*wl.smooth_periodic(8192, dtype=np.float32))  # noqa: E731
    c2 = lambda: wl.four_quadrant(2048, npart=8)  # noqa: E731
    c5 = lambda: wl.spray_field(2048)  # noqa: E731
    return [
        ("c1", "advection 128^2 periodic", "advection", "f64", "single", lambda: wl.advection_bump(128), 100, 10),
        ("c2_f64", "euler 2048^2 four-quadrant", "euler", "f64", "single", c2, 20, 2),
        ("c2_f32", "euler 2048^2 four-quadrant", "euler", "f32", "single", c2, 100, 10),
        ("c3_f32", "euler 8192^2 smooth periodic", "euler", "f32", "single", c3, 20, 3),
        ("c3_f64", "euler 8192^2 smooth periodic", "euler", "f64", "single", c3, 4, 1),
        ("c3_bf16", "euler 8192^2 smooth periodic", "euler", "bf16", "single", c3, 20, 3),
        ("c3_inplace_f32", "euler 8192^2 smooth periodic", "euler", "f32", "inplace", c3, 20, 3),
        ("c3_inplace_f64", "euler 8192^2 smooth periodic", "euler", "f64", "inplace", c3, 4, 1),
        ("c3_inplace_bf16", "euler 8192^2 smooth periodic", "euler", "bf16", "inplace", c3, 20, 3),
        ("c3_two_step_f32", "euler 8192^2 smooth periodic, fixed dt", "euler", "f32", "two-step", c3f, 20, 4),
        ("c3_two_step_bf16", "euler 8192^2 smooth periodic, fixed dt", "euler", "bf16", "two-step", c3f, 20, 4),
        ("c4", "512 batched euler four-quadrant instances", "euler", "f32", "batch", None, 40, 4),
        ("c5_f64", "spray 2048^2 periodic", "spray", "f64", "single", c5, 10, 3),
        ("c5_f32", "spray 2048^2 periodic", "spray", "f32", "single", c5, 10, 3),
    ]


def _median_time(run, steps, reps=3):
    import torch
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return sorted(ts)[len(ts) // 2]


def tune_single(fvlib, torch, prim, d, precision, mode, steps, warm):
    """Rates of every candidate of a single-instance mode: [(kernel, rate)]."""
    dev = torch.from_numpy(prim).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    cells = d["nx"] * d["ny"]
    out = []
    k = 0
    while True:
        try:
            s = fvlib.Solver(d, precision, stream=stream, tune=2 + k)
        except fvlib.FvError:
            break
        with s:
            try:
                if mode == "inplace":
                    s.set_inplace(True)
                elif mode == "two-step":
                    s.set_time_blocking(2)
            except fvlib.FvError:
                break
            s.set_state(dev, primitive=True)
            s.run(warm)
            torch.cuda.synchronize()
            sec = _median_time(lambda n: s.run(n), steps)
            name = s.two_step_kernel() if mode == "two-step" else s.kernel_info()[1].split(", ")[0]
            out.append((name, cells * steps / sec))
        k += 1
    return out


def tune_batch(fvlib, torch, precision, steps, warm):
    import workloads as wl
    insts = wl.batched_quadrants(512)
    cells = sum(d["nx"] * d["ny"] for _, _, d in insts)
    stream = torch.cuda.current_stream().cuda_stream
    out = []
    k = 0
    while True:
        try:
            b = fvlib.Batch([d for _, _, d in insts], precision, stream=stream, tune=2 + k)
        except fvlib.FvError:
            break
        with b:
            for i, (_, prim, _) in enumerate(insts):
                b.set_state(i, prim, primitive=True)
            b.run(warm)
            torch.cuda.synchronize()
            sec = _median_time(lambda n: b.run(n), steps)
            out.append((b.kernel_info()[1], cells * steps / sec))
        k += 1
    return out, cells


def write_table(results, inc_path, json_path):
    lines = ["// Written by python -m paper_1701_05431_gb300.autotune on one GB300: for each",
             "// (system, precision, grid-size class, mode) the candidate measured fastest, its",
             "// cell-updates/s and the workload it was measured on (CUDA events, median of 3).",
             "// {system, precision, size class, mode, kernel, rate, workload}"]
    for r in results:
        best = max(r["candidates"], key=lambda kv: kv[1])
        lines.append(f'    {{{SYS_ID[r["system"]]}, {PREC_ID[r["precision"]]}, {r["size_class"]}, '
                     f'{MODE_ID[r["mode"]]}, "{best[0]}", {best[1]:.4e}, "{r["workload"]}"}},')
    with open(inc_path, "w") as f:
        f.write("\n".join(lines) + "\n")
    with open(json_path, "w") as f:
        json.dump(results, f, indent=1)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--out-dir", default=None)
    ap.add_argument("--only", nargs="*", default=None, help="configuration names to tune (default: all)")
    ap.add_argument("--merge", default=None,
                    help="an existing tune_table.json whose other configurations are kept in the table written")
    a = ap.parse_args(argv)
    import torch
    from paper_1701_05431_gb300 import fvlib
    assert torch.cuda.is_available(), "the autotuner times kernels on a GPU"
    results = []
    for name, desc, system, precision, mode, build, steps, warm in configurations():
        if a.only and name not in a.only:
            continue
        t0 = time.time()
        if mode == "batch":
            cand, cells = tune_batch(fvlib, torch, precision, steps, warm)
        else:
            prim, d = build()
            cells = d["nx"] * d["ny"]
            cand = tune_single(fvlib, torch, prim, d, precision, mode, steps, warm)
            del prim
        torch.cuda.empty_cache()
        r = {"name": name, "workload": desc, "system": system, "precision": precision, "mode": mode,
             "cells": cells, "size_class": size_class(cells), "steps_timed": steps,
             "candidates": cand, "seconds": round(time.time() - t0, 1)}
        results.append(r)
        best = max(cand, key=lambda kv: kv[1])
        print(json.dumps({"name": name, "best": best[0], "rate": best[1], "candidates": len(cand)}), flush=True)
    if a.merge:
        with open(a.merge) as f:
            kept = [r for r in json.load(f) if r["name"] not in {x["name"] for x in results}]
        order = [c[0] for c in configurations()]
        results = sorted(kept + results, key=lambda r: order.index(r["name"]) if r["name"] in order else len(order))
    inc = os.path.join(a.out_dir or os.path.join(HERE, "csrc"), "fv_tune_table.inc")
    js = os.path.join(a.out_dir or HERE, "tune_table.json")
    write_table(results, inc, js)
    print(f"wrote {inc} and {js}")


if __name__ == "__main__":
    main()
