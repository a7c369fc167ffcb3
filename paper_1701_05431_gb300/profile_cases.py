"""Small, self-contained invocations of each kernel, for profiling with ncu.

  python -m paper_1701_05431_gb300.profile_cases step --system euler --precision f32 --n 4096 --steps 3 [--inplace | --two-step]
  python -m paper_1701_05431_gb300.profile_cases batch --instances 96 --steps 4 --tune 2
  python -m paper_1701_05431_gb300.profile_cases spray --precision f64 --n 1024 --steps 3
  python -m paper_1701_05431_gb300.profile_cases sweep --workload c3 --precision f32

Each of the first three cases builds its seeded synthetic input (the
`workloads` generators), copies it to the device, sets the state through the
C ABI and advances the given number of time steps once; nothing is timed.
`--tune K` (K >= 2) forces kernel candidate K - 2, so that a capture sees a
known kernel.  `sweep` times every compiled candidate in turn on one workload
(c3: Euler 8192^2 smooth periodic; c2: four-quadrant 2048^2; c4: 512 batched
instances; c3tb: the c3 grid in fixed-dt mode with two-step passes;
c3inplace: the c3 grid with one state buffer) with CUDA events and prints one
JSON line per candidate.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _device(a):
    import numpy as np
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def step_case(system: str, precision: str, n: int, steps: int, tune: int, inplace: bool = False,
              two_step: bool = False) -> str:
    import torch
    import workloads as wl
    from paper_1701_05431_gb300 import fvlib
    if system == "euler":
        prim, d = wl.smooth_periodic(n)
    elif system == "advection":
        prim, d = wl.advection_bump(n)
    else:
        prim, d = wl.spray_field(n)
    if two_step:
        # the paper's fixed dt: 0.4 min(dx, dy) / lmax(W^0) (Euler)
        import numpy as np
        rho, u, v, p = (np.asarray(q, dtype=np.float64) for q in prim)
        lam0 = float(np.max(np.maximum(np.abs(u), np.abs(v)) + np.sqrt(1.4 * p / rho)))
        d = dict(d, fixed_dt=0.4 * min(1.0 / d["nx"], 1.0 / d["ny"]) / lam0)
    stream = torch.cuda.current_stream().cuda_stream
    with fvlib.Solver(d, precision, stream=stream, tune=tune) as s:
        if inplace:
            s.set_inplace(True)
        if two_step:
            s.set_time_blocking(2)
        s.set_state(_device(prim), primitive=True)
        s.run(steps)
        torch.cuda.synchronize()
        return s.two_step_kernel() or s.kernel_info()[1]


def batch_case(instances: int, steps: int, tune: int, precision: str = "f32") -> str:
    import torch
    import workloads as wl
    from paper_1701_05431_gb300 import fvlib
    insts = wl.batched_quadrants(instances)
    stream = torch.cuda.current_stream().cuda_stream
    with fvlib.Batch([d for _, _, d in insts], precision, stream=stream, tune=tune) as b:
        for k, (_, prim, _) in enumerate(insts):
            b.set_state(k, prim, primitive=True)
        b.run(steps)
        torch.cuda.synchronize()
        return b.kernel_info()[1]


def _timed(fn, reps=3):
    """Median device time (s) of fn() after one untimed call."""
    import torch
    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return sorted(ts)[len(ts) // 2]


def sweep(workload: str, precision: str, steps: int) -> None:
    import json
    import numpy as np
    import torch
    import workloads as wl
    from paper_1701_05431_gb300 import fvlib
    stream = torch.cuda.current_stream().cuda_stream
    if workload == "c4":
        insts = wl.batched_quadrants(512)
        ncells = sum(d["nx"] * d["ny"] for _, _, d in insts)
        k = 0
        while True:
            try:
                b = fvlib.Batch([d for _, _, d in insts], precision, stream=stream, tune=2 + k)
            except fvlib.FvError:
                break
            with b:
                for i, (_, prim, _) in enumerate(insts):
                    b.set_state(i, prim, primitive=True)
                sec = _timed(lambda: b.run(steps), 2)
                print(json.dumps({"workload": workload, "precision": precision, "kernel": b.kernel_info()[1],
                                  "cell_updates_per_s": ncells * steps / sec}), flush=True)
            k += 1
        return
    if workload == "c3inplace":
        # one state buffer, every in-place candidate
        prim, d = wl.smooth_periodic(8192, dtype=np.float32)
        dev = _device(prim)
        k = 0
        while True:
            with fvlib.Solver(d, precision, stream=stream, tune=2 + k) as s:
                try:
                    s.set_inplace(True)
                except fvlib.FvError:
                    break
                s.set_state(dev, primitive=True)
                sec = _timed(lambda: s.run(steps))
                print(json.dumps({"workload": workload, "precision": precision, "kernel": s.kernel_info()[1],
                                  "cell_updates_per_s": d["nx"] * d["ny"] * steps / sec}), flush=True)
            k += 1
        return
    if workload == "c3tb":
        # two-step passes, fixed dt = 0.4 min(dx, dy) / lmax(W^0), every two-step candidate
        prim, d = wl.smooth_periodic(8192, dtype=np.float32)
        rho, u, v, p = (np.asarray(q, dtype=np.float64) for q in prim)
        lam0 = float(np.max(np.maximum(np.abs(u), np.abs(v)) + np.sqrt(1.4 * p / rho)))
        d = dict(d, fixed_dt=0.4 / 8192 / lam0)
        dev = _device(prim)
        k = 0
        while True:
            with fvlib.Solver(d, precision, stream=stream, tune=2 + k) as s:
                try:
                    s.set_time_blocking(2)
                except fvlib.FvError:
                    break
                s.set_state(dev, primitive=True)
                sec = _timed(lambda: s.run(steps))
                print(json.dumps({"workload": workload, "precision": precision, "candidate": k,
                                  "cell_updates_per_s": d["nx"] * d["ny"] * steps / sec}), flush=True)
            k += 1
        return
    if workload == "c3":
        prim, d = wl.smooth_periodic(8192, dtype=np.float32)
    else:
        prim, d = wl.four_quadrant(2048, npart=8)
    dev = _device(prim)
    for k in range(len(fvlib.kernel_candidates("euler", precision))):
        with fvlib.Solver(d, precision, stream=stream, tune=2 + k) as s:
            s.set_state(dev, primitive=True)
            sec = _timed(lambda: s.run(steps))
            print(json.dumps({"workload": workload, "precision": precision, "kernel": s.kernel_info()[1],
                              "cell_updates_per_s": d["nx"] * d["ny"] * steps / sec}), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["step", "batch", "spray", "sweep"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c4", "c3tb", "c3inplace"])
    ap.add_argument("--system", default="euler", choices=["euler", "advection"])
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "bf16"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--instances", type=int, default=96)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--tune", type=int, default=0)
    ap.add_argument("--inplace", action="store_true", help="step case: one state buffer (fv_set_inplace)")
    ap.add_argument("--two-step", action="store_true",
                    help="step case (Euler): fixed dt and two time steps per launch (fv_set_time_blocking)")
    a = ap.parse_args(argv)
    if a.case == "sweep":
        sweep(a.workload, a.precision, a.steps)
        return
    if a.case == "step":
        k = step_case(a.system, a.precision, a.n, a.steps, a.tune, a.inplace, a.two_step)
    elif a.case == "spray":
        k = step_case("spray", a.precision, a.n, a.steps, a.tune)
    else:
        k = batch_case(a.instances, a.steps, a.tune, "f32" if a.precision == "bf16" else a.precision)
    print(f"{a.case}: {k}")


if __name__ == "__main__":
    main()
