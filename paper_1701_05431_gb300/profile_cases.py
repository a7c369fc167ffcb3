"""Small, self-contained invocations of each kernel, for profiling with ncu.

  python -m paper_1701_05431_gb300.profile_cases step --system euler --precision f32 --n 4096 --steps 3 [--inplace | --two-step]
  python -m paper_1701_05431_gb300.profile_cases batch --instances 96 --steps 4 --tune 2
  python -m paper_1701_05431_gb300.profile_cases spray --precision f64 --n 1024 --steps 3
  python -m paper_1701_05431_gb300.profile_cases peak --seconds 0.02

Each of the first three cases builds its seeded synthetic input (the
`workloads` generators), copies it to the device, sets the state through the
C ABI and advances the given number of time steps once; nothing is timed.
`--tune K` (K >= 2) forces kernel candidate K - 2, so that a capture sees a
known kernel.  `peak` runs the FMA-pipe throughput measurement
(fv_fma_peak) in FP64 and FP32 once each.
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


def peak_case(seconds: float) -> str:
    from paper_1701_05431_gb300 import fvlib
    r64 = fvlib.fma_peak("f64", seconds)
    r32 = fvlib.fma_peak("f32", seconds)
    return f"DFMA {r64:.4g}/s, FFMA {r32:.4g}/s"


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["step", "batch", "spray", "peak"])
    ap.add_argument("--seconds", type=float, default=0.02, help="peak case: length of each timed launch")
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
    if a.case == "peak":
        k = peak_case(a.seconds)
    elif a.case == "step":
        k = step_case(a.system, a.precision, a.n, a.steps, a.tune, a.inplace, a.two_step)
    elif a.case == "spray":
        k = step_case("spray", a.precision, a.n, a.steps, a.tune)
    else:
        k = batch_case(a.instances, a.steps, a.tune, "f32" if a.precision == "bf16" else a.precision)
    print(f"{a.case}: {k}")


if __name__ == "__main__":
    main()
