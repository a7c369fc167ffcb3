"""Write sampled FP64-oracle outputs of the full-size workloads.

The full-size configurations take the CPU oracle minutes, too long to rerun
inside every GPU test, so this script runs them once and stores, for each, the
conserved variables at a fixed set of cells after the stated step count plus
the oracle's dt history.  It calls only the oracle (oracle/) and the input
generators (workloads/).

  python tests/golden/make_oracle_samples.py [c2] [c3] [c5]

Outputs tests/golden/<name>_oracle_samples.npz with arrays
  flat_index (cells sampled, j * nx + i), W (nvar x samples), dts, steps, t.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402
from tests.helpers import oracle_problem  # noqa: E402

CASES = {
    "c2": (lambda: wl.four_quadrant(2048, npart=8), 500),
    "c3": (lambda: wl.smooth_periodic(8192), 100),
    "c5": (lambda: wl.spray_field(2048), 40),
}


def sample_indices(nx, ny, seed=1701):
    rng = np.random.default_rng(seed)
    idx = set(rng.integers(0, nx * ny, size=4096).tolist())
    for j in (0, ny // 2, ny - 1):           # three full-ish row segments
        for i in range(0, min(nx, 512)):
            idx.add(j * nx + i)
        for i in range(max(0, nx - 64), nx):
            idx.add(j * nx + i)
    for i in (0, nx // 2, nx - 1):           # column segments
        for j in range(0, min(ny, 256)):
            idx.add(j * nx + i)
    return np.array(sorted(idx), dtype=np.int64)


def make(name):
    build, steps = CASES[name]
    prim, d = build()
    P = oracle_problem(d)
    W0 = oracle.prim_to_cons(P, prim)
    del prim
    t0 = time.time()
    r = oracle.run(P, W0, steps)
    el = time.time() - t0
    assert r.status == oracle.OK and r.steps == steps, (r.status, r.steps)
    idx = sample_indices(d["nx"], d["ny"])
    W = r.W.reshape(r.W.shape[0], -1)[:, idx]
    out = os.path.join(HERE, f"{name}_oracle_samples.npz")
    np.savez_compressed(out, flat_index=idx, W=W, dts=r.dts, steps=steps, t=r.t)
    print(f"{name}: {steps} steps in {el:.1f} s on {oracle.max_threads()} threads -> {out}")


if __name__ == "__main__":
    names = sys.argv[1:] or ["c2", "c3"]
    for n in names:
        make(n)
