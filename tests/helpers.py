"""Test-side helpers: translate a workload description into the oracle's
problem type and compare arrays the way the tests state their tolerances."""
from __future__ import annotations

import numpy as np

import oracle

SYSTEMS = {"advection": oracle.ADVECTION, "euler": oracle.EULER, "spray": oracle.SPRAY}
BCS = {"periodic": oracle.PERIODIC, "transmissive": oracle.TRANSMISSIVE,
       "dirichlet": oracle.DIRICHLET}


def oracle_problem(d: dict, **over) -> oracle.Problem:
    d = dict(d, **over)
    return oracle.Problem(nx=d["nx"], ny=d["ny"], system=SYSTEMS[d["system"]],
                          npart_x=d.get("npart_x", 1), npart_y=d.get("npart_y", 1),
                          xmin=d.get("xmin", 0.0), xmax=d.get("xmax", 1.0),
                          ymin=d.get("ymin", 0.0), ymax=d.get("ymax", 1.0),
                          bc=tuple(BCS[b] for b in d["bc"]), bc_state=tuple(d.get("bc_state", ())),
                          cfl=d.get("cfl", 0.4), fixed_dt=d.get("fixed_dt", 0.0),
                          params=tuple(d["params"]))


def rel_linf(a, b, axis_vars=True):
    """Per-variable relative L-infinity error max|a-b| / max|b|."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = []
    for v in range(b.shape[0]):
        den = np.max(np.abs(b[v]))
        out.append(np.max(np.abs(a[v] - b[v])) / (den if den > 0 else 1.0))
    return np.array(out)


def rel_l1(a, b):
    """Per-variable relative L1 error sum|a-b| / sum|b| (dx dy cancels)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = []
    for v in range(b.shape[0]):
        den = np.sum(np.abs(b[v]))
        out.append(np.sum(np.abs(a[v] - b[v])) / (den if den > 0 else 1.0))
    return np.array(out)


def transpose_state(W, system):
    """Swap x and y: transpose every plane and exchange the x/y momentum
    components (Euler: vars 1, 2; spray: vars 4, 5)."""
    Wt = np.ascontiguousarray(np.transpose(W, (0, 2, 1)))
    if system == "euler":
        Wt[[1, 2]] = Wt[[2, 1]]
    elif system == "spray":
        Wt[[4, 5]] = Wt[[5, 4]]
    return Wt


def euler_lmax(prim, gamma=1.4):
    """lmax of a primitive Euler field over the two axis normals:
    max(|u|, |v|) + sqrt(gamma p / rho)."""
    rho, u, v, p = prim
    return float(np.max(np.maximum(np.abs(u), np.abs(v)) + np.sqrt(gamma * p / rho)))


def with_fixed_dt(d, prim, cfl):
    """The problem in the paper's fixed-dt mode, dt = cfl min(dx, dy) / lmax(W^0)."""
    h = min((d["xmax"] - d["xmin"]) / d["nx"], (d["ymax"] - d["ymin"]) / d["ny"])
    return dict(d, fixed_dt=cfl * h / euler_lmax(prim))
