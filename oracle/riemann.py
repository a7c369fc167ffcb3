"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

TEST INFRASTRUCTURE ONLY (oracle side).  Used to pin the Euler flux of
Sec. 5, Eq. (Euler) against an exact solution: y-constant data on the 2D grid
must converge to it at first order.

Written from the wave relations of gas dynamics: across a shock the
Rankine-Hugoniot conditions give the velocity jump
    f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),
    A_K = 2 / ((gamma+1) rho_K),  B_K = (gamma-1)/(gamma+1) p_K,
and across a rarefaction the isentropic Riemann invariant gives
    f_K(p) = 2 c_K / (gamma-1) ((p/p_K)^((gamma-1)/(2 gamma)) - 1).
The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0 (Newton); the
solution is self-similar in xi = (x - x0)/t.
"""
from __future__ import annotations

import math

import numpy as np


def _f(p, rho, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (p + B)) * (1.0 - 0.5 * (p - pk) / (p + B))
    else:
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4):
    """(p*, u*) for primitive states left=(rho,u,p), right=(rho,u,p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _f(p, rl, pl, cl, g)
        fr, dfr = _f(p, rr, pr, cr, g)
        F = fl + fr + (ur - ul)
        dp = F / (dfl + dfr)
        pn = max(1e-14, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, cl, g)
    fr, _ = _f(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, g=1.4):
    """Primitive (rho, u, p) arrays at similarity coordinates xi."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    gm = (g - 1.0) / (g + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, s in enumerate(xi.ravel()):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    r, uu, pp = rl, ul, pl
                else:
                    r = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                    uu, pp = us, ps
            else:  # left rarefaction
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                head, tail = ul - cl, us - cs
                if s <= head:
                    r, uu, pp = rl, ul, pl
                elif s >= tail:
                    r = rl * (ps / pl) ** (1.0 / g)
                    uu, pp = us, ps
                else:
                    uu = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    r = rl * (c / cl) ** (2.0 / (g - 1))
                    pp = pl * (c / cl) ** (2.0 * g / (g - 1))
        else:  # right of contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    r, uu, pp = rr, ur, pr
                else:
                    r = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                    uu, pp = us, ps
            else:  # right rarefaction
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                head, tail = ur + cr, us + cs
                if s >= head:
                    r, uu, pp = rr, ur, pr
                elif s <= tail:
                    r = rr * (ps / pr) ** (1.0 / g)
                    uu, pp = us, ps
                else:
                    uu = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    r = rr * (c / cr) ** (2.0 / (g - 1))
                    pp = pr * (c / cr) ** (2.0 * g / (g - 1))
        rho.flat[k], u.flat[k], p.flat[k] = r, uu, pp
    return rho, u, p


def cell_average(left, right, x_edges, x0, t, g=1.4, sub=64):
    """Cell averages of (rho, rho u, rho E) of the exact solution over cells
    with the given edges, by `sub`-point midpoint sampling per cell."""
    x_edges = np.asarray(x_edges, dtype=np.float64)
    n = len(x_edges) - 1
    h = np.diff(x_edges)
    offs = (np.arange(sub) + 0.5) / sub
    xs = x_edges[:-1, None] + h[:, None] * offs[None, :]
    rho, u, p = sample(left, right, (xs - x0) / t, g)
    m = rho * u
    E = p / (g - 1.0) + 0.5 * rho * u * u
    return rho.mean(axis=1), m.mean(axis=1), E.mean(axis=1)
