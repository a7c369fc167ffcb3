"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws and lays out initial data; it holds none of the
finite-volume method's arithmetic (no flux, no equation of state, no
conversion to conserved variables -- each side does that itself).  Every
generator returns PRIMITIVE fields as a float64 array of shape
(nvar, ny, nx), x fastest, evaluated at cell centres
x_i = xmin + (i + 1/2) dx, y_j = ymin + (j + 1/2) dy:

  advection: (u,)
  euler:     (rho, u, v, p)
  spray:     (m0, m1/2, m1, m3/2, u, v)

together with a plain-dict problem description (grid, system, boundary
conditions, CFL, parameters) that both sides translate into their own types.

Workloads (the paper's test problems are analytic, so nothing stands in for a
dataset):
  advection_bump     scalar advection, a = (1, 0.5), 128^2, periodic
  four_quadrant      Euler four-quadrant Riemann data, 2048^2, transmissive
  smooth_periodic    Euler smooth periodic sinusoids, 8192^2
  batched_quadrants  512 Euler four-quadrant instances of random sizes
  spray_field        spray moments drawn inside the moment space
plus the paper's validation cases (localized cosine, isentropic vortex,
Sec. 5.1) and the Sod shock tube.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 1701054310

BC_NAMES = ("periodic", "transmissive", "dirichlet")


def centres(n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def problem(system: str, nx: int, ny: int, **kw) -> dict:
    d = dict(system=system, nx=nx, ny=ny, npart_x=1, npart_y=1, xmin=0.0, xmax=1.0, ymin=0.0,
             ymax=1.0, bc=("periodic",) * 4, bc_state=(), cfl=0.4, fixed_dt=0.0)
    if system == "advection":
        d["params"] = (1.0, 0.5)
    elif system == "euler":
        d["params"] = (1.4,)
    else:
        d["params"] = (0.1, 0.2, 1.0, 32.0, 1e-13)
    d.update(kw)
    return d


def _sin_sum(x, y, terms, amp):
    """amp * sum_k sin(2 pi (kx x + ky y) + phi) on the grid, evaluated in the
    separable form sin(a + b) = cos b sin a + sin b cos a as one small matrix
    product (rows: y factors, columns: x factors)."""
    cols_y, cols_x = [], []
    for kx, ky, phi in terms:
        a = 2.0 * math.pi * kx * x + phi
        b = 2.0 * math.pi * ky * y
        cols_y += [np.cos(b), np.sin(b)]
        cols_x += [np.sin(a), np.cos(a)]
    Y = np.stack(cols_y, axis=1)
    X = np.stack(cols_x, axis=0)
    return amp * (Y @ X)


# ---------------------------------------------------------------- advection
def advection_bump(n: int = 128):
    """u0 = 1 + exp(-((x-.5)^2 + (y-.5)^2)/0.01), a = (1, 0.5), CFL 0.5."""
    x = centres(n)
    y = centres(n)
    r2 = (x[None, :] - 0.5) ** 2 + (y[:, None] - 0.5) ** 2
    prim = (1.0 + np.exp(-r2 / 0.01))[None]
    return prim, problem("advection", n, n, cfl=0.5, params=(1.0, 0.5))


# ---------------------------------------------------------------- euler
FOUR_QUADRANT = {  # (rho, u, v, p)
    "NE": (1.5, 0.0, 0.0, 1.5),
    "NW": (0.5323, 1.206, 0.0, 0.3),
    "SW": (0.138, 1.206, 1.206, 0.029),
    "SE": (0.5323, 0.0, 1.206, 0.3),
}


def _quadrants(nx, ny, states, split=(0.5, 0.5)):
    x = centres(nx)
    y = centres(ny)
    east = (x > split[0])[None, :]
    north = (y > split[1])[:, None]
    prim = np.empty((4, ny, nx))
    for v in range(4):
        prim[v] = np.where(north, np.where(east, states["NE"][v], states["NW"][v]),
                           np.where(east, states["SE"][v], states["SW"][v]))
    return prim


def four_quadrant(n: int = 2048, npart: int = 8):
    """Four-quadrant Riemann data split at (0.5, 0.5), transmissive sides."""
    prim = _quadrants(n, n, FOUR_QUADRANT)
    return prim, problem("euler", n, n, npart_x=npart, npart_y=npart, bc=("transmissive",) * 4,
                         cfl=0.4)


def smooth_terms(seed: int = SEED):
    """Wave numbers and phases of the smooth periodic data: for each field
    (rho, u, v) and k = 1..4: kx, ky ~ U{1..8}, phi ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    terms = []
    for _field in range(3):
        t = []
        for _k in range(4):
            kx = int(rng.integers(1, 9))
            ky = int(rng.integers(1, 9))
            phi = float(rng.uniform(0.0, 2.0 * math.pi))
            t.append((kx, ky, phi))
        terms.append(t)
    return terms


def smooth_periodic(n: int = 8192, seed: int = SEED, dtype=np.float64):
    """rho = 1 + 0.2 sum_k sin(...), u, v = 0.3 sum_k sin(...), p = 1."""
    x = centres(n)
    y = centres(n)
    tr, tu, tv = smooth_terms(seed)
    prim = np.empty((4, n, n), dtype=dtype)
    prim[0] = 1.0 + _sin_sum(x, y, tr, 0.2)
    prim[1] = _sin_sum(x, y, tu, 0.3)
    prim[2] = _sin_sum(x, y, tv, 0.3)
    prim[3] = 1.0
    return prim, problem("euler", n, n, cfl=0.4)


def batched_sizes(n_inst: int = 512, seed: int = SEED, lo: int = 64, hi: int = 1024):
    rng = np.random.default_rng(seed + 4)
    specs = []
    for _ in range(n_inst):
        nx = int(rng.integers(lo, hi + 1))
        ny = int(rng.integers(lo, hi + 1))
        st = {}
        for q in ("NE", "NW", "SW", "SE"):
            rho = float(rng.uniform(0.1, 2.0))
            u = float(rng.uniform(-1.0, 1.0))
            v = float(rng.uniform(-1.0, 1.0))
            p = float(rng.uniform(0.1, 2.0))
            st[q] = (rho, u, v, p)
        specs.append((nx, ny, st))
    return specs


def batched_quadrants(n_inst: int = 512, seed: int = SEED, lo: int = 64, hi: int = 1024,
                      only=None):
    """Independent four-quadrant Euler instances on the unit square with
    Nx, Ny ~ U{lo..hi}, rho, p ~ U[0.1, 2], u, v ~ U[-1, 1] per quadrant,
    transmissive sides, CFL 0.4 each.  `only` selects a subset of indices."""
    specs = batched_sizes(n_inst, seed, lo, hi)
    out = []
    for k, (nx, ny, st) in enumerate(specs):
        if only is not None and k not in only:
            continue
        prim = _quadrants(nx, ny, st)
        out.append((k, prim, problem("euler", nx, ny, bc=("transmissive",) * 4, cfl=0.4)))
    return out


# ---------------------------------------------------------------- spray
def canonical_to_moments(m0, p1, p2, p3):
    """Moments (c0..c3) on [0,1] from the mass c0 and the canonical moments
    p1, p2, p3 in (0,1): zeta_1 = p1, zeta_k = (1 - p_{k-1}) p_k, and the
    Jacobi recurrence alpha_1 = zeta_1, beta_1 = zeta_1 zeta_2,
    alpha_2 = zeta_2 + zeta_3 gives c1 = c0 alpha_1, c2 = c0 (alpha_1^2 +
    beta_1), c3 = c0 (alpha_1^3 + 2 alpha_1 beta_1 + alpha_2 beta_1).
    (Input sampling only: any p in (0,1)^3 gives a point strictly inside the
    moment space.)"""
    z1 = p1
    z2 = (1.0 - p1) * p2
    z3 = (1.0 - p2) * p3
    a1 = z1
    b1 = z1 * z2
    a2 = z2 + z3
    c1 = m0 * a1
    c2 = m0 * (a1 * a1 + b1)
    c3 = m0 * (a1 ** 3 + 2.0 * a1 * b1 + a2 * b1)
    return m0, c1, c2, c3


def spray_terms(seed: int = SEED):
    rng = np.random.default_rng(seed + 5)
    def term():
        return (int(rng.integers(1, 5)), int(rng.integers(1, 5)), float(rng.uniform(0, 2 * math.pi)))
    centre = (2.0 / 3.0, 0.25, 0.6)  # canonical moments of n(S) = const
    pbar = [c + float(rng.uniform(-0.05, 0.05)) for c in centre]
    mbar = float(rng.uniform(0.5, 1.5))
    tp = [term() for _ in range(3)]
    tm = term()
    tu = term()
    tv = term()
    return pbar, mbar, tp, tm, tu, tv


def spray_field(n: int = 2048, seed: int = SEED):
    """Spray moments inside the moment space with smooth modulation:
    canonical moments p_k = pbar_k + 0.08 sin(...), with pbar_k drawn within
    +-0.05 of (2/3, 1/4, 3/5), the canonical moments of a constant density
    n(S) = C (so the reconstructed densities stay bounded at S = 0);
    m0 = mbar (1 + 0.3 sin(...)), mbar ~ U[0.5, 1.5]; u, v = 0.5 sin(...).
    Periodic unit square, CFL 0.4, K = 0.1, theta = 0.2, Taylor-Green gas
    velocity, 32 quadrature nodes."""
    x = centres(n)
    y = centres(n)
    pbar, mbar, tp, tm, tu, tv = spray_terms(seed)
    p = [pbar[k] + _sin_sum(x, y, [tp[k]], 0.08) for k in range(3)]
    m0 = mbar * (1.0 + _sin_sum(x, y, [tm], 0.3))
    c = canonical_to_moments(m0, p[0], p[1], p[2])
    prim = np.empty((6, n, n))
    for k in range(4):
        prim[k] = c[k]
    prim[4] = _sin_sum(x, y, [tu], 0.5)
    prim[5] = _sin_sum(x, y, [tv], 0.5)
    return prim, problem("spray", n, n, cfl=0.4)


def spray_field_wide(n: int = 2048, seed: int = SEED):
    """Spray moments spread over the moment space: canonical moments
    p_k = pbar_k + 0.2 sin(...) clipped to [0.05, 0.95], pbar_k ~ U[0.25, 0.75];
    m0 = mbar (1 + 0.3 sin(...)), mbar ~ U[0.5, 1.5]; u, v = 0.5 sin(...).
    The densities reach far from a constant (n(0) up to a few hundred), so
    forward-Euler evaporation can leave the moment space after some steps.
    Same problem description as spray_field."""
    rng = np.random.default_rng(seed + 11)

    def term():
        return (int(rng.integers(1, 5)), int(rng.integers(1, 5)), float(rng.uniform(0, 2 * math.pi)))
    pbar = [float(rng.uniform(0.25, 0.75)) for _ in range(3)]
    mbar = float(rng.uniform(0.5, 1.5))
    tp = [term() for _ in range(3)]
    tm, tu, tv = term(), term(), term()
    x = centres(n)
    y = centres(n)
    p = [np.clip(pbar[k] + _sin_sum(x, y, [tp[k]], 0.2), 0.05, 0.95) for k in range(3)]
    m0 = mbar * (1.0 + _sin_sum(x, y, [tm], 0.3))
    c = canonical_to_moments(m0, p[0], p[1], p[2])
    prim = np.empty((6, n, n))
    for k in range(4):
        prim[k] = c[k]
    prim[4] = _sin_sum(x, y, [tu], 0.5)
    prim[5] = _sin_sum(x, y, [tv], 0.5)
    return prim, problem("spray", n, n, cfl=0.4)


# ---------------------------------------------------------------- validation cases
def localized_cosine(n: int, repaired: bool = True, gamma: float = 1.4):
    """Sec. 5.1.1: density bump advected by (1, 1), p = 1/gamma.  The printed
    profile rho = 1 + (r < 0.25) cos(4 pi r) vanishes at r -> 0.25; the
    repaired profile 1 + (r < 0.25) (1 + cos(4 pi r))/2 is continuous."""
    x = centres(n)
    y = centres(n)
    r = np.sqrt((x[None, :] - 0.5) ** 2 + (y[:, None] - 0.5) ** 2)
    if repaired:
        rho = 1.0 + (r < 0.25) * 0.5 * (1.0 + np.cos(4.0 * math.pi * r))
    else:
        rho = 1.0 + (r < 0.25) * np.cos(4.0 * math.pi * r)
    prim = np.empty((4, n, n))
    prim[0] = rho
    prim[1] = 1.0
    prim[2] = 1.0
    prim[3] = 1.0 / gamma
    return prim, problem("euler", n, n, cfl=0.4, params=(gamma,))


def localized_cosine_exact(n: int, t: float, repaired: bool = True):
    """Density of Eq. (LCAnalytic) at the cell centres at time t (point values)."""
    x = centres(n)
    y = centres(n)
    xs = x[None, :] - t
    ys = y[:, None] - t
    r = np.sqrt((xs - np.floor(xs) - 0.5) ** 2 + (ys - np.floor(ys) - 0.5) ** 2)
    if repaired:
        return 1.0 + (r < 0.25) * 0.5 * (1.0 + np.cos(4.0 * math.pi * r))
    return 1.0 + (r < 0.25) * np.cos(4.0 * math.pi * r)


def isentropic_vortex(n: int, gamma: float = 1.4, R: float = 0.1, wbar: float = 1.0,
                      ubar=(1.0, 1.0), t: float = 0.0):
    """Sec. 5.1.2, Eq. (RotatingGaussian)/(SetUp), centred at (0.5, 0.5) and
    advected by ubar (periodic wrap) to time t."""
    x = centres(n)
    y = centres(n)
    xs = x[None, :] - ubar[0] * t
    ys = y[:, None] - ubar[1] * t
    dx = xs - np.floor(xs) - 0.5
    dy = ys - np.floor(ys) - 0.5
    r2 = dx ** 2 + dy ** 2
    w = wbar * np.exp(-r2 / (2.0 * R * R))
    rho = (1.0 - (gamma - 1.0) / 2.0 * w ** 2) ** (1.0 / (gamma - 1.0))
    prim = np.empty((4, n, n))
    prim[0] = rho
    prim[1] = ubar[0] - dy / R * w
    prim[2] = ubar[1] + dx / R * w
    prim[3] = rho ** gamma / gamma
    return prim, problem("euler", n, n, cfl=0.4, params=(gamma,))


SOD_LEFT = (1.0, 0.0, 1.0)      # rho, u, p
SOD_RIGHT = (0.125, 0.0, 0.1)


def sod_x(nx: int, ny: int = 4, x0: float = 0.5):
    """Sod shock tube along x, constant in y, transmissive in x, periodic in y."""
    x = centres(nx)
    left = (x < x0)[None, :]
    prim = np.empty((4, ny, nx))
    prim[0] = np.where(left, SOD_LEFT[0], SOD_RIGHT[0])
    prim[1] = np.where(left, SOD_LEFT[1], SOD_RIGHT[1])
    prim[2] = 0.0
    prim[3] = np.where(left, SOD_LEFT[2], SOD_RIGHT[2])
    bc = ("transmissive", "periodic", "transmissive", "periodic")
    return prim, problem("euler", nx, ny, bc=bc, cfl=0.4)


def random_smooth_euler(n: int, seed: int, ny: int = None):
    """Small random smooth periodic Euler data (parity and invariance tests)."""
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    x = centres(n)
    y = centres(ny)
    def field(amp):
        t = [(int(rng.integers(1, 4)), int(rng.integers(1, 4)), float(rng.uniform(0, 2 * math.pi)))
             for _ in range(3)]
        return _sin_sum(x, y, t, amp)
    prim = np.empty((4, ny, n))
    prim[0] = 1.0 + field(0.15)
    prim[1] = field(0.3)
    prim[2] = field(0.3)
    prim[3] = 1.0 + field(0.1)
    return prim, problem("euler", n, ny, cfl=0.4)
