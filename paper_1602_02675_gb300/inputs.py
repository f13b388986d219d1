"""Seeded synthetic inputs shaped like the paper's workloads.

Primitive fields and workload descriptions only (densities, velocities,
pressures, sizes, seeds); nothing here computes any step of the method.
Both the CUDA path and the oracle convert these primitives themselves.

Workloads (Section V.C shock tube and its extensions):
* sod_1d          - 1000-node Sod tube on [0, 1], diaphragm at 0.5, t = 0.2
* sod_2d          - 4096 x 512 square lattice, x-only Sod jump, transmissive
                    x ends, reflecting y walls, t = 0.2
* tubes_batch     - many independent 1-D tubes with seeded lengths and
                    Riemann states
* cylinder_2d     - 8192^2 periodic box, circle r < 0.4 about (0.5, 0.5)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED = 20260

SOD_LEFT = (1.0, 0.0, 1.0)     # (rho, u, p), Section V.C
SOD_RIGHT = (0.125, 0.0, 0.1)
GAMMA = 1.4


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    nx: int
    ny: int
    t_end: float
    bc_x: int
    bc_y: int
    geom: int              # 0 planar x-jump, 1 circle
    inner: tuple           # (rho, u, v, p)
    outer: tuple
    a0: float = 0.5        # diaphragm x, or circle centre x
    a1: float = 0.5        # circle centre y
    radius: float = 0.0
    steps: int | None = None   # fixed step count (else from t_end)


def _p4(s):
    return s if len(s) == 4 else (s[0], s[1], 0.0, s[2])


SOD_1D = Workload("sod_1d_1000", 1, 1000, 1, 0.2, 0, 1, 0, _p4(SOD_LEFT),
                  _p4(SOD_RIGHT))
SOD_2D = Workload("sod_2d_4096x512", 2, 4096, 512, 0.2, 0, 1, 0,
                  _p4(SOD_LEFT), _p4(SOD_RIGHT))
CYLINDER_2D = Workload("cylinder_2d_8192x8192", 2, 8192, 8192, 0.0, 2, 2, 1,
                       (1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1), 0.5, 0.5,
                       0.4, steps=2000)


def random_smooth_prims(dim: int, nx: int, ny: int, seed: int,
                        vmax: float = 0.9, jump: bool = True):
    """Smooth random primitive fields (rho, u, v, p), optionally with a
    contact/shock-like jump, x fastest.  v is None in 1-D."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny if dim == 2 else np.zeros(1)
    X, Y = np.meshgrid(x, y)
    ph = rng.uniform(0.0, 2.0 * np.pi, 8)
    k = rng.integers(1, 4, 4)
    rho = 1.0 + 0.4 * np.sin(2 * np.pi * k[0] * X + ph[0]) * np.cos(
        2 * np.pi * k[1] * Y + ph[1])
    u = vmax * np.sin(2 * np.pi * k[2] * X + ph[2])
    v = vmax * np.cos(2 * np.pi * k[3] * Y + ph[3]) if dim == 2 else None
    p = 1.0 + 0.5 * np.cos(2 * np.pi * (X + Y) + ph[4])
    if jump:
        xd = rng.uniform(0.3, 0.7)
        rho = np.where(X < xd, rho, 0.2 * rho)
        p = np.where(X < xd, p, 0.15 * p)
    out = [rho.ravel(), u.ravel(), None if v is None else v.ravel(), p.ravel()]
    return out


def banded_prims(nx: int, ny: int, seed: int, u_band=(0.1, 0.8),
                 v_band=(-0.8, -0.1), p_over_rho: float = 1.0):
    """Smooth random 2-D primitive fields (rho, u, v, p), x fastest, whose
    velocities stay inside the given open bands and whose p/rho stays within
    15 % of p_over_rho, so that every node starts with the same floor of
    its lattice velocity (at lambda = 1) and the same level speeds."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    ph = rng.uniform(0.0, 2.0 * np.pi, 6)
    k = rng.integers(1, 4, 6)

    def wave(i, j):
        return np.sin(2 * np.pi * (k[i] * X + k[j] * Y) + ph[i])

    def band(lo, hi, w):
        mid, half = 0.5 * (lo + hi), 0.45 * (hi - lo)
        return mid + half * w

    rho = 1.0 + 0.3 * wave(0, 1)
    u = band(u_band[0], u_band[1], wave(2, 3))
    v = band(v_band[0], v_band[1], wave(4, 5))
    p = rho * p_over_rho * (1.0 + 0.15 * np.cos(2 * np.pi * (X - Y) + ph[1]))
    return [rho.ravel(), u.ravel(), v.ravel(), p.ravel()]


def patch_prims(nx: int, ny: int, seed: int, patch: int = 7,
                u_max: float = 1.3, p_over_rho=(0.3, 3.5)):
    """2-D primitive fields (rho, u, v, p), x fastest, made of square
    patches of `patch` nodes with their own random velocity (|u|, |v| <
    u_max) and p/rho (log-uniform in the given range), each with a gentle
    smooth ripple: at lambda = 1 a window of a few dozen patches holds
    lattice shifts floor(V) of both signs on both axes and several level
    speeds at once (c1 up to 2, reach up to 6 over the first steps)."""
    rng = np.random.default_rng(seed)
    px, py = -(-nx // patch), -(-ny // patch)
    u = rng.uniform(-u_max, u_max, (py, px))
    v = rng.uniform(-u_max, u_max, (py, px))
    por = np.exp(rng.uniform(np.log(p_over_rho[0]), np.log(p_over_rho[1]),
                             (py, px)))
    rho = rng.uniform(0.5, 1.5, (py, px))
    iy = np.arange(ny) // patch
    ix = np.arange(nx) // patch
    X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
    ripple = 1.0 + 0.02 * np.sin(2 * np.pi * (3 * X + 2 * Y) + rng.uniform(0, 6))
    R = rho[iy][:, ix] * ripple
    U = u[iy][:, ix] * ripple
    V = v[iy][:, ix] / ripple
    P = R * por[iy][:, ix]
    return [R.ravel(), U.ravel(), V.ravel(), P.ravel()]


def random_node_prims(dim: int, n: int, seed: int):
    """Independent random states per node (harsh: exercises every level
    count, fractional velocities of both signs, large reach)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.1, 3.0, n)
    u = rng.uniform(-1.8, 1.8, n)
    v = rng.uniform(-1.8, 1.8, n) if dim == 2 else None
    p = np.exp(rng.uniform(np.log(0.02), np.log(3.0), n)) * rho
    return [rho, u, v, p]


@dataclass(frozen=True)
class Tube:
    n: int
    left: tuple   # (rho, u, p)
    right: tuple

    def lattice_speed_scale(self) -> float:
        """lambda0 = dt/dx before rounding to a whole number of steps:
        1 unless one side is hotter (larger p/rho) than the left Sod state
        (1, 0, 1); then scaled down so that the hottest initial state has
        that same lattice temperature: lambda0^2 max(p/rho) = 1."""
        t = max(self.left[2] / self.left[0], self.right[2] / self.right[0])
        return min(1.0, (1.0 / t) ** 0.5)

    def steps_and_lambda(self, t_end: float = 0.2):
        """Whole number of steps reaching t_end with dt/dx <= lambda0."""
        dx = 1.0 / self.n
        n = max(1, int(math.ceil(t_end / (self.lattice_speed_scale() * dx)
                                 - 1e-9)))
        return n, t_end / (n * dx)


def tubes_batch(count: int = 4096, seed: int = SEED + 2,
                nmin: int = 256, nmax: int = 16384):
    """Independent 1-D tubes: lengths uniform in [nmin, nmax], pressure ratio
    log-uniform in [2, 100], density ratio uniform in [1, 10], at rest; the
    left state is (1, 0, 1)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, count)
    pr = np.exp(rng.uniform(np.log(2.0), np.log(100.0), count))
    dr = rng.uniform(1.0, 10.0, count)
    return [Tube(int(n), (1.0, 0.0, 1.0), (1.0 / d, 0.0, 1.0 / q))
            for n, q, d in zip(ns, pr, dr)]
