"""Seeded synthetic extension problems shaped like the paper's test problems.

This module only draws inputs (level set function phi, field f, grid sizes, boundary rules and
arrival times).  It holds none of the extension method's arithmetic and imports neither the CUDA
binding nor the oracle, so both sides can be fed the same inputs.

Every instance uses one numpy PCG64 generator seeded with ``seed + index``.  Grids are placed on
[-1, 1]^2: cell-centred (x_i = -1 + (i + 1/2) h, h = 2/n) on symmetric and periodic axes, and, on
Dirichlet axes, n interior nodes with the zero boundary nodes one spacing outside the grid
(x_i = -1 + (i + 1) h, h = 2/(n + 1)), as in Algorithm 1's padding.

Families (all returned as float32 arrays of shape [ny][nx]):

* ``circle``: phi = r - 0.5, f = cos(2x) sin(3y) + 0.5 x, field known inside.  Example-1-like.
* ``star``: phi = r - R0 (1 + a cos(m theta)), f = exp(-r^2)(1 + 0.3 sin 4x), known outside.
* ``wobbly``: phi = r - 0.4 (1 + sum_{k=2..6} a_k cos(k theta + b_k)), a_k ~ U(0, 0.05),
  b_k ~ U(0, 2 pi); f a random sum of 8 plane-wave modes (wavenumber pi k in a random direction,
  amplitude N(0, 1)/k^2, random phase), known inside.
* ``circles``: phi = min_i (|x - c_i| - rho_i) over three circles, c_i ~ U[-0.5, 0.5]^2,
  rho_i ~ U(0.2, 0.35); f as for ``wobbly``, known outside.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1704
SYMMETRIC, PERIODIC, DIRICHLET = "symmetric", "periodic", "dirichlet"
EXTEND_OUT, EXTEND_IN = "out", "in"


@dataclass
class Problem:
    """One extension problem: inputs plus the boundary rule and direction (no solution)."""
    phi: np.ndarray            # float32 [ny][nx]
    f: np.ndarray              # float32 [ny][nx]; only values at known nodes matter
    bc_x: str = SYMMETRIC
    bc_y: str = SYMMETRIC
    direction: str = EXTEND_OUT
    hx: float = 1.0
    hy: float = 1.0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.phi.shape[1])

    @property
    def ny(self) -> int:
        return int(self.phi.shape[0])


def axis_nodes(n: int, bc: str, lo: float = -1.0, hi: float = 1.0):
    """Node coordinates and spacing of one axis (cell-centred, or Dirichlet interior nodes)."""
    if bc == DIRICHLET:
        h = (hi - lo) / (n + 1)
        return lo + (np.arange(n) + 1.0) * h, h
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h, h


def grid(nx: int, ny: int, bc_x: str, bc_y: str, lo=-1.0, hi=1.0):
    xs, hx = axis_nodes(nx, bc_x, lo, hi)
    ys, hy = axis_nodes(ny, bc_y, lo, hi)
    X, Y = np.meshgrid(xs, ys)  # [ny][nx]
    return X, Y, hx, hy


def _plane_wave_field(rng, X, Y, modes: int = 8):
    c = rng.standard_normal(modes) / (np.arange(1, modes + 1) ** 2)
    psi = rng.uniform(0.0, 2 * np.pi, modes)
    vth = rng.uniform(0.0, 2 * np.pi, modes)
    f = np.zeros_like(X)
    for k in range(1, modes + 1):
        d = X * math.cos(psi[k - 1]) + Y * math.sin(psi[k - 1])
        f += c[k - 1] * np.cos(np.pi * k * d + vth[k - 1])
    return f


def circle(n: int = 64, bc: str = SYMMETRIC, direction: str = EXTEND_OUT) -> Problem:
    """phi = r - 0.5, f = cos(2x) sin(3y) + 0.5 x (deterministic; the small FP64 case)."""
    X, Y, hx, hy = grid(n, n, bc, bc)
    phi = np.sqrt(X * X + Y * Y) - 0.5
    f = np.cos(2 * X) * np.sin(3 * Y) + 0.5 * X
    return Problem(phi.astype(np.float32), f.astype(np.float32), bc, bc, direction, hx, hy,
                   name=f"circle{n}")


def star(n: int = 1024, bc: str = PERIODIC, direction: str = EXTEND_IN, amp: float = 0.15,
         lobes: int = 6, radius: float = 0.5) -> Problem:
    """phi = r - radius (1 + amp cos(lobes theta)), f = exp(-r^2)(1 + 0.3 sin 4x)."""
    X, Y, hx, hy = grid(n, n, bc, bc)
    r = np.sqrt(X * X + Y * Y)
    th = np.arctan2(Y, X)
    phi = r - radius * (1.0 + amp * np.cos(lobes * th))
    f = np.exp(-(X * X + Y * Y)) * (1.0 + 0.3 * np.sin(4 * X))
    return Problem(phi.astype(np.float32), f.astype(np.float32), bc, bc, direction, hx, hy,
                   name=f"star{n}")


def wobbly(n: int, index: int = 0, seed: int = BASE_SEED, bc: str = SYMMETRIC,
           direction: str = EXTEND_OUT) -> Problem:
    rng = np.random.default_rng(seed + index)
    a = rng.uniform(0.0, 0.05, 5)
    b = rng.uniform(0.0, 2 * np.pi, 5)
    X, Y, hx, hy = grid(n, n, bc, bc)
    r = np.sqrt(X * X + Y * Y)
    th = np.arctan2(Y, X)
    R = np.ones_like(r)
    for k in range(2, 7):
        R += a[k - 2] * np.cos(k * th + b[k - 2])
    phi = r - 0.4 * R
    f = _plane_wave_field(rng, X, Y)
    return Problem(phi.astype(np.float32), f.astype(np.float32), bc, bc, direction, hx, hy,
                   name=f"wobbly{n}#{index}")


def circles(n: int, index: int = 0, seed: int = BASE_SEED, bc: str = SYMMETRIC,
            direction: str = EXTEND_IN, count: int = 3) -> Problem:
    rng = np.random.default_rng(seed + index)
    c = rng.uniform(-0.5, 0.5, (count, 2))
    rho = rng.uniform(0.2, 0.35, count)
    X, Y, hx, hy = grid(n, n, bc, bc)
    phi = np.full_like(X, np.inf)
    for i in range(count):
        phi = np.minimum(phi, np.sqrt((X - c[i, 0]) ** 2 + (Y - c[i, 1]) ** 2) - rho[i])
    f = _plane_wave_field(rng, X, Y)
    return Problem(phi.astype(np.float32), f.astype(np.float32), bc, bc, direction, hx, hy,
                   name=f"circles{n}#{index}")


# ------------------------------------------------------------------------------------------------
# The five workloads
# ------------------------------------------------------------------------------------------------
def single_fp64_case() -> Problem:
    """64x64 circle, field known inside, extend out, symmetric edges."""
    return circle(64, SYMMETRIC, EXTEND_OUT)


def single_star_case(n: int = 1024) -> Problem:
    """1024x1024 six-lobed star, field known outside, extend in, periodic edges."""
    return star(n, PERIODIC, EXTEND_IN)


BATCH_SIDES = (128, 192, 256, 384, 512)


def batch_sides(count: int = 256, seed: int = BASE_SEED):
    rng = np.random.default_rng(seed)
    return [int(s) for s in rng.choice(BATCH_SIDES, size=count)]


def batch_case(count: int = 256, seed: int = BASE_SEED, sides=None):
    """Uneven batch: sides drawn uniformly from {128, 192, 256, 384, 512}, wobbly interfaces."""
    sides = batch_sides(count, seed) if sides is None else list(sides)
    return [wobbly(s, i, seed) for i, s in enumerate(sides)]


def large_circles_case(n: int = 4096, seed: int = BASE_SEED) -> Problem:
    """4096x4096, three merged circles, field known outside, extend in, symmetric edges."""
    return circles(n, 0, seed + 3000, SYMMETRIC, EXTEND_IN)


@dataclass
class Request:
    arrival_s: float
    problem: Problem


def serving_stream(count: int = 10000, rate: float = 500.0, seed: int = BASE_SEED,
                   side_lo: int = 64, side_hi: int = 2048, build=True):
    """Poisson arrivals of extension requests with log-uniform sides in [side_lo, side_hi].

    Each request: star (amplitude U(0.1, 0.2), 3..8 lobes) or 1..3 circles (50/50), extend in or
    out (50/50), symmetric or periodic edges on both axes (50/50).  With ``build=False`` only the
    request descriptors are returned (no grids), for sizing.
    """
    rng = np.random.default_rng(seed + 7000)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    reqs = []
    for i in range(count):
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        kind = "star" if rng.random() < 0.5 else "circles"
        direction = EXTEND_IN if rng.random() < 0.5 else EXTEND_OUT
        bc = SYMMETRIC if rng.random() < 0.5 else PERIODIC
        amp = float(rng.uniform(0.1, 0.2))
        lobes = int(rng.integers(3, 9))
        ncirc = int(rng.integers(1, 4))
        desc = dict(side=side, kind=kind, direction=direction, bc=bc, amp=amp, lobes=lobes,
                    circles=ncirc, index=i)
        if not build:
            reqs.append((float(t[i]), desc))
            continue
        if kind == "star":
            p = star(side, bc, direction, amp=amp, lobes=lobes)
            sub = np.random.default_rng(seed + 20000 + i)
            X, Y, _, _ = grid(side, side, bc, bc)
            p.f = _plane_wave_field(sub, X, Y).astype(np.float32)
        else:
            p = circles(side, i, seed + 20000, bc, direction, count=ncirc)
        p.meta.update(desc)
        reqs.append(Request(float(t[i]), p))
    return reqs
