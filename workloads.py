"""Seeded synthetic inputs for the infinite-domain Poisson solver.

This module holds only the problem definitions (grid sizes, mesh widths,
domain boxes) and the density generators.  It contains none of the solver's
arithmetic, so both the CPU oracle and the CUDA path may use it.

Array convention: a d-dimensional node array has shape ``n = (n_0, ..., n_{d-1})``
in C order (last axis contiguous); axis s has ``M_s = n_s - 1`` panels of
width ``h_s`` and nodes ``lo_s + i * h_s``, ``i = 0..M_s`` (section 3).  The
paper's coordinates (x, y, z) map to array axes (0, 1, 2).

Densities:
  * ``bump``: the un-normalised radial polynomial ``(1 - |x - c|^2/eps^2)^p``
    for ``|x - c| < eps`` (the test family of section 6, eq. Bepsilon, without
    the unit-integral factor; the method is linear so the factor is immaterial).
  * ``gauss_sum``: a seeded sum of Gaussians multiplied by a C-infinity taper
    that vanishes within 0.15 of every box edge (a smooth, mixed-sign density
    whose support keeps the distance from the boundary the method assumes,
    section 2).
  * ``points``: seeded random values on a few scattered interior nodes, zero
    elsewhere (most lines and slices of the array are then exactly zero, some
    are not: the case the solver's zero-line and zero-slice skipping must
    get right).
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np

# ----------------------------------------------------------------------------
# problem description


@dataclasses.dataclass(frozen=True)
class Problem:
    """One solve: node counts, box and the density recipe."""

    name: str
    n: tuple            # node counts per array axis (includes boundary nodes)
    lo: tuple           # lower box corner per axis
    hi: tuple           # upper box corner per axis
    density: str        # "bump", "gauss", "random" or "points"
    params: dict        # density parameters

    @property
    def d(self) -> int:
        return len(self.n)

    @property
    def M(self) -> tuple:
        return tuple(k - 1 for k in self.n)

    @property
    def h(self) -> tuple:
        return tuple((b - a) / (k - 1) for a, b, k in zip(self.lo, self.hi, self.n))

    @property
    def points(self) -> int:
        return int(np.prod(self.n))

    def coords(self) -> list:
        return [self.lo[s] + np.arange(self.n[s], dtype=np.float64) * self.h[s]
                for s in range(self.d)]

    def rho(self) -> np.ndarray:
        """FP64 density on every node, C order.  Boundary nodes are zero."""
        if self.density == "bump":
            r = bump(self.coords(), **self.params)
        elif self.density == "gauss":
            r = gauss_sum(self.coords(), self.lo, self.hi, **self.params)
        elif self.density == "random":
            r = random_interior(self.n, **self.params)
        elif self.density == "points":
            r = point_sources(self.n, **self.params)
        else:
            raise ValueError(self.density)
        return np.ascontiguousarray(r, dtype=np.float64)


# ----------------------------------------------------------------------------
# density generators


def _radius2(coords: Sequence[np.ndarray], centre: Sequence[float]) -> np.ndarray:
    d = len(coords)
    r2 = None
    for s in range(d):
        shape = [1] * d
        shape[s] = coords[s].size
        t = (coords[s] - centre[s]).reshape(shape) ** 2
        r2 = t if r2 is None else r2 + t
    return r2


def bump(coords, centre, eps, p):
    """(1 - r^2/eps^2)^p for r < eps, 0 elsewhere; r = |x - centre|."""
    u = _radius2(coords, centre) / (eps * eps)
    out = np.where(u < 1.0, np.clip(1.0 - u, 0.0, None) ** p, 0.0)
    return out


def smooth_step(t):
    """C-infinity step: 0 for t <= 0, 1 for t >= 1."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    inside = (t > 0) & (t < 1)
    ti = t[inside]
    a = np.exp(-1.0 / ti)
    b = np.exp(-1.0 / (1.0 - ti))
    out[inside] = a / (a + b)
    out[t >= 1] = 1.0
    return out


def taper(xi):
    """Box-relative taper: 0 for xi <= 0.15 or xi >= 0.85, 1 on [0.3, 0.7]."""
    xi = np.asarray(xi, dtype=np.float64)
    up = smooth_step((xi - 0.15) / 0.15)
    down = smooth_step((0.85 - xi) / 0.15)
    return np.minimum(up, down)


def gauss_params(seed: int, count: int = 6, d: int = 3):
    """Seeded Gaussian-sum parameters (centres box-relative, sigma absolute)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.3, 0.7, size=(count, d))
    sigma = rng.uniform(0.04, 0.1, size=count)
    amp = rng.uniform(-1.0, 1.0, size=count)
    return centres, sigma, amp


def gauss_sum(coords, lo, hi, seed, count=6):
    d = len(coords)
    centres, sigma, amp = gauss_params(seed, count, d)
    out = 0.0
    for j in range(count):
        c = [lo[s] + centres[j, s] * (hi[s] - lo[s]) for s in range(d)]
        r2 = _radius2(coords, c)
        out = out + amp[j] * np.exp(-r2 / (2.0 * sigma[j] ** 2))
    tap = None
    for s in range(d):
        shape = [1] * d
        shape[s] = coords[s].size
        xi = (coords[s] - lo[s]) / (hi[s] - lo[s])
        t = taper(xi).reshape(shape)
        tap = t if tap is None else tap * t
    return out * tap


def random_interior(n, seed, margin=0):
    """Uniform random values on interior nodes (zero on the boundary and on
    ``margin`` further layers); used for linear-algebra checks only."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n, dtype=np.float64)
    sl = tuple(slice(1 + margin, k - 1 - margin) for k in n)
    out[sl] = rng.uniform(-1.0, 1.0, size=out[sl].shape)
    return out


def point_sources(n, seed, count):
    """``count`` seeded uniform(-1, 1) values at seeded random interior nodes."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n, dtype=np.float64)
    idx = tuple(rng.integers(1, k - 1, size=count) for k in n)
    out[idx] = rng.uniform(-1.0, 1.0, size=count)
    return out


# ----------------------------------------------------------------------------
# the named workloads

C1_BUMP = dict(centre=(0.1, -0.05), eps=0.8, p=8)
C2_BUMP = dict(centre=(0.05, 0.1, -0.08), eps=0.7, p=10)


def c1_2d(n: int = 65) -> Problem:
    """2-D, 65 x 65 nodes on [-1,1]^2, bump eps=0.8 p=8 centred (0.1,-0.05)."""
    return Problem("2d_bump_%d" % n, (n, n), (-1.0, -1.0), (1.0, 1.0), "bump", C1_BUMP)


def c2_3d(n: int = 129) -> Problem:
    """3-D, n^3 nodes on [-1,1]^3, bump eps=0.7 p=10 centred (0.05,0.1,-0.08)."""
    return Problem("3d_bump_%d" % n, (n, n, n), (-1.0,) * 3, (1.0,) * 3, "bump", C2_BUMP)


def c3_large(n: int = 513) -> Problem:
    """3-D, n^3 nodes on [0,2]x[0,1]x[0,1], six seeded Gaussians (seed 2108)."""
    return Problem("3d_gauss_%d" % n, (n, n, n), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0),
                   "gauss", dict(seed=2108))


def c4_sweep(interior: tuple = (256, 256, 256)) -> Problem:
    """3-D, given interior node counts on [0,1]^3, Gaussian sum (seed 2108)."""
    n = tuple(k + 2 for k in interior)
    return Problem("3d_gauss_int%s" % "x".join(map(str, interior)), n, (0.0,) * 3,
                   (1.0,) * 3, "gauss", dict(seed=2108))


C5_SIZES = (33, 65, 97, 129, 193, 257)


def c5_batch(count: int = 96, seed: int = 21081) -> list:
    """Independent 3-D problems with per-axis node counts drawn from C5_SIZES."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.array(C5_SIZES), size=(count, 3))
    out = []
    for j in range(count):
        n = tuple(int(v) for v in sizes[j])
        out.append(Problem("batch_%d" % j, n, (0.0,) * 3, (1.0,) * 3, "gauss",
                           dict(seed=2108 + j)))
    return out


def scaled_bump(n: Sequence[int], lo=None, hi=None, centre=None, eps=None, p=10) -> Problem:
    """A bump on an arbitrary box (defaults: [-1,1]^d, C2-like parameters)."""
    d = len(n)
    lo = tuple(lo) if lo is not None else (-1.0,) * d
    hi = tuple(hi) if hi is not None else (1.0,) * d
    if centre is None:
        centre = C2_BUMP["centre"][:d] if d == 3 else C1_BUMP["centre"]
    if eps is None:
        eps = 0.7 if d == 3 else 0.8
    return Problem("bump_" + "x".join(map(str, n)), tuple(n), lo, hi, "bump",
                   dict(centre=tuple(centre), eps=eps, p=p))
