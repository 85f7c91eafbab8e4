"""The method with fast transforms on the CPU: a timing baseline, not a checker.

TEST INFRASTRUCTURE ONLY (like the rest of this package): ``bench.py`` times it
beside the oracle as the CPU form of the method closest to the paper's own
implementation, which used FFTW on a multicore CPU (section 6).  It computes
exactly the oracle's discrete result (tests/test_oracle_fft_baseline.py holds
it to the oracle at 1e-12), with scipy's multithreaded FFTs in place of the
oracle's direct sums:

  * phi* and the two solves with L4_0: scipy.fft.dstn(type=1), whose output is
    twice the sine sum of section 3 (y_k = 2 sum_i x_i sin(pi k i / M));
  * g: the convolution rearrangement of section 4 (eqs. Trap2D,
    Trap2Dconvolution, convolution), each (d-1)-dimensional aperiodic
    convolution as a zero-padded cyclic one of length 2 M_b per axis, by
    scipy.fft.rfftn / irfftn;
  * gtilde, R and its cubic extrapolation: the oracle's stencils (section 5).
"""
import os

import numpy as np
import scipy.fft as sfft

from . import harmonic
from .dst import continuum_eigenvalues
from .greens import green


def _sine_sums(a: np.ndarray, workers: int) -> np.ndarray:
    """sum_i a_i prod_s sin(pi k_s i_s / M_s) along every axis (section 3)."""
    return sfft.dstn(a, type=1, workers=workers) / float(2 ** a.ndim)


def _forward(interior: np.ndarray, workers: int) -> np.ndarray:
    """beta = prod_s (2/M_s) times the sine sums (section 3, eq. for beta)."""
    scale = 1.0
    for n in interior.shape:
        scale *= 2.0 / (n + 1)
    return scale * _sine_sums(interior, workers)


def phi_star(rho: np.ndarray, h, workers: int) -> np.ndarray:
    """Delta phi* = rho, phi* = 0 on the boundary (section 3)."""
    M = [n - 1 for n in rho.shape]
    inner = tuple(slice(1, n - 1) for n in rho.shape)
    alpha = _forward(rho[inner], workers) / continuum_eigenvalues(M, h)
    out = np.zeros(rho.shape)
    out[inner] = _sine_sums(alpha, workers)
    return out


def solve_L4_0(rhs: np.ndarray, h, workers: int) -> np.ndarray:
    """L4_0 u = rhs with zero Dirichlet data, by sine transforms (section 5)."""
    M = [n + 1 for n in rhs.shape]
    return _sine_sums(_forward(rhs, workers) / harmonic.lambda4(M, h), workers)


def boundary_values(rho: np.ndarray, h, workers: int, chunk: int = 16) -> np.ndarray:
    """g on the boundary nodes (0 inside) by the convolution form of section 4:
    for the faces of axis a, g = h_a sum_p (K_p * rho_p) over the slices p, with
    K_p = G(sqrt(dist_p^2 + |.|^2)) and dist_p = p h_a (face 0), (M_a - p) h_a
    (face M_a).  The face nodes shared by several axes take the last axis's."""
    d = rho.ndim
    n = rho.shape
    M = [k - 1 for k in n]
    out = np.zeros(n)
    for a in range(d):
        others = [b for b in range(d) if b != a]
        r = np.moveaxis(rho, a, 0)[1:M[a]]
        shape2 = tuple(2 * M[b] for b in others)
        pad = np.zeros((M[a] - 1,) + shape2)
        inner = tuple(slice(1, n[b] - 1) for b in others)
        pad[(slice(None),) + inner] = r[(slice(None),) + inner]
        axes = tuple(range(1, d))
        R = sfft.rfftn(pad, axes=axes, workers=workers)
        off2 = 0.0
        for j, b in enumerate(others):
            t = np.arange(2 * M[b])
            o = np.minimum(t, 2 * M[b] - t) * h[b]
            sh = [1] * (d - 1)
            sh[j] = 2 * M[b]
            off2 = off2 + (o ** 2).reshape(sh)
        acc = [0.0, 0.0]
        for p0 in range(1, M[a], chunk):
            ps = np.arange(p0, min(M[a], p0 + chunk))
            for side, dist in enumerate((ps * h[a], (M[a] - ps) * h[a])):
                K = sfft.rfftn(green(np.sqrt(dist.reshape((-1,) + (1,) * (d - 1)) ** 2 + off2), d),
                               axes=axes, workers=workers)
                acc[side] = acc[side] + (R[ps - 1] * K).sum(axis=0)
        keep = tuple(slice(0, n[b]) for b in others)
        face = np.moveaxis(out, a, 0)
        scale = float(np.prod(h))
        for side in range(2):
            w = sfft.irfftn(acc[side], s=shape2, axes=tuple(range(d - 1)), workers=workers)
            face[0 if side == 0 else M[a]] = w[keep] * scale
    return out


def solve(rho: np.ndarray, h, order: int = 6, workers: int = None) -> np.ndarray:
    """phi = phi* + phi_H on every node (section 2), d = 2 or 3."""
    workers = workers or os.cpu_count()
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    h = tuple(float(v) for v in h)
    ps = phi_star(rho, h, workers)
    g = boundary_values(rho, h, workers)
    inner = tuple(slice(1, k - 1) for k in rho.shape)
    u = g.copy()
    u[inner] = solve_L4_0(harmonic.gtilde(g, h), h, workers)
    if order == 6:
        u[inner] = u[inner] + solve_L4_0(harmonic.rhs6(u, h), h, workers)
    return ps + u
