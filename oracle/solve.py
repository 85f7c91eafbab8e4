"""The full method: phi = phi* + phi_H on every grid node (section 2)."""
import numpy as np

from . import dst, greens, harmonic


def boundary_values(rho: np.ndarray, h, method: str = "direct") -> np.ndarray:
    if method == "direct":
        return greens.boundary_direct_nodes(rho, h)
    if method == "convolution":
        return greens.boundary_convolution(rho, h)
    raise ValueError(method)


def solve(rho: np.ndarray, h, order: int = 6, boundary: str = "direct",
          parts: dict = None) -> np.ndarray:
    """phi on all nodes of the grid for density ``rho`` (node array, C order).

    phi* solves the Dirichlet-0 problem (eq. PhiStarEqn); phi_H is harmonic
    with boundary values g = trapezoid sum of G * rho (eq. PhiHeqn); on the
    boundary phi* = 0, so phi = g there.  d = 1 uses the exact linear
    harmonic function between the two end values (section 5).
    """
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    h = tuple(float(v) for v in h)
    ps = dst.phi_star(rho, h)
    if rho.ndim == 1:
        g = greens.boundary_direct_nodes(rho, h)
        M = rho.shape[0] - 1
        t = np.arange(M + 1) / M
        phi_h = g[0] * (1 - t) + g[M] * t
    else:
        g = boundary_values(rho, h, boundary)
        phi_h = harmonic.harmonic_correction(g, h, order, parts)
    if parts is not None:
        parts["phistar"] = ps
        parts["g"] = g
    return ps + phi_h
