"""Discrete sine transforms and the spectral Dirichlet solve (section 3).

Notation: axis s has M_s panels, mesh width h_s, length L_s = M_s h_s; the
interior nodes are i_s = 1..M_s-1 and the sine modes k_s = 1..M_s-1.
"""
import numpy as np


def sine_matrix(M: int) -> np.ndarray:
    """S[k-1, i-1] = sin(pi k i / M) for k, i = 1..M-1.

    The integer product k*i is reduced modulo 2M before the sine is taken,
    so every entry is sin(pi m / M) with 0 <= m < 2M.
    """
    k = np.arange(1, M, dtype=np.int64)
    m = np.outer(k, k) % (2 * M)
    return np.sin(np.pi * m.astype(np.float64) / M)


def sine_transform(a: np.ndarray) -> np.ndarray:
    """Apply the unnormalised sine sum along every axis of an interior array.

    Along axis s of length M_s - 1 this computes
    b_k = sum_{i=1}^{M_s-1} a_i sin(pi k i / M_s)  (the sums of eqs.
    rhoSinSeries / phiStarSoln2D), one axis after the other.
    """
    out = np.asarray(a, dtype=np.float64)
    for s in range(out.ndim):
        S = sine_matrix(out.shape[s] + 1)
        out = np.moveaxis(np.tensordot(S, np.moveaxis(out, s, 0), axes=(1, 0)), 0, s)
    return np.ascontiguousarray(out)


def forward_coefficients(interior: np.ndarray) -> np.ndarray:
    """beta_k = prod_s (2/L_s) h_s * sum_i f_i prod_s sin(pi k_s i_s / M_s).

    Section 3, eq. for beta: the factor (2/L_s) h_s equals 2/M_s.
    """
    scale = 1.0
    for n in interior.shape:
        scale *= 2.0 / (n + 1)
    return scale * sine_transform(interior)


def continuum_eigenvalues(M, h) -> np.ndarray:
    """-(pi^2) sum_s k_s^2 / L_s^2 on the mode grid (section 3, eq. for alpha)."""
    d = len(M)
    lam = 0.0
    for s in range(d):
        L = M[s] * h[s]
        k = np.arange(1, M[s], dtype=np.float64)
        shape = [1] * d
        shape[s] = M[s] - 1
        lam = lam + (-(np.pi ** 2) * k ** 2 / L ** 2).reshape(shape)
    return lam


def discrete_eigenvalues_1d(M: int, h: float) -> np.ndarray:
    """Eigenvalues of D^2 with zero Dirichlet data on the sine modes k = 1..M-1.

    D^2 sin(pi k i/M) = (2cos(pi k/M) - 2)/h^2 sin(pi k i/M)
                      = -(4/h^2) sin^2(pi k/(2M)) sin(pi k i/M)   (section 5).
    """
    k = np.arange(1, M, dtype=np.float64)
    return -(4.0 / h ** 2) * np.sin(np.pi * k / (2.0 * M)) ** 2


def phi_star(rho: np.ndarray, h) -> np.ndarray:
    """phi* on all nodes: Delta phi* = rho, phi* = 0 on the boundary (section 3).

    beta from the forward sums, alpha = beta / lambda_continuum (the eq. for
    alpha: alpha = -beta (sum k^2 pi^2 / L^2)^-1), phi* = sum alpha * sines
    (eq. phiStarSoln2D).  Boundary values of rho are not used.
    """
    d = rho.ndim
    M = [n - 1 for n in rho.shape]
    inner = tuple(slice(1, n - 1) for n in rho.shape)
    beta = forward_coefficients(rho[inner])
    alpha = beta / continuum_eigenvalues(M, h)
    out = np.zeros_like(rho, dtype=np.float64)
    out[inner] = sine_transform(alpha)
    return out
