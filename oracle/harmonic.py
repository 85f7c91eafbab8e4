"""4th- and 6th-order harmonic correction (section 5).

The harmonic part u satisfies Delta u = 0 in Omega, u = g on the boundary
(eq. harmonicEQ).  Operators on node arrays (all nodes, boundary included):

  D2_s u      = (u[i+e_s] - 2 u[i] + u[i-e_s]) / h_s^2        (3-point stencil)
  L4          = sum_s D2_s + sum_{s<r} (h_s^2 + h_r^2)/12 D2_s D2_r
                (eqs. harmonic4thOrder2D / harmonic4thOrder3D, grouped per pair)
  R(u)        = sum_{s != r} (h_s^4/240 + h_s^2 h_r^2/144) D2_s D2_s D2_r u
                (right-hand sides of eqs. 6thOrderRelation2D / 6thOrderRelation3D)

Steps: gtilde = -L4(g extended by zero) on interior nodes (eq.
harmonic4thOrderNH2D: the boundary contributions moved to the right-hand side);
u1 solves L4_0 u1 = gtilde with discrete sine transforms (the sines are the
eigenvectors of L4_0); for order 6, R(u1) is evaluated where its width-2
stencil fits, extended to the layers next to the boundary by cubic
extrapolation, and u2 = u1 + L4_0^{-1} R.
"""
import numpy as np

from .dst import discrete_eigenvalues_1d, forward_coefficients, sine_transform


def d2(u: np.ndarray, axis: int, h: float) -> np.ndarray:
    """Second difference along ``axis``; the result loses one node at each end."""
    n = u.shape[axis]
    lo = [slice(None)] * u.ndim
    mid = [slice(None)] * u.ndim
    hi = [slice(None)] * u.ndim
    lo[axis] = slice(0, n - 2)
    mid[axis] = slice(1, n - 1)
    hi[axis] = slice(2, n)
    return (u[tuple(hi)] - 2.0 * u[tuple(mid)] + u[tuple(lo)]) / (h * h)


def _trim(a: np.ndarray, full_shape, keep_axes, target_lo: int):
    """Slice ``a`` so that every axis covers nodes target_lo..M-target_lo.

    ``keep_axes[s]`` is how many nodes axis s of ``a`` already lost per end."""
    sl = []
    for s, n in enumerate(full_shape):
        lost = keep_axes[s]
        start = target_lo - lost
        stop = (n - target_lo) - lost
        sl.append(slice(start, stop))
    return a[tuple(sl)]


def apply_L4(u: np.ndarray, h) -> np.ndarray:
    """L4 u on the interior nodes (1..M_s-1 on every axis)."""
    d = u.ndim
    out = 0.0
    for s in range(d):
        lost = [0] * d
        lost[s] = 1
        out = out + _trim(d2(u, s, h[s]), u.shape, lost, 1)
    for s in range(d):
        for r in range(s + 1, d):
            lost = [0] * d
            lost[s] = lost[r] = 1
            c = (h[s] ** 2 + h[r] ** 2) / 12.0
            out = out + c * _trim(d2(d2(u, r, h[r]), s, h[s]), u.shape, lost, 1)
    return out


def gtilde(g: np.ndarray, h) -> np.ndarray:
    """Right-hand side of L4_0 u = gtilde on interior nodes (eq. harmonic4thOrderNH2D).

    ``g`` is a node array whose boundary entries hold the Dirichlet data; its
    interior entries are ignored (treated as zero)."""
    gb = np.array(g, dtype=np.float64, copy=True)
    gb[tuple(slice(1, n - 1) for n in g.shape)] = 0.0
    return -apply_L4(gb, h)


def lambda4(M, h) -> np.ndarray:
    """Eigenvalues of L4_0 on the mode grid:
    Lambda4 = sum_s lam_s + sum_{s<r} (h_s^2 + h_r^2)/12 lam_s lam_r."""
    d = len(M)
    lam = []
    for s in range(d):
        shape = [1] * d
        shape[s] = M[s] - 1
        lam.append(discrete_eigenvalues_1d(M[s], h[s]).reshape(shape))
    out = 0.0
    for s in range(d):
        out = out + lam[s]
    for s in range(d):
        for r in range(s + 1, d):
            out = out + (h[s] ** 2 + h[r] ** 2) / 12.0 * lam[s] * lam[r]
    return out


def solve_L4_0(rhs: np.ndarray, h) -> np.ndarray:
    """u on interior nodes with L4_0 u = rhs (zero Dirichlet data), by sine
    transform, division by Lambda4, inverse sine transform (section 5)."""
    M = [n + 1 for n in rhs.shape]
    return sine_transform(forward_coefficients(rhs) / lambda4(M, h))


def rhs6_core(u: np.ndarray, h) -> np.ndarray:
    """R(u) on the nodes whose indices all lie in 2..M_s-2 (the width-2 stencil fits).

    R = sum over ordered pairs s != r of (h_s^4/240 + h_s^2 h_r^2/144) D2_s D2_s D2_r u
    (eqs. 6thOrderRelation2D / 6thOrderRelation3D, the six 3-D terms summed)."""
    d = u.ndim
    out = 0.0
    for s in range(d):
        for r in range(d):
            if r == s:
                continue
            c = h[s] ** 4 / 240.0 + h[s] ** 2 * h[r] ** 2 / 144.0
            t = d2(d2(d2(u, r, h[r]), s, h[s]), s, h[s])
            lost = [0] * d
            lost[s] = 2
            lost[r] = 1
            out = out + c * _trim(t, u.shape, lost, 2)
    return out


def extrapolate_cubic(core: np.ndarray) -> np.ndarray:
    """Extend R from nodes 2..M-2 to nodes 1..M-1 on every axis.

    The value next to the boundary comes from the cubic through the four
    nearest core values (R_1 = 4R_2 - 6R_3 + 4R_4 - R_5, mirrored at the far
    end), applied axis by axis over the extent already filled."""
    out = np.asarray(core, dtype=np.float64)
    for s in range(out.ndim):
        a = np.moveaxis(out, s, 0)
        first = 4 * a[0] - 6 * a[1] + 4 * a[2] - a[3]
        last = 4 * a[-1] - 6 * a[-2] + 4 * a[-3] - a[-4]
        a = np.concatenate([first[None], a, last[None]], axis=0)
        out = np.moveaxis(a, 0, s)
    return np.ascontiguousarray(out)


def rhs6(u: np.ndarray, h) -> np.ndarray:
    """R on all interior nodes: core values plus cubic extrapolation."""
    return extrapolate_cubic(rhs6_core(u, h))


def harmonic_correction(g: np.ndarray, h, order: int, parts: dict = None) -> np.ndarray:
    """phi_H on all nodes: boundary = g, interior = u1 (order 4) or u2 (order 6)."""
    if order not in (4, 6):
        raise ValueError("order must be 4 or 6")
    inner = tuple(slice(1, n - 1) for n in g.shape)
    gt = gtilde(g, h)
    u = np.array(g, dtype=np.float64, copy=True)
    u[inner] = solve_L4_0(gt, h)
    if parts is not None:
        parts["gtilde"] = gt
        parts["u1"] = u.copy()
    if order == 6:
        R = rhs6(u, h)
        u[inner] = u[inner] + solve_L4_0(R, h)
        if parts is not None:
            parts["R"] = R
    return u
