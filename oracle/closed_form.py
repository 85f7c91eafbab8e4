"""Exact potentials of the radial bump densities (section 6, eq. Bepsilon).

For rho = (1 - u)^p with u = r^2/eps^2 inside r < eps (no normalising
factor), phi = G * rho solves Delta phi = rho in R^d with the Green's-function
behaviour at infinity.  Written from the radial form of Poisson's equation
(Newton's theorem for radial densities):

  2-D: r phi'(r) = m(r) = int_0^r s rho(s) ds = eps^2 (1 - (1-u)^{p+1}) / (2(p+1)),
       phi(r) = (Q/2pi) log r for r >= eps, Q = pi eps^2/(p+1),
       phi(r) = (Q/2pi) log eps - eps^2/(4(p+1)) sum_{k=1}^{p+1} (1-u)^k / k inside.
  3-D: r^2 phi'(r) = A(r) = int_0^r rho(s) s^2 ds,
       phi(r) = -A(r)/r - eps^2 (1-u)^{p+1} / (2(p+1)) inside, -A(eps)/r outside.
A(r) is a polynomial integral evaluated with Gauss-Legendre quadrature
exact for its degree (2p + 2).
"""
import numpy as np


def bump_potential_2d(r, eps: float, p: int):
    r = np.asarray(r, dtype=np.float64)
    Q = np.pi * eps ** 2 / (p + 1)
    u = np.minimum(r ** 2 / eps ** 2, 1.0)
    inside = -eps ** 2 / (4.0 * (p + 1)) * sum((1.0 - u) ** k / k for k in range(1, p + 2))
    inside = inside + Q / (2 * np.pi) * np.log(eps)
    with np.errstate(divide="ignore"):
        outside = Q / (2 * np.pi) * np.log(np.maximum(r, eps))
    return np.where(r < eps, inside, outside)


def _A(r, eps: float, p: int):
    """int_0^r (1 - s^2/eps^2)^p s^2 ds for 0 <= r <= eps (vectorised)."""
    x, w = np.polynomial.legendre.leggauss(p + 4)
    r = np.asarray(r, dtype=np.float64)
    s = 0.5 * r[..., None] * (x + 1.0)
    f = (1.0 - s ** 2 / eps ** 2) ** p * s ** 2
    return 0.5 * r * (f * w).sum(axis=-1)


def bump_potential_3d(r, eps: float, p: int):
    # inside the support: -A(r)/r - B(r); outside: -A(eps)/r (the quadrature
    # runs only where r < eps)
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    inner = r < eps
    ro = r[~inner]
    out[~inner] = -float(_A(np.array(eps), eps, p)) / ro
    ri = r[inner]
    A = _A(ri, eps, p)
    u = ri ** 2 / eps ** 2
    B = eps ** 2 * (1.0 - u) ** (p + 1) / (2.0 * (p + 1))
    out[inner] = np.where(ri > 0, -A / np.where(ri > 0, ri, 1.0), 0.0) - B
    return out


def bump_total_charge(eps: float, p: int, d: int) -> float:
    """Integral of (1 - r^2/eps^2)^p over R^d."""
    if d == 2:
        return np.pi * eps ** 2 / (p + 1)
    if d == 3:
        return 4.0 * np.pi * float(_A(np.array(eps), eps, p))
    raise ValueError(d)


def bump_potential_on_grid(problem) -> np.ndarray:
    """Exact phi on every node for a workloads.Problem with a bump density."""
    prm = problem.params
    coords = problem.coords()
    d = problem.d
    r2 = 0.0
    for s in range(d):
        shape = [1] * d
        shape[s] = coords[s].size
        r2 = r2 + ((coords[s] - prm["centre"][s]) ** 2).reshape(shape)
    r = np.sqrt(r2)
    if d == 2:
        return bump_potential_2d(r, prm["eps"], prm["p"])
    return bump_potential_3d(r, prm["eps"], prm["p"])
