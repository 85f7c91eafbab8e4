"""Pins of the exact radial potentials (section 6) that the oracle is checked
against: independent of the oracle's code and of the closed forms' own
derivation, they check that each is a solution of Poisson's equation with the
Green's-function behaviour at infinity."""
import numpy as np
import pytest
from scipy import integrate

from oracle import closed_form


def _radial_laplacian(f, r, d, dr=1e-4):
    # f'' + (d - 1)/r f', central differences (error O(dr^2))
    fp, f0, fm = f(r + dr), f(r), f(r - dr)
    return (fp - 2 * f0 + fm) / dr ** 2 + (d - 1) / r * (fp - fm) / (2 * dr)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("eps,p", [(0.7, 10), (0.4, 3), (0.55, 8)])
def test_closed_form_solves_poisson(d, eps, p):
    pot = closed_form.bump_potential_2d if d == 2 else closed_form.bump_potential_3d
    f = lambda r: pot(np.asarray(r, dtype=np.float64), eps, p)
    rho = lambda r: np.where(r < eps, np.clip(1 - r ** 2 / eps ** 2, 0, None) ** p, 0.0)
    r = np.linspace(0.05, 3.0, 301) * eps
    r = r[np.abs(r - eps) > 2e-3]             # away from the kink of rho's p-th derivative
    lap = _radial_laplacian(f, r, d)
    assert np.abs(lap - rho(r)).max() < 1e-5
    # no jump at the edge of the support (a wrong constant in either branch would
    # show as one of order 1e-3; the slope alone moves phi by ~1e-10 here)
    assert abs(f(eps * (1 - 1e-9)) - f(eps * (1 + 1e-9))) < 1e-9
    # the far field of the total charge Q (by independent quadrature)
    if d == 2:
        Q = 2 * np.pi * integrate.quad(lambda s: s * (1 - s ** 2 / eps ** 2) ** p, 0, eps, epsabs=1e-14)[0]
        far = np.array([2.0, 5.0, 40.0]) * eps
        assert np.allclose(f(far), Q / (2 * np.pi) * np.log(far), rtol=0, atol=1e-13)
    else:
        Q = 4 * np.pi * integrate.quad(lambda s: s * s * (1 - s ** 2 / eps ** 2) ** p, 0, eps, epsabs=1e-14)[0]
        far = np.array([1.5, 4.0, 30.0]) * eps
        assert np.allclose(f(far), -Q / (4 * np.pi * far), rtol=1e-13, atol=0)
    assert abs(closed_form.bump_total_charge(eps, p, d) - Q) < 1e-13 * Q


@pytest.mark.parametrize("c,eps,p", [(0.1, 0.6, 10), (-0.3, 0.25, 4)])
def test_closed_form_1d_solves_poisson(c, eps, p):
    # phi'' = rho, and phi = (Q/2)|x - c| outside the support (G = |x|/2)
    from tests.test_oracle_full import _bump_potential_1d
    f = lambda x: _bump_potential_1d(np.atleast_1d(x), c, eps, p)
    x = c + np.linspace(-2.0, 2.0, 201) * eps
    x = x[np.abs(np.abs(x - c) - eps) > 2e-3]
    dx = 1e-4
    lap = (f(x + dx) - 2 * f(x) + f(x - dx)) / dx ** 2
    rho = np.where(np.abs(x - c) < eps, np.clip(1 - (x - c) ** 2 / eps ** 2, 0, None) ** p, 0.0)
    assert np.abs(lap - rho).max() < 1e-5
    Q = integrate.quad(lambda s: (1 - s ** 2 / eps ** 2) ** p, -eps, eps, epsabs=1e-14)[0]
    far = c + np.array([-3.0, -1.5, 1.2, 4.0]) * eps
    assert np.allclose(f(far), 0.5 * Q * np.abs(far - c), rtol=1e-12, atol=0)
