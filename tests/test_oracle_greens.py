"""Pins for the oracle's boundary values g (section 4)."""
import math

import numpy as np
import pytest

import workloads as w
from oracle import closed_form, greens


def test_direct_sum_matches_brute_force_python_loop():
    # tiny anisotropic 3-D grid, random interior rho: C sum vs a plain loop
    n = (5, 6, 7)
    h = (0.3, 0.2, 0.25)
    rho = w.random_interior(n, seed=1)
    got = greens.boundary_direct_nodes(rho, h)
    mask = greens.boundary_mask(n)
    for b in np.argwhere(mask):
        s = 0.0
        for p in np.argwhere(rho != 0):
            r = math.sqrt(sum(((b[k] - p[k]) * h[k]) ** 2 for k in range(3)))
            s += -1.0 / (4 * math.pi * r) * rho[tuple(p)]
        assert abs(got[tuple(b)] - s * 0.3 * 0.2 * 0.25) < 1e-14


@pytest.mark.parametrize("n,h", [((9, 12), (0.1, 0.07)), ((7, 9, 11), (0.11, 0.09, 0.05)),
                                 ((17, 17, 17), (0.125,) * 3)])
def test_convolution_form_equals_direct_sum(n, h):
    # the rearrangement of eqs. Trap2D/convolution is an identity: agree to rounding
    rho = w.random_interior(n, seed=7)
    a = greens.boundary_direct_nodes(rho, h)
    b = greens.boundary_convolution(rho, h)
    m = greens.boundary_mask(n)
    assert np.abs(a - b)[m].max() <= 1e-13 * np.abs(a[m]).max()
    assert np.all(b[~m] == 0)


@pytest.mark.parametrize("d,n,tol", [(3, 33, 1e-9), (3, 65, 1e-12), (2, 33, 1e-9), (2, 65, 5e-12)])
def test_direct_sum_converges_to_closed_form(d, n, tol):
    # outside the support the exact potential is (Q/2pi) log r or -Q/(4 pi r);
    # the trapezoid sum of a smooth integrand vanishing at the edge is spectral
    p = w.c2_3d(n) if d == 3 else w.c1_2d(n)
    g = greens.boundary_direct_nodes(p.rho(), p.h)
    ex = closed_form.bump_potential_on_grid(p)
    m = greens.boundary_mask(p.n)
    assert np.abs(g - ex)[m].max() / np.abs(ex[m]).max() < tol


def test_green_function_normalisation():
    # flux of grad G through a sphere (3-D) / circle (2-D) is 1
    r = 0.37
    eps = 1e-6
    dG3 = (greens.green(r + eps, 3) - greens.green(r - eps, 3)) / (2 * eps)
    dG2 = (greens.green(r + eps, 2) - greens.green(r - eps, 2)) / (2 * eps)
    assert abs(4 * math.pi * r * r * dG3 - 1) < 1e-8
    assert abs(2 * math.pi * r * dG2 - 1) < 1e-8
