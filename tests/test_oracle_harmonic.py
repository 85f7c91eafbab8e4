"""Pins for the oracle's harmonic correction (section 5)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import harmonic


def _grid(n, box):
    coords = [np.linspace(lo, hi, k) for (lo, hi), k in zip(box, n)]
    h = tuple(c[1] - c[0] for c in coords)
    return np.meshgrid(*coords, indexing="ij"), h


HARMONIC_2D = [lambda x, y: x * x - y * y, lambda x, y: x * y,
               lambda x, y: x ** 3 - 3 * x * y * y,
               lambda x, y: x ** 4 - 6 * x * x * y * y + y ** 4,
               lambda x, y: x ** 5 - 10 * x ** 3 * y * y + 5 * x * y ** 4]
HARMONIC_3D = [lambda x, y, z: x * y * z, lambda x, y, z: x * x + y * y - 2 * z * z,
               lambda x, y, z: x ** 3 - 3 * x * z * z + y,
               lambda x, y, z: (x ** 4 - 6 * x * x * y * y + y ** 4) * 1.0 + z,
               lambda x, y, z: x * y * z * (x * x - y * y)]


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("f", HARMONIC_2D)
def test_harmonic_polynomials_reproduced_2d(f, order):
    # L4 u = 0 exactly for harmonic polynomials of degree <= 5, and then R(u) = 0
    (X, Y), h = _grid((13, 17), ((-0.5, 0.7), (0.1, 1.4)))
    u = f(X, Y)
    uh = harmonic.harmonic_correction(u, h, order)
    np.testing.assert_allclose(uh, u, atol=1e-11 * max(1.0, np.abs(u).max()))


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("f", HARMONIC_3D)
def test_harmonic_polynomials_reproduced_3d(f, order):
    (X, Y, Z), h = _grid((9, 11, 13), ((-0.5, 0.7), (0.1, 1.4), (-1.0, 0.2)))
    u = f(X, Y, Z)
    uh = harmonic.harmonic_correction(u, h, order)
    np.testing.assert_allclose(uh, u, atol=1e-11 * max(1.0, np.abs(u).max()))


def _rates(make, sizes, order):
    errs = []
    for n in sizes:
        u, h = make(n)
        uh = harmonic.harmonic_correction(u, h, order)
        errs.append(np.abs(uh - u).max() / np.abs(u).max())
    return [np.log2(a / b) for a, b in zip(errs, errs[1:])]


def _exp_sin_2d(n):
    (X, Y), h = _grid((n, int(1.5 * (n - 1)) + 1), ((0.0, 1.0), (0.0, 1.3)))
    return np.exp(np.pi * X) * np.sin(np.pi * Y), h


def _exp_sin_3d(n):
    (X, Y, Z), h = _grid((n, int(1.5 * (n - 1)) + 1, n), ((0.0, 1.0), (0.0, 1.3), (0.0, 0.8)))
    return np.exp(np.hypot(1 / 1.3, 1 / 0.8) * np.pi * X) * np.sin(np.pi * Y / 1.3) * np.sin(np.pi * Z / 0.8), h


@pytest.mark.parametrize("make,sizes", [(_exp_sin_2d, (17, 33, 65)), (_exp_sin_3d, (9, 17, 33))])
def test_convergence_rates_4_and_6(make, sizes):
    # anisotropic h so that the 4th-order scheme is not accidentally 6th order
    r4 = _rates(make, sizes, 4)
    r6 = _rates(make, sizes, 6)
    assert abs(r4[-1] - 4.0) < 0.3, r4
    assert abs(r6[-1] - 6.0) < 0.5, r6


def _second_difference_matrix(M, h):
    n = M - 1
    return sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / h ** 2


def test_L4_0_sine_solve_matches_sparse_direct_solve():
    # L4_0 assembled from 1-D tridiagonal matrices with Kronecker products
    M = (7, 9, 6)
    h = (0.13, 0.1, 0.21)
    D = [_second_difference_matrix(m, hh) for m, hh in zip(M, h)]
    I = [sp.identity(m - 1) for m in M]

    def lift(ops):
        out = ops[0]
        for o in ops[1:]:
            out = sp.kron(out, o)
        return out
    A = 0
    for s in range(3):
        ops = list(I)
        ops[s] = D[s]
        A = A + lift(ops)
    for s in range(3):
        for r in range(s + 1, 3):
            ops = list(I)
            ops[s] = D[s]
            ops[r] = D[r]
            A = A + (h[s] ** 2 + h[r] ** 2) / 12 * lift(ops)
    b = np.random.default_rng(0).standard_normal(tuple(m - 1 for m in M))
    ref = spla.spsolve(A.tocsc(), b.ravel()).reshape(b.shape)
    np.testing.assert_allclose(harmonic.solve_L4_0(b, h), ref, atol=1e-12 * np.abs(ref).max())


def test_rhs6_coefficients_on_a_monomial():
    # u = x^4 y^2: D2x D2x D2y u = 48 exactly and D2y D2y D2x u = 0,
    # so R = 48 (hx^4/240 + hx^2 hy^2/144) on the core
    (X, Y), h = _grid((11, 13), ((0.0, 1.0), (0.0, 0.6)))
    R = harmonic.rhs6_core(X ** 4 * Y ** 2, h)
    c = h[0] ** 4 / 240 + h[0] ** 2 * h[1] ** 2 / 144
    np.testing.assert_allclose(R, 48 * c, rtol=1e-8)
    assert R.shape == (11 - 4, 13 - 4)


def test_cubic_extrapolation_exact_for_cubics():
    i = np.arange(1, 12)
    j = np.arange(1, 10)
    I, J = np.meshgrid(i, j, indexing="ij")
    full = (I ** 3 - 2.0 * I + 1) * (0.5 * J ** 3 + J ** 2)
    core = full[1:-1, 1:-1]
    np.testing.assert_allclose(harmonic.extrapolate_cubic(core), full, rtol=1e-12)


def test_gtilde_lives_on_the_shell():
    g = np.random.default_rng(1).standard_normal((8, 9, 10))
    gt = harmonic.gtilde(g, (0.1, 0.2, 0.3))
    assert np.all(gt[1:-1, 1:-1, 1:-1] == 0.0)
    assert np.abs(gt[0]).max() > 0
