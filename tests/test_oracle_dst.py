"""Pins for the oracle's sine transforms and phi* solve (section 3)."""
import numpy as np
import pytest
import scipy.fft

from oracle import dst


@pytest.mark.parametrize("M", [2, 3, 5, 8, 9, 16, 33, 64])
def test_sine_matrix_squares_to_scaled_identity(M):
    # S^2 = (M/2) I: the discrete orthogonality that makes (2/M) S the inverse
    S = dst.sine_matrix(M)
    np.testing.assert_allclose(S @ S, (M / 2) * np.eye(M - 1), atol=1e-12 * M)


@pytest.mark.parametrize("n", [1, 7, 31, 100])
def test_sine_sum_is_library_dst1(n):
    # scipy's DST-I is y_k = 2 sum_j x_j sin(pi (j+1)(k+1)/(n+1))
    x = np.random.default_rng(n).standard_normal(n)
    np.testing.assert_allclose(dst.sine_transform(x), scipy.fft.dst(x, type=1) / 2,
                               rtol=0, atol=1e-12 * np.abs(x).sum())


def test_sine_transform_is_separable_library_dstn():
    x = np.random.default_rng(3).standard_normal((6, 9, 4))
    ref = scipy.fft.dstn(x, type=1) / 8
    np.testing.assert_allclose(dst.sine_transform(x), ref, atol=1e-12)


@pytest.mark.parametrize("shape,box,modes", [
    ((17, 21), ((0.0, 1.0), (-0.5, 0.8)), (3, 2)),
    ((9, 12, 15), ((0.0, 1.0), (0.0, 2.0), (-1.0, 1.0)), (1, 4, 5)),
])
def test_phi_star_exact_on_a_sine_mode(shape, box, modes):
    # rho = prod sin(k pi (x-a)/L) is resolved exactly; Delta^-1 of it is
    # rho / (-(pi^2) sum k^2/L^2)  (closed form)
    d = len(shape)
    coords = [np.linspace(lo, hi, n) for (lo, hi), n in zip(box, shape)]
    h = [c[1] - c[0] for c in coords]
    grids = np.meshgrid(*coords, indexing="ij")
    rho = np.ones(shape)
    lam = 0.0
    for s in range(d):
        L = box[s][1] - box[s][0]
        rho = rho * np.sin(modes[s] * np.pi * (grids[s] - box[s][0]) / L)
        lam += (modes[s] * np.pi / L) ** 2
    phi = dst.phi_star(rho, h)
    np.testing.assert_allclose(phi, -rho / lam, atol=1e-13 * np.abs(rho / lam).max())
    # boundary values of phi* are zero
    for s in range(d):
        assert np.all(np.take(phi, 0, axis=s) == 0) and np.all(np.take(phi, -1, axis=s) == 0)


def test_phi_star_converges_spectrally_to_dirichlet_solution():
    # -Delta of a smooth compactly supported bump in a box: compare against a
    # 4x finer solve; error must drop by far more than h^2 when h halves
    import workloads as w
    errs = []
    for n in (17, 33):
        p = w.scaled_bump((n, n), p=8)
        fine = w.scaled_bump((4 * (n - 1) + 1,) * 2, p=8)
        a = dst.phi_star(p.rho(), p.h)
        b = dst.phi_star(fine.rho(), fine.h)[::4, ::4]
        errs.append(np.abs(a - b).max())
    assert errs[1] < errs[0] / 2 ** 5


@pytest.mark.parametrize("M,h", [(8, 0.3), (33, 0.01)])
def test_discrete_eigenvalues_match_second_difference(M, h):
    # D2 sin(pi k i/M) = lambda_k sin(pi k i/M) with zero end values
    i = np.arange(M + 1)
    lam = dst.discrete_eigenvalues_1d(M, h)
    for k in (1, M // 2, M - 1):
        v = np.sin(np.pi * k * i / M)
        v[0] = v[-1] = 0.0
        d2v = (v[2:] - 2 * v[1:-1] + v[:-2]) / h ** 2
        np.testing.assert_allclose(d2v, lam[k - 1] * v[1:-1], atol=1e-9 / h ** 2)
