"""End-to-end pins of the oracle against exact potentials (sections 2 and 6)."""
import os

import numpy as np
import pytest

import workloads as w
from oracle import closed_form, solve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_rates.txt")


@pytest.mark.parametrize("order", [4, 6])
def test_2d_workload_65_matches_exact_potential(order):
    p = w.c1_2d(65)
    phi = solve.solve(p.rho(), p.h, order)
    ex = closed_form.bump_potential_on_grid(p)
    assert np.abs(phi - ex).max() / np.abs(ex).max() < 1e-10


def test_3d_rates_under_refinement():
    err = {}
    for n in (33, 65):
        p = w.c2_3d(n)
        ex = closed_form.bump_potential_on_grid(p)
        for order in (4, 6):
            phi = solve.solve(p.rho(), p.h, order, boundary="convolution")
            err[n, order] = np.abs(phi - ex).max() / np.abs(ex).max()
    r4 = np.log2(err[33, 4] / err[65, 4])
    r6 = np.log2(err[33, 6] / err[65, 6])
    assert 3.6 < r4 < 4.6, r4
    assert r6 > 5.5, r6
    assert err[65, 6] < 1e-10


def _golden_rates():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return {int(r[0]): (float(r[1]), float(r[2])) for r in rows}


# The paper's 6th-order window: h in [0.02, 0.1], i.e. M = 20..100 panels on [-1,1]^3
TABLE1_M6 = (20, 28, 40, 56, 80, 100)


def _table1_rate6(p):
    centre = (1 / np.sqrt(31), 0.2, 0.1)
    hs, es = [], []
    for M in TABLE1_M6:
        pr = w.scaled_bump((M + 1,) * 3, centre=centre, eps=0.4, p=p)
        phi = solve.solve(pr.rho(), pr.h, 6, boundary="convolution")
        ex = closed_form.bump_potential_on_grid(pr)
        hs.append(2.0 / M)
        es.append(np.abs(phi - ex).max() / np.abs(ex).max())
    return float(np.polyfit(np.log(hs), np.log(es), 1)[0]), es


@pytest.mark.parametrize("diff,p", [(0, 1), (4, 5), (6, 7), (8, 9)])
def test_table1_sixth_order_rates_over_the_papers_window(diff, p):
    # section 6, Table 1: rho = B_{0.4,p}(x - a) with (p - 1) continuous
    # derivatives, 6th-order rates fitted over the paper's h in [0.02, 0.1]
    paper = _golden_rates()[diff][1]
    rate, es = _table1_rate6(p)
    if diff <= 4:
        # limited smoothness: the rate is the density's, and the paper's value is
        # reproduced to the second digit
        assert abs(rate - paper) < 0.2, (rate, paper)
    elif diff == 8:
        # the finest grid (M = 100) reaches the rounding floor (error ~7e-12), which
        # pulls the fitted slope below the paper's 10.8
        assert es[-1] < 2e-11
        assert abs(rate - paper) < 1.0, (rate, paper)
    else:
        # C^6: the method as read gives a steady 8.6 (pairwise slopes 9.2, 8.4, 8.7,
        # 8.6, 8.5), the paper prints 9.8; the other extrapolation reading of section 5
        # gives the same errors, and no choice of fit points gets above 9
        assert 8.0 < rate < paper, (rate, paper)


def test_linearity_and_boundary_assembly():
    p = w.scaled_bump((17, 19, 21), p=6)
    q = w.Problem("r", p.n, p.lo, p.hi, "random", dict(seed=3, margin=2))
    a, b = p.rho(), q.rho()
    parts = {}
    phi_ab = solve.solve(a + 0.5 * b, p.h, 6, parts=parts)
    phi_a = solve.solve(a, p.h, 6)
    phi_b = solve.solve(b, p.h, 6)
    np.testing.assert_allclose(phi_ab, phi_a + 0.5 * phi_b, atol=1e-13 * np.abs(phi_ab).max())
    from oracle import greens
    m = greens.boundary_mask(p.n)
    np.testing.assert_array_equal(phi_ab[m], parts["g"][m])


def _bump_potential_1d(x, c, eps, p):
    """(1/2) int |x - y| (1 - (y-c)^2/eps^2)^p dy over |y - c| < eps, exactly
    (polynomial algebra): the free-space potential of the bump in 1-D, G = |x|/2."""
    from numpy.polynomial import polynomial as P
    q = P.polypow([1.0, 0.0, -1.0 / eps ** 2], p)   # in s = y - c
    Q0 = P.polyint(q)                                # int q
    Q1 = P.polyint(P.polymul(q, [0.0, 1.0]))         # int s q
    out = []
    for xv in x:
        t = xv - c
        s = min(max(t, -eps), eps)
        left = t * (P.polyval(s, Q0) - P.polyval(-eps, Q0)) - (P.polyval(s, Q1) - P.polyval(-eps, Q1))
        right = (P.polyval(eps, Q1) - P.polyval(s, Q1)) - t * (P.polyval(eps, Q0) - P.polyval(s, Q0))
        out.append(0.5 * (left + right))
    return np.array(out)


def test_1d_solve_matches_exact_potential():
    # d = 1 (section 5): phi* by the sine series and the straight line through
    # the trapezoid end values g(a), g(b); the whole potential converges to the
    # exact one, fast (the bump is C^9 and vanishes with its derivatives at the ends)
    errs = []
    for n in (33, 65):   # 129 is at the rounding floor (2e-14)
        p = w.scaled_bump((n,), centre=(0.1,), eps=0.6, p=10)
        phi = solve.solve(p.rho(), p.h, 6)
        ex = _bump_potential_1d(p.coords()[0], 0.1, 0.6, 10)
        errs.append(np.abs(phi - ex).max() / np.abs(ex).max())
    assert errs[1] < 1e-12
    assert errs[0] / errs[1] > 2.0 ** 8
    # the end values are the trapezoid sums themselves: phi(a) = (h^2/2) sum p rho_p
    p = w.scaled_bump((33,), centre=(-0.2,), eps=0.5, p=4)
    rho = p.rho()
    phi = solve.solve(rho, p.h, 4)
    M, h = 32, p.h[0]
    k = np.arange(1, M)
    assert abs(phi[0] - 0.5 * h * h * np.dot(k, rho[1:M])) < 1e-15 * np.abs(phi).max()
    assert abs(phi[M] - 0.5 * h * h * np.dot(M - k, rho[1:M])) < 1e-15 * np.abs(phi).max()
