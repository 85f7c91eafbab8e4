"""The CPU fast-transform form of the method (the bench's paper-method CPU
baseline) computes the oracle's discrete result."""
import numpy as np
import pytest

import workloads as w
from oracle import fft_baseline, solve as osolve

pytest.importorskip("scipy")


@pytest.mark.parametrize("prob", [w.c1_2d(33), w.Problem("a", (17, 33, 25), (0.0,) * 3, (1.0, 1.5, 0.9), "gauss",
                                                        dict(seed=3)), w.c2_3d(33)],
                         ids=["2d_33", "3d_17x33x25", "3d_33"])
@pytest.mark.parametrize("order", [4, 6])
def test_fft_baseline_equals_the_oracle(prob, order):
    rho = prob.rho()
    ref = osolve.solve(rho, prob.h, order, boundary="direct")
    got = fft_baseline.solve(rho, prob.h, order, workers=2)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12
