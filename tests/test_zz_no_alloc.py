"""The allocation-free right-hand-side entry point (idp_rhs6_noalloc).

It is meant for callers that cannot let the library allocate device memory
(their own pool allocator owns the GPU's memory, or their loop cannot pay
for cudaMalloc's synchronisation).  Through the C ABI, on the u1 of the
plan-based solver (IDP_STAGE_U1), its R must equal the oracle's stencil R of
the same u1 within the rounding of a sixth difference (the propagation bound of
the parity tests with du = 4 eps max|u1|), and consecutive calls that share the
library's fixed scratch must give the same bits.  (The plan's own R, computed
in spectral form, is held to the oracle in test_gpu_parity.py.)  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as w
from oracle import harmonic as oharm
from tests.gpu_util import device, r_amplification, run_stage, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def idp():
    import paper_2108_11871_gb300 as m
    device()
    m.library()
    return m


def _reference(idp, prob):
    """u1 from the plan-based entry point, the oracle's R of that u1, and the
    plan-based entry point's own R (IDP_STAGE_R, spectral form)."""
    plan = idp.create_plan(prob.d, prob.n, prob.h, 6)
    r = to_dev(prob.rho())
    u1 = run_stage(idp, plan, idp.IDP_STAGE_U1, r, prob.n)
    R_plan = run_stage(idp, plan, idp.IDP_STAGE_R, r, tuple(k - 2 for k in prob.n))
    return u1, oharm.rhs6(u1, prob.h), R_plan


def test_noalloc_rhs_matches_plan_rhs_on_consecutive_calls(idp):
    import torch
    probs = [w.Problem("a", (33, 17, 65), (0.0, 0.0, 0.0), (1.0, 0.5, 2.0), "gauss", dict(seed=4)),
             w.c1_2d(65),
             w.c2_3d(65)]
    refs = [_reference(idp, p) for p in probs]
    first = {}
    # two calls in a row per problem, problems interleaved, so each call starts
    # from scratch contents left by a different problem
    for rep in range(2):
        for p, (u1, Rref, R_plan) in zip(probs, refs):
            u1d = to_dev(u1)
            out = torch.full(tuple(k - 2 for k in p.n), float("nan"), dtype=torch.float64,
                             device=u1d.device)
            idp.rhs6_noalloc(p.d, p.n, p.h, u1d, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            du = 4 * np.finfo(np.float64).eps * np.abs(u1).max()
            amp = r_amplification(p.h)
            core = tuple(slice(1, -1) for _ in got.shape)
            assert np.abs(got - Rref)[core].max() <= amp * du, (rep, p.name)
            assert np.abs(got - Rref).max() <= amp * 15 ** p.d * du, (rep, p.name)
            # the same R as the existing entry point: the plan's IDP_STAGE_R is formed
            # in spectral form from u1's sine coefficients, so the two differ by the
            # stencil applied to the rounding of u1's nodal values, which come out of
            # an FP64 transform (at most 2 eps per FFT stage, log2(n) stages per axis)
            du_t = 2 * sum(np.log2(k) for k in p.n) * np.finfo(np.float64).eps * np.abs(u1).max()
            assert np.abs(got - R_plan)[core].max() <= amp * du_t, (rep, p.name)
            assert np.abs(got - R_plan).max() <= amp * 15 ** p.d * du_t, (rep, p.name)
            if rep == 0:
                first[p.name] = got
            else:
                assert np.array_equal(got, first[p.name]), p.name


def test_noalloc_rejects_problems_beyond_its_scratch(idp):
    import torch
    n = (129, 129, 129)           # 2 146 689 nodes > IDP_RHS6_NOALLOC_MAX_NODES
    assert np.prod(n) > idp.IDP_RHS6_NOALLOC_MAX_NODES
    x = torch.zeros(8, dtype=torch.float64, device=device())
    lib = idp.library()
    rc = lib.idp_rhs6_noalloc(3, (ctypes.c_int64 * 3)(*n), (ctypes.c_double * 3)(0.1, 0.1, 0.1),
                              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr() + 8),
                              None)
    assert rc == idp.IDP_ESCRATCH
    assert "scratch" in idp.strerror(rc)
    # node counts whose product would overflow 64 bits are refused the same way
    huge = (2 ** 31 + 8, 2 ** 31 + 8, 8)
    rc = lib.idp_rhs6_noalloc(3, (ctypes.c_int64 * 3)(*huge), (ctypes.c_double * 3)(0.1, 0.1, 0.1),
                              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr() + 8),
                              None)
    assert rc == idp.IDP_ESCRATCH
