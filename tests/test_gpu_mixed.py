"""Tensor-core (mixed-precision) sine transforms against the FP64 oracle.

IDP_PRECISION_MIXED_BF16X3 replaces the sine transforms of rho, of R and the
final inverse by dense sine-matrix products on the tensor cores: operands
split into three BF16 pieces, the six products with piece indices i + j <= 2,
FP32 accumulation.  The transform producing u1 stays FP64 because R is a
sixth difference of u1 (section 5) and would amplify its rounding.  The dropped products are below 2^-24 relative; the FP32
accumulation of n terms gives a relative error of order sqrt(n) 2^-24 per
pass.  Stated accuracy (checked here and at 513^3 in test_gpu_parity.py):
max-norm error relative to max|phi| below 1e-6 * sqrt(n_max) for phi* and the
full solve, n_max the longest line (1.1e-5 for the 129^3 grid).

IDP_PRECISION_MIXED_TF32X3 splits the operands into two TF32 pieces (hi + lo,
11 significant bits each, ~22 kept against ~24 for three BF16 pieces) and keeps
the three products hi*hi, hi*lo, lo*hi: the dropped lo*lo term and the rounding
of lo are ~2^-22 relative, four times the BF16X3 bound, so its stated accuracy
is 4e-6 * sqrt(n_max).
"""
import numpy as np
import pytest

import workloads as w
from oracle import dst as odst, solve as osolve
from tests.gpu_util import device, rel_max, run_stage, to_dev

pytestmark = pytest.mark.gpu
MIXED_TOL = 1e-6 * np.sqrt(127)
TF32_TOL = 4e-6 * np.sqrt(127)
VARIANTS = ["bf16x3", "tf32x3"]


def _prec(idp, variant):
    return idp.IDP_PRECISION_MIXED_TF32X3 if variant == "tf32x3" else idp.IDP_PRECISION_MIXED_BF16X3


def _tol(variant):
    return TF32_TOL if variant == "tf32x3" else MIXED_TOL


@pytest.fixture(scope="module")
def idp():
    import paper_2108_11871_gb300 as m
    device()
    m.library()
    return m


def _plan(idp, prob, order=6, variant="bf16x3"):
    plan = idp.create_plan(prob.d, prob.n, prob.h, order)
    idp.plan_set(plan, idp.IDP_KEY_PRECISION, _prec(idp, variant))
    return plan


@pytest.mark.parametrize("variant", VARIANTS)
def test_mixed_phistar_of_a_sine_mode(idp, variant):
    n = (33, 65, 129)
    box = ((0.0, 1.0), (0.0, 0.7), (-1.0, 1.5))
    coords = [np.linspace(a, b, k) for (a, b), k in zip(box, n)]
    h = [c[1] - c[0] for c in coords]
    X = np.meshgrid(*coords, indexing="ij")
    modes = (3, 7, 40)
    rho = np.ones(n)
    lam = 0.0
    for s in range(3):
        L = box[s][1] - box[s][0]
        rho = rho * np.sin(modes[s] * np.pi * (X[s] - box[s][0]) / L)
        lam += (modes[s] * np.pi / L) ** 2
    plan = idp.create_plan(3, n, h, 4)
    idp.plan_set(plan, idp.IDP_KEY_PRECISION, _prec(idp, variant))
    ps = run_stage(idp, plan, idp.IDP_STAGE_PHISTAR, to_dev(rho), n)
    err = rel_max(ps, -rho / lam)
    print("phistar sine mode", variant, err)
    assert err < _tol(variant)


@pytest.mark.parametrize("prob", [w.c2_3d(33), w.c1_2d(65),
                                  w.Problem("g", (65, 33, 129), (0.0,) * 3, (1.0, 1.0, 2.0), "gauss",
                                            dict(seed=2108)),
                                  w.c2_3d(129)], ids=["3d_33", "2d_65", "3d_65x33x129", "3d_129"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_mixed_solve_against_oracle(idp, prob, variant):
    rho = prob.rho()
    plan = _plan(idp, prob, variant=variant)
    r = to_dev(rho)
    ps = run_stage(idp, plan, idp.IDP_STAGE_PHISTAR, r, prob.n)
    e1 = rel_max(ps, odst.phi_star(rho, prob.h))
    phi = to_dev(np.zeros(prob.n))
    idp.solve(plan, r, phi)
    idp.plan_status(plan)
    ref = osolve.solve(rho, prob.h, 6, boundary="convolution")
    err = rel_max(phi.cpu().numpy(), ref)
    print("mixed", variant, prob.n, e1, err)
    assert e1 < _tol(variant)
    assert err < _tol(variant), err


def test_switching_precision_back_to_fp64_restores_fp64_results(idp):
    prob = w.c2_3d(33)
    rho = to_dev(prob.rho())
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    a = to_dev(np.zeros(prob.n))
    idp.solve(plan, rho, a)
    outs = []
    for variant in VARIANTS + ["bf16x3"]:
        idp.plan_set(plan, idp.IDP_KEY_PRECISION, _prec(idp, variant))
        b = to_dev(np.zeros(prob.n))
        idp.solve(plan, rho, b)
        outs.append(b)
    idp.plan_set(plan, idp.IDP_KEY_PRECISION, idp.IDP_PRECISION_FP64)
    c = to_dev(np.zeros(prob.n))
    idp.solve(plan, rho, c)
    idp.plan_status(plan)
    a, c = a.cpu().numpy(), c.cpu().numpy()
    b16, t32, b16b = (o.cpu().numpy() for o in outs)
    assert np.array_equal(a, c)
    assert 0 < rel_max(b16, a) < MIXED_TOL
    assert 0 < rel_max(t32, a) < TF32_TOL
    assert not np.array_equal(b16, t32)
    assert np.array_equal(b16, b16b)   # switching variants back and forth repeats the bits


@pytest.mark.parametrize("variant", VARIANTS)
def test_bounded_wait_expires_into_a_status_not_a_hang(idp, variant):
    # failure handling without a GPU fault: the stall-test hook makes one
    # tensor-core pass issue no products, so its mbarrier wait runs out after
    # its bound; the kernel records it, frees its tensor memory and returns
    prob = w.c2_3d(33)
    rho = to_dev(prob.rho())
    plan = _plan(idp, prob, variant=variant)
    out = to_dev(np.zeros(prob.n))
    idp.plan_set(plan, idp.IDP_KEY_STALL_TEST, 1)
    idp.solve(plan, rho, out)
    with pytest.raises(idp.IdpError) as e:
        idp.plan_status(plan)
    assert e.value.code == idp.IDP_ETIMEOUT
    # the context and the plan remain usable
    idp.solve(plan, rho, out)
    idp.plan_status(plan)
    ref = osolve.solve(prob.rho(), prob.h, 6, boundary="convolution")
    assert rel_max(out.cpu().numpy(), ref) < _tol(variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_mixed_with_double_float_boundary_against_oracle(idp, variant):
    # IDP_KEY_MIXED_BOUNDARY_DF32 = 1: the 3-D boundary convolutions of a tensor-core
    # mode in double-float arithmetic (48 bits): the result stays within the mode's
    # stated bound, and its boundary values within the double-float bound of g
    prob = w.Problem("g", (65, 33, 129), (0.0,) * 3, (1.0, 1.0, 2.0), "gauss", dict(seed=2108))
    rho = prob.rho()
    plan = _plan(idp, prob, variant=variant)
    idp.plan_set(plan, idp.IDP_KEY_MIXED_BOUNDARY_DF32, 1)
    r = to_dev(rho)
    parts = {}
    ref = osolve.solve(rho, prob.h, 6, boundary="convolution", parts=parts)
    g = run_stage(idp, plan, idp.IDP_STAGE_BOUNDARY, r, prob.n)
    from oracle import greens as ogreens
    mask = ogreens.boundary_mask(prob.n)
    assert rel_max(g[mask], parts["g"][mask]) < 1e-12
    phi = to_dev(np.zeros(prob.n))
    idp.solve(plan, r, phi)
    idp.plan_status(plan)
    err = rel_max(phi.cpu().numpy(), ref)
    assert err < _tol(variant), err
    # switching it off gives back the FP64 boundary
    idp.plan_set(plan, idp.IDP_KEY_MIXED_BOUNDARY_DF32, 0)
    g64 = run_stage(idp, plan, idp.IDP_STAGE_BOUNDARY, r, prob.n)
    fp = idp.create_plan(prob.d, prob.n, prob.h, 6)
    assert np.array_equal(g64, run_stage(idp, fp, idp.IDP_STAGE_BOUNDARY, r, prob.n))
