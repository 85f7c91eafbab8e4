"""Plans solved on the grid as given (idp_create_plan_exact), for panel counts
without an FFT here, against the FP64 oracle on the same grid.

The sine transforms of such lengths run as direct sums (FP64 in precision FP64,
double-float otherwise), or on the tensor cores in the tensor-core modes, which
take any length; the boundary convolutions use the next FFT length 2P >= 2M.
Tolerances: 1e-12 (FP64), 4e-12 (double-float), 1e-6 sqrt(n_max) (BF16x3) and
4e-6 sqrt(n_max) (TF32x3), as for the padded plans.  The precision sweep's
stated sizes, 256^3 interior points (M = 257, prime), are checked here too.
"""
import numpy as np
import pytest

import workloads as w
from oracle import greens as ogreens, solve as osolve
from tests.gpu_util import device, r_amplification, rel_max, run_stage, to_dev

pytestmark = pytest.mark.gpu
SMALL = [
    # panel counts 33, 49, 40: none has an FFT here (2^a, 3 2^a only)
    ("3d_34x50x41", w.Problem("x1", (34, 50, 41), (0.0, 0.0, 0.0), (1.0, 1.4, 1.2), "gauss", dict(seed=41))),
    ("2d_45x70", w.Problem("x2", (45, 70), (-1.0, -1.2), (1.0, 1.3), "bump",
                           dict(centre=(0.05, -0.03), eps=0.7, p=8))),
]
PRECS = {"fp64": ("FP64", 1e-12), "df32": ("DF32", 4e-12), "bf16x3": ("MIXED_BF16X3", 1e-6),
         "tf32x3": ("MIXED_TF32X3", 4e-6)}
_REF = {}


@pytest.fixture(scope="module")
def idp():
    import paper_2108_11871_gb300 as m
    device()
    m.library()
    return m


def _oracle(name, prob, order=6):
    if (name, order) not in _REF:
        parts = {}
        phi = osolve.solve(prob.rho(), prob.h, order, boundary="convolution", parts=parts)
        parts["phi"] = phi
        _REF[name, order] = parts
    return _REF[name, order]


def _tol(prec, prob):
    base = PRECS[prec][1]
    return base * np.sqrt(max(prob.n) - 2) if prec in ("bf16x3", "tf32x3") else base


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("name,prob", SMALL, ids=[c[0] for c in SMALL])
def test_exact_plan_matches_oracle(idp, name, prob, prec):
    ref = _oracle(name, prob)
    plan = idp.create_plan(prob.d, prob.n, prob.h, 6, exact=True)
    assert idp.plan_grid(plan)[0] == list(prob.n)       # no padding
    idp.plan_set(plan, idp.IDP_KEY_PRECISION, getattr(idp, "IDP_PRECISION_" + PRECS[prec][0]))
    r = to_dev(prob.rho())
    tol = _tol(prec, prob)
    g = run_stage(idp, plan, idp.IDP_STAGE_BOUNDARY, r, prob.n)
    mask = ogreens.boundary_mask(prob.n)
    gtol = 1e-12 if prec == "fp64" else 4e-12   # the boundary is FP64 or double-float in every mode
    assert rel_max(g[mask], ref["g"][mask]) < gtol
    ps = run_stage(idp, plan, idp.IDP_STAGE_PHISTAR, r, prob.n)
    assert rel_max(ps, ref["phistar"]) < tol
    u1 = run_stage(idp, plan, idp.IDP_STAGE_U1, r, prob.n)
    assert rel_max(u1, ref["u1"]) < (1e-12 if prec == "fp64" else 4e-12)
    if prec == "fp64":
        ishape = tuple(k - 2 for k in prob.n)
        gt = run_stage(idp, plan, idp.IDP_STAGE_GTILDE, r, ishape)
        assert rel_max(gt, ref["gtilde"]) < tol
        R = run_stage(idp, plan, idp.IDP_STAGE_R, r, ishape)
        du = np.abs(u1 - ref["u1"]).max() + 4 * np.finfo(np.float64).eps * np.abs(ref["u1"]).max()
        amp = r_amplification(prob.h)
        core = tuple(slice(1, -1) for _ in ishape)
        assert np.abs(R - ref["R"])[core].max() <= amp * du
        assert np.abs(R - ref["R"]).max() <= amp * 15 ** prob.d * du
    out = to_dev(np.zeros(prob.n))
    idp.solve(plan, r, out)
    idp.plan_status(plan)
    err = rel_max(out.cpu().numpy(), ref["phi"])
    print("exact", name, prec, err)
    assert err < tol


def test_exact_plan_equals_the_padded_plan_where_no_padding_is_needed(idp):
    # on a grid whose panel counts all have FFTs the exact plan is the ordinary one
    prob = w.Problem("x3", (33, 49, 65), (0.0,) * 3, (1.0, 1.5, 2.0), "gauss", dict(seed=43))
    r = to_dev(prob.rho())
    outs = []
    for exact in (False, True):
        plan = idp.create_plan(3, prob.n, prob.h, 6, exact=exact)
        o = to_dev(np.zeros(prob.n))
        idp.solve(plan, r, o)
        idp.plan_status(plan)
        outs.append(o.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_precision_sweep_at_its_stated_size(idp, prec):
    # 256^3 interior points (258^3 nodes, M = 257 on every axis): the tensor-core
    # transforms take the length as given
    prob = w.c4_sweep((256, 256, 256))
    ref = _oracle("c4_258", prob)
    plan = idp.create_plan(3, prob.n, prob.h, 6, exact=True)
    idp.plan_set(plan, idp.IDP_KEY_PRECISION, getattr(idp, "IDP_PRECISION_" + PRECS[prec][0]))
    r = to_dev(prob.rho())
    ps = run_stage(idp, plan, idp.IDP_STAGE_PHISTAR, r, prob.n)
    out = to_dev(np.zeros(prob.n))
    idp.solve(plan, r, out)
    idp.plan_status(plan)
    tol = _tol(prec, prob)
    e1, e2 = rel_max(ps, ref["phistar"]), rel_max(out.cpu().numpy(), ref["phi"])
    print("sweep 258^3", prec, e1, e2)
    assert e1 < tol and e2 < tol


def test_exact_plan_rejects_too_small_and_too_large_grids(idp):
    lib = idp.library()
    import ctypes
    out = ctypes.c_void_p()
    h = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    assert lib.idp_create_plan_exact(ctypes.byref(out), 3, (ctypes.c_int64 * 3)(7, 20, 20), h, 6) == idp.IDP_EINVAL
    assert lib.idp_create_plan_exact(ctypes.byref(out), 3, (ctypes.c_int64 * 3)(514, 20, 20), h, 6) == \
        idp.IDP_ESUPPORT
