"""Out-of-bounds writes, checked without a memory checker: every device buffer a
plan allocates sits between two 256-byte guard regions filled with a fixed byte,
and idp_plan_check_guards reports one that was overwritten.  Every path of the
library runs here on small ragged grids (all stages, every precision, autotuning,
host buffers, batches, padded and 1-D plans), then the guards are checked."""
import numpy as np
import pytest

import workloads as w
from tests.gpu_util import device, run_stage, to_dev

pytestmark = pytest.mark.gpu

GRIDS = [
    w.Problem("g1", (17, 33, 17), (-1.0, -1.0, -0.8), (1.0, 1.2, 1.0), "bump",
              dict(centre=(0.05, 0.1, 0.05), eps=0.6, p=10)),
    w.Problem("g2", (65, 33, 129), (0.0, 0.0, 0.0), (1.0, 1.0, 2.0), "points", dict(seed=11, count=9)),
    w.Problem("g3", (49, 97, 33), (0.0, 0.0, 0.0), (1.0, 1.5, 0.8), "gauss", dict(seed=7)),
    w.Problem("g4", (41, 50, 37), (-1.0, -1.2, -0.9), (1.0, 1.25, 0.9), "bump",
              dict(centre=(0.05, 0.0, 0.02), eps=0.6, p=10)),
    w.Problem("g5", (33, 65), (-1.0, -1.2), (1.0, 1.3), "bump", dict(centre=(0.1, -0.05), eps=0.7, p=8)),
    w.Problem("g6", (97, 49), (-1.0, -0.7), (1.0, 0.8), "random", dict(seed=3, margin=2)),
    w.Problem("g7", (17,), (0.0,), (1.0,), "random", dict(seed=4)),
    w.Problem("g8", (513,), (0.0,), (3.0,), "gauss", dict(seed=5)),
]


@pytest.fixture(scope="module")
def idp():
    import paper_2108_11871_gb300 as m
    device()
    m.library()
    return m


@pytest.mark.parametrize("prob", GRIDS, ids=[g.name + "_" + "x".join(map(str, g.n)) for g in GRIDS])
def test_guards_stay_intact_on_every_path(idp, prob):
    import torch
    rho = prob.rho()
    r = to_dev(rho)
    plan = idp.create_plan(prob.d, prob.n, prob.h, 6)
    padded = idp.plan_grid(plan)[0] != list(prob.n)
    idp.plan_set(plan, idp.IDP_KEY_AUTOTUNE, 1)
    precisions = [idp.IDP_PRECISION_FP64]
    if prob.d > 1:
        precisions += [idp.IDP_PRECISION_DF32, idp.IDP_PRECISION_MIXED_BF16X3, idp.IDP_PRECISION_MIXED_TF32X3]
    for prec in precisions:
        idp.plan_set(plan, idp.IDP_KEY_PRECISION, prec)
        out = to_dev(np.zeros(prob.n))
        idp.solve(plan, r, out)
        idp.plan_status(plan)
        if not padded:
            ishape = tuple(k - 2 for k in prob.n)
            stages = [(idp.IDP_STAGE_BOUNDARY, prob.n), (idp.IDP_STAGE_PHISTAR, prob.n),
                      (idp.IDP_STAGE_U1, prob.n)]
            if prob.d > 1:
                stages += [(idp.IDP_STAGE_GTILDE, ishape), (idp.IDP_STAGE_R, ishape)]
            for stage, shape in stages:
                run_stage(idp, plan, stage, r, shape)
    idp.plan_set(plan, idp.IDP_KEY_PRECISION, idp.IDP_PRECISION_FP64)
    idp.plan_set(plan, idp.IDP_KEY_VALIDATE, 2)
    rp = torch.from_numpy(rho).pin_memory()
    pp = torch.zeros(prob.n, dtype=torch.float64).pin_memory()
    idp.solve_host(plan, rp.data_ptr(), pp.data_ptr())
    idp.plan_set(plan, idp.IDP_KEY_VALIDATE, 0)
    idp.solve_host(plan, rp.data_ptr(), pp.data_ptr())
    idp.solve_host(plan, rho, pp.numpy())                  # pageable buffers: plain copies
    try:
        idp.plan_status(plan)
    except idp.IdpError as e:
        assert e.code == idp.IDP_ESUPPORT                  # validation: rho near the boundary
    other = idp.create_plan(3, (17, 17, 17), (0.1, 0.1, 0.1), 6)
    o2 = to_dev(np.zeros((17, 17, 17)))
    idp.solve_batched([plan, other], [r, to_dev(w.random_interior((17, 17, 17), seed=2, margin=3))],
                      [to_dev(np.zeros(prob.n)), o2])
    torch.cuda.synchronize()
    idp.plan_check_guards(plan)
    idp.plan_check_guards(other)


def test_guard_check_detects_a_changed_guard_byte(idp):
    # the check itself: a guard byte changed from the host (inside the allocation,
    # through the test hook) is reported as IDP_EGUARD; restored, the check passes
    plan = idp.create_plan(3, (17, 17, 17), (0.1, 0.1, 0.1), 6)
    idp.plan_check_guards(plan)
    idp.plan_set(plan, idp.IDP_KEY_GUARD_TEST, 1)
    with pytest.raises(idp.IdpError) as e:
        idp.plan_check_guards(plan)
    assert e.value.code == idp.IDP_EGUARD
    idp.plan_set(plan, idp.IDP_KEY_GUARD_TEST, 0)
    idp.plan_check_guards(plan)
