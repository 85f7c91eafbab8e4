"""GPU path (through the C ABI) against the FP64 oracle, component by component.

Tolerance: max-norm error relative to the component's max |value|, 1e-12 for
every FP64 result (the FP64 parity target).

The 6th-order right-hand side R (section 5) is a difference quotient of u1:
a perturbation du of u1 changes R on the core by at most A * max|du| with
A = sum_{s != r} c_sr * 64 / (h_s^4 h_r^2), and the cubic extrapolation
(weights 4, -6, 4, -1; absolute sum 15 per axis) multiplies that by up to 15^d
next to the boundary.  With du = (measured max|u1_gpu - u1_oracle|) + 4 eps max|u1|
(the input difference plus the rounding of the stencil itself), R is checked
against A du on the core and 15^d A du on the extrapolated layers -- the
propagation bound of the operation, not a loosened target.  u1 itself is held
to 1e-12, and so is phi, which R feeds through the smoothing solve L4_0^{-1}.
"""
import numpy as np
import pytest

import workloads as w
from oracle import greens as ogreens, solve as osolve
from tests.gpu_util import device, r_amplification, rel_max, run_stage, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-12

CASES = [
    # (name, problem) -- several tiles, ragged tails, anisotropic h
    ("2d_33x65", w.Problem("a", (33, 65), (-1.0, -1.2), (1.0, 1.3), "bump",
                           dict(centre=(0.1, -0.05), eps=0.7, p=8))),
    ("2d_65", w.c1_2d(65)),
    ("3d_17x33x17", w.Problem("b", (17, 33, 17), (-1.0, -1.0, -0.8), (1.0, 1.2, 1.0), "bump",
                              dict(centre=(0.05, 0.1, 0.05), eps=0.6, p=10))),
    ("3d_33", w.c2_3d(33)),
    ("3d_65x33x129", w.Problem("c", (65, 33, 129), (0.0, 0.0, 0.0), (1.0, 1.0, 2.0), "gauss",
                               dict(seed=2108))),
    # panel counts 3 * 2^a (radix-3 FFT stage): 48, 96, 32 and 96, 48
    ("3d_49x97x33", w.Problem("d", (49, 97, 33), (0.0, 0.0, 0.0), (1.0, 1.5, 0.8), "gauss",
                              dict(seed=7))),
    ("2d_97x49", w.Problem("e", (97, 49), (-1.0, -0.7), (1.0, 0.8), "bump",
                           dict(centre=(0.05, 0.0), eps=0.6, p=8))),
    # scattered point values: most lines / slices exactly zero, some blocks of
    # lines partly zero (the zero-line and zero-slice skipping of section 4's stages)
    ("3d_65x33x129_points", w.Problem("f", (65, 33, 129), (0.0, 0.0, 0.0), (1.0, 1.0, 2.0), "points",
                                      dict(seed=11, count=9))),
    ("2d_65x33_points", w.Problem("g", (65, 33), (0.0, 0.0), (1.0, 0.5), "points",
                                  dict(seed=12, count=4))),
]


@pytest.fixture(scope="module")
def idp():
    import paper_2108_11871_gb300 as m
    device()
    m.library()
    return m


def _oracle_parts(prob, order):
    parts = {}
    phi = osolve.solve(prob.rho(), prob.h, order, boundary="convolution", parts=parts)
    parts["phi"] = phi
    return parts


_DIRECT = {}


def _direct_g(name, prob):
    """g on every boundary node by the direct trapezoid sum (eq. TrapOrig2D), cached."""
    if name not in _DIRECT:
        _DIRECT[name] = ogreens.boundary_direct_nodes(prob.rho(), prob.h)
    return _DIRECT[name]


@pytest.mark.parametrize("precision", ["fp64", "df32"])
@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("name,prob", CASES, ids=[c[0] for c in CASES])
def test_components_match_oracle(idp, name, prob, order, precision):
    # fp64: FP64 transforms; df32: double-float transforms on the FP32 pipe,
    # held to the same 1e-12 target
    rho = prob.rho()
    ref = _oracle_parts(prob, order)
    plan = idp.create_plan(prob.d, prob.n, prob.h, order)
    if precision == "df32":
        idp.plan_set(plan, idp.IDP_KEY_PRECISION, idp.IDP_PRECISION_DF32)
    r = to_dev(rho)
    nshape = prob.n
    ishape = tuple(k - 2 for k in prob.n)
    g = run_stage(idp, plan, idp.IDP_STAGE_BOUNDARY, r, nshape)
    mask = ogreens.boundary_mask(prob.n)
    assert rel_max(g[mask], ref["g"][mask]) < TOL
    # and against the direct trapezoid sum of section 4 on every boundary node
    assert rel_max(g[mask], _direct_g(name, prob)[mask]) < TOL
    assert np.all(g[~mask] == 0)
    ps = run_stage(idp, plan, idp.IDP_STAGE_PHISTAR, r, nshape)
    assert rel_max(ps, ref["phistar"]) < TOL
    gt = run_stage(idp, plan, idp.IDP_STAGE_GTILDE, r, ishape)
    assert rel_max(gt, ref["gtilde"]) < TOL
    u1 = run_stage(idp, plan, idp.IDP_STAGE_U1, r, nshape)
    assert rel_max(u1, ref["u1"]) < TOL
    du = np.abs(u1 - ref["u1"]).max() + 4 * np.finfo(np.float64).eps * np.abs(ref["u1"]).max()
    if order == 6:
        R = run_stage(idp, plan, idp.IDP_STAGE_R, r, ishape)
        amp = r_amplification(prob.h)
        core = tuple(slice(1, -1) for _ in ishape)
        assert np.abs(R - ref["R"])[core].max() <= amp * du
        assert np.abs(R - ref["R"]).max() <= amp * 15 ** prob.d * du
    phi = run_stage(idp, plan, idp.IDP_STAGE_PHI, r, nshape)
    assert rel_max(phi, ref["phi"]) < TOL
    # the solve entry point gives the same bits as the staged run
    out = to_dev(np.zeros(nshape))
    idp.solve(plan, r, out)
    idp.plan_status(plan)
    assert np.array_equal(out.cpu().numpy(), phi)


def test_single_sine_transform_pass_against_library_dst(idp):
    # phi* of a single sine mode is exact (closed form) -- checks the sine
    # transforms and the continuum eigenvalues through the C ABI
    n = (65, 33, 129)
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
    ps = run_stage(idp, plan, idp.IDP_STAGE_PHISTAR, to_dev(rho), n)
    assert rel_max(ps, -rho / lam) < TOL


@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_129_cube_sampled_against_direct_sum_and_full_oracle(idp, precision):
    # the bench workload (129^3 bump, order 6) in the bench's configuration
    # (autotuned plan, graph replay): g at sampled boundary nodes against the
    # direct trapezoid sum, and phi against the oracle everywhere
    prob = w.c2_3d(129)
    rho = prob.rho()
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    if precision == "df32":
        idp.plan_set(plan, idp.IDP_KEY_PRECISION, idp.IDP_PRECISION_DF32)
    idp.plan_set(plan, idp.IDP_KEY_AUTOTUNE, 1)
    r = to_dev(rho)
    g = run_stage(idp, plan, idp.IDP_STAGE_BOUNDARY, r, prob.n)
    idx = ogreens.boundary_indices(prob.n)
    rng = np.random.default_rng(5)
    pick = idx[rng.choice(len(idx), 2048, replace=False)]
    corners = np.array([[i, j, k] for i in (0, 128) for j in (0, 128) for k in (0, 128)], dtype=np.int32)
    pick = np.concatenate([pick, corners])
    ref = ogreens.boundary_direct(rho, prob.h, pick)
    assert rel_max(g[tuple(pick.T)], ref) < TOL
    phi = to_dev(np.zeros(prob.n))
    idp.solve(plan, r, phi)
    idp.plan_status(plan)
    ref_phi = osolve.solve(rho, prob.h, 6, boundary="convolution")
    assert rel_max(phi.cpu().numpy(), ref_phi) < TOL


def test_host_entry_point_matches_device_entry_point(idp):
    prob = w.c2_3d(33)
    rho = prob.rho()
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    out_h = np.zeros(prob.n)
    idp.solve_host(plan, rho, out_h)
    out_d = to_dev(np.zeros(prob.n))
    idp.solve(plan, to_dev(rho), out_d)
    idp.plan_status(plan)
    assert np.array_equal(out_h, out_d.cpu().numpy())


@pytest.mark.parametrize("mode,order", [("fp64", 6), ("fp64", 4), ("df32", 6), ("mixed", 6)])
def test_pinned_host_solve_gives_the_device_bits(idp, mode, order):
    # from page-locked host buffers the kernels that produce phi write the host
    # buffer directly (a graph of its own): the result must be the device entry
    # point's, bit for bit, on repeated calls and after the host buffers change
    import torch
    prob = w.Problem("h", (65, 33, 129), (0.0, 0.0, 0.0), (1.0, 1.0, 2.0), "gauss", dict(seed=5))
    plan = idp.create_plan(3, prob.n, prob.h, order)
    if mode != "fp64":
        idp.plan_set(plan, idp.IDP_KEY_PRECISION,
                     idp.IDP_PRECISION_DF32 if mode == "df32" else idp.IDP_PRECISION_MIXED_BF16X3)
    rho = prob.rho()
    ref = to_dev(np.zeros(prob.n))
    idp.solve(plan, to_dev(rho), ref)
    ref = ref.cpu().numpy()
    rho_p = [torch.from_numpy(rho).pin_memory(), torch.from_numpy(rho.copy()).pin_memory()]
    phi_p = [torch.zeros(prob.n, dtype=torch.float64).pin_memory() for _ in range(2)]
    for k in (0, 0, 1, 0):
        phi_p[k].zero_()
        idp.solve_host(plan, rho_p[k].data_ptr(), phi_p[k].data_ptr())
        idp.plan_status(plan)
        assert np.array_equal(phi_p[k].numpy(), ref), k


def test_graph_and_plain_launches_agree_and_repeat(idp):
    prob = w.c3_large(65)
    rho = to_dev(prob.rho())
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    outs = []
    for use_graph in (1, 0, 1):
        idp.plan_set(plan, idp.IDP_KEY_USE_GRAPH, use_graph)
        o = to_dev(np.zeros(prob.n))
        idp.solve(plan, rho, o)
        idp.solve(plan, rho, o)
        idp.plan_status(plan)
        outs.append(o.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_nvtx_ranges_give_the_same_bits(idp):
    # IDP_KEY_NVTX: ranges around every launch and stage, plain launches; the same
    # bits as the graph replay, in single, host-buffer and batched solves
    prob = w.c3_large(65)
    rho = to_dev(prob.rho())
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    ref = to_dev(np.zeros(prob.n))
    idp.solve(plan, rho, ref)
    idp.plan_status(plan)
    idp.plan_set(plan, idp.IDP_KEY_NVTX, 1)
    o = to_dev(np.zeros(prob.n))
    idp.solve(plan, rho, o)
    idp.plan_status(plan)
    assert np.array_equal(o.cpu().numpy(), ref.cpu().numpy())
    import torch
    rh = torch.from_numpy(prob.rho()).pin_memory()
    ph = torch.zeros(prob.n, dtype=torch.float64).pin_memory()
    idp.solve_host(plan, rh.data_ptr(), ph.data_ptr())
    idp.plan_status(plan)
    assert np.array_equal(ph.numpy(), ref.cpu().numpy())
    ob = to_dev(np.zeros(prob.n))
    idp.solve_batched([plan], [rho], [ob])
    idp.plan_status(plan)
    assert np.array_equal(ob.cpu().numpy(), ref.cpu().numpy())
    idp.plan_set(plan, idp.IDP_KEY_NVTX, 0)


def test_batched_equals_single(idp):
    probs = [w.c3_large(33), w.c2_3d(65), w.Problem("x", (33, 65, 17), (0.0,) * 3, (1.0,) * 3,
                                                     "gauss", dict(seed=11))]
    plans = [idp.create_plan(3, p.n, p.h, 6) for p in probs]
    rhos = [to_dev(p.rho()) for p in probs]
    outs = [to_dev(np.zeros(p.n)) for p in probs]
    idp.solve_batched(plans, rhos, outs)
    for pl, r, o, p in zip(plans, rhos, outs, probs):
        single = to_dev(np.zeros(p.n))
        idp.solve(pl, r, single)
        idp.plan_status(pl)
        assert np.array_equal(single.cpu().numpy(), o.cpu().numpy())


def test_batched_graph_uneven_sizes_cache_and_recapture(idp):
    # several problems of different sizes in one graph launch; a second launch
    # replays the cached graph, a changed output pointer recaptures it
    sizes = [(17, 33, 65), (65, 17, 33), (33, 33, 33), (17, 17, 129), (65, 65, 17)]
    probs = [w.Problem("b%d" % i, n, (0.0,) * 3, (1.0,) * 3, "gauss", dict(seed=100 + i))
             for i, n in enumerate(sizes)]
    plans = [idp.create_plan(3, p.n, p.h, 6) for p in probs]
    rhos = [to_dev(p.rho()) for p in probs]
    singles = []
    for pl, r, p in zip(plans, rhos, probs):
        o = to_dev(np.zeros(p.n))
        idp.solve(pl, r, o)
        idp.plan_status(pl)
        singles.append(o.cpu().numpy())
    outs = [to_dev(np.full(p.n, np.nan)) for p in probs]
    for _ in range(2):
        idp.solve_batched(plans, rhos, outs)
        for pl in plans:
            idp.plan_status(pl)
        for o, s in zip(outs, singles):
            assert np.array_equal(o.cpu().numpy(), s)
    outs[2] = to_dev(np.zeros(probs[2].n))
    idp.solve_batched(plans, rhos, outs)
    idp.plan_status(plans[0])
    assert np.array_equal(outs[2].cpu().numpy(), singles[2])


def test_batched_sizes_of_the_batched_workload(idp):
    # the first problems of the 96-problem batched workload (per-axis nodes from
    # {33, 65, 97, 129, 193, 257}), solved in one graph launch, against the oracle
    probs = [p for p in w.c5_batch() if max(p.n) <= 129][:4]
    plans = [idp.create_plan(3, p.n, p.h, 6) for p in probs]
    rhos = [to_dev(p.rho()) for p in probs]
    outs = [to_dev(np.zeros(p.n)) for p in probs]
    idp.solve_batched(plans, rhos, outs)
    for pl in plans:
        idp.plan_status(pl)
    for p, o in zip(probs, outs):
        ref = osolve.solve(p.rho(), p.h, 6, boundary="convolution")
        assert rel_max(o.cpu().numpy(), ref) < TOL, p.n


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_plan_still_matches_oracle(idp, precision):
    prob = w.Problem("t", (65, 33, 129), (0.0, 0.0, 0.0), (1.0, 1.0, 2.0), "gauss", dict(seed=3))
    rho = prob.rho()
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    tol = TOL
    if precision == "mixed":
        idp.plan_set(plan, idp.IDP_KEY_PRECISION, idp.IDP_PRECISION_MIXED_BF16X3)
        tol = 1e-6 * np.sqrt(127)
    idp.plan_set(plan, idp.IDP_KEY_AUTOTUNE, 1)
    info = idp.plan_tuning(plan)
    assert info["tuned"]
    for nch, pch, np_ in zip(info["face_chunks"], info["slices_per_chunk"], (63, 31, 127)):
        assert 1 <= nch <= np_ and nch * pch >= np_ and (nch - 1) * pch < np_
    out = to_dev(np.zeros(prob.n))
    idp.solve(plan, to_dev(rho), out)
    idp.plan_status(plan)
    ref = osolve.solve(rho, prob.h, 6, boundary="convolution")
    assert rel_max(out.cpu().numpy(), ref) < tol


def test_batched_rejects_outputs_that_overlap_other_problems(idp):
    # the problems of a batch run concurrently: phi[i] overlapping rho[j] or phi[j]
    # (i != j) is refused before anything is queued
    import torch
    n = (17, 17, 17)
    plans = [idp.create_plan(3, n, (0.1, 0.1, 0.1), 6) for _ in range(2)]
    big = torch.zeros(3 * 17 ** 3, dtype=torch.float64, device=device())
    k = 17 ** 3
    rho0, rho1 = to_dev(np.zeros(n)), to_dev(np.zeros(n))
    cases = [([rho0, rho1], [big[:k], big[k // 2:k // 2 + k]]),      # outputs overlap
             ([rho0, big[:k]], [big[k // 2:k // 2 + k], big[2 * k:]])]   # an output overlaps another input
    for rhos, phis in cases:
        with pytest.raises(idp.IdpError) as e:
            idp.solve_batched(plans, rhos, phis)
        assert e.value.code == idp.IDP_EALIAS
    idp.solve_batched(plans, [rho0, rho1], [big[:k], big[k:2 * k]])
    for pl in plans:
        idp.plan_status(pl)


def test_alias_and_bad_arguments_are_rejected(idp):
    prob = w.c2_3d(33)
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    r = to_dev(prob.rho())
    with pytest.raises(idp.IdpError) as e:
        idp.solve(plan, r, r)
    assert e.value.code == idp.IDP_EALIAS
    with pytest.raises(idp.IdpError) as e:
        idp.solve_stage(plan, 99, r, to_dev(np.zeros(prob.n)))
    assert e.value.code == idp.IDP_EINVAL


def test_513_cube_large_grid(idp):
    # the largest supported grid (513^3, M = 512: 256-point sine FFTs and
    # 1024-point face FFTs): a sine mode through all three precision modes
    # (closed form), the boundary sum at sampled nodes (direct sum), and phi
    # of a bump against its exact potential (discretisation error ~1e-13 here)
    import torch
    n = (513, 513, 513)
    prob = w.scaled_bump(n, p=10)
    plan = idp.create_plan(3, n, prob.h, 6)
    x = [torch.linspace(-1, 1, 513, dtype=torch.float64, device=device())] * 3
    # low modes: the inverse Laplacian amplifies rounding in low modes by
    # lambda_mode / lambda_min, so a high mode would test conditioning, not the code
    rho = (torch.sin(3 * np.pi * (x[0][:, None, None] + 1) / 2) * torch.sin(5 * np.pi * (x[1][None, :, None] + 1) / 2)
           * torch.sin(7 * np.pi * (x[2][None, None, :] + 1) / 2))
    lam = (np.pi / 2) ** 2 * (9 + 25 + 49)
    out = torch.empty_like(rho)
    # mixed precision: FP32 accumulation of n = 511 terms per pass, stated
    # accuracy 1e-6 * sqrt(n_max) (see test_gpu_mixed.py)
    for prec, tol in ((idp.IDP_PRECISION_FP64, TOL), (idp.IDP_PRECISION_DF32, TOL),
                      (idp.IDP_PRECISION_MIXED_BF16X3, 1e-6 * np.sqrt(511))):
        idp.plan_set(plan, idp.IDP_KEY_PRECISION, prec)
        idp.solve_stage(plan, idp.IDP_STAGE_PHISTAR, rho, out)
        idp.plan_status(plan)
        err = ((out + rho / lam).abs().max() / (rho / lam).abs().max()).item()
        assert err < tol, (prec, err)
    del rho
    idp.plan_set(plan, idp.IDP_KEY_PRECISION, idp.IDP_PRECISION_FP64)
    rho_h = prob.rho()
    r = to_dev(rho_h)
    idp.solve_stage(plan, idp.IDP_STAGE_BOUNDARY, r, out)
    idp.plan_status(plan)
    idx = ogreens.boundary_indices(n)
    pick = idx[np.random.default_rng(9).choice(len(idx), 48, replace=False)]
    g = out.cpu().numpy()[tuple(pick.T)]
    assert rel_max(g, ogreens.boundary_direct(rho_h, prob.h, pick)) < TOL
    idp.solve(plan, r, out)
    idp.plan_status(plan)
    from oracle import closed_form
    # exact potential on every 4th node (129^3 points of the 513^3 grid)
    sub = w.scaled_bump((129, 129, 129), p=10)
    exact = closed_form.bump_potential_on_grid(sub)
    assert rel_max(out[::4, ::4, ::4].cpu().numpy(), exact) < 1e-11


_SHAPE_PROB = w.Problem("c", (65, 33, 129), (0.0, 0.0, 0.0), (1.0, 1.0, 2.0), "gauss", dict(seed=2108))
_SHAPE_REF = {}


def _solve_with_shape(idp, prob, shape):
    import torch
    plan = idp.create_plan(prob.d, prob.n, prob.h, 6)
    idp.plan_set(plan, idp.IDP_KEY_DST_SHAPE, shape)
    rho = to_dev(prob.rho())
    phi = torch.empty_like(rho)
    idp.solve(plan, rho, phi, None)
    torch.cuda.synchronize()
    idp.plan_status(plan)
    return phi.cpu().numpy()


@pytest.mark.parametrize("shape", [8, -8, 32, 16])
def test_dst_block_shapes_give_the_same_bits(idp, shape):
    # every block shape of the full-volume sine passes runs the same arithmetic per
    # line (M = 64, 32, 128 here: the 8-line, 128-thread and 32-line blocks apply,
    # 16 falls back): phi matches the oracle and the default shape bit for bit
    if "ref" not in _SHAPE_REF:
        _SHAPE_REF["ref"] = osolve.solve(_SHAPE_PROB.rho(), _SHAPE_PROB.h, 6, boundary="convolution")
        _SHAPE_REF["default"] = _solve_with_shape(idp, _SHAPE_PROB, 0)
    got = _solve_with_shape(idp, _SHAPE_PROB, shape)
    assert rel_max(got, _SHAPE_REF["ref"]) < TOL
    assert np.array_equal(got, _SHAPE_REF["default"])


_SHAPE_PROB_256 = w.Problem("c", (33, 17, 257), (0.0, 0.0, 0.0), (1.0, 0.5, 2.0), "gauss", dict(seed=2109))


@pytest.mark.parametrize("shape", [8, 16, 4])
def test_dst_block_shapes_at_m256_give_the_same_bits(idp, shape):
    # M = 256 along axis 2: the 16-line and the 4-line, 128-thread blocks apply there
    # (the FFT of a line by one warp, or by the block, in the same order of operations)
    if "ref256" not in _SHAPE_REF:
        _SHAPE_REF["ref256"] = osolve.solve(_SHAPE_PROB_256.rho(), _SHAPE_PROB_256.h, 6, boundary="convolution")
        _SHAPE_REF["default256"] = _solve_with_shape(idp, _SHAPE_PROB_256, 0)
    got = _solve_with_shape(idp, _SHAPE_PROB_256, shape)
    assert rel_max(got, _SHAPE_REF["ref256"]) < TOL
    assert np.array_equal(got, _SHAPE_REF["default256"])


def test_dst_shape_key_rejects_unknown_values(idp):
    plan = idp.create_plan(3, (33, 33, 33), (0.1, 0.1, 0.1), 6)
    lib = idp.library()
    assert lib.idp_plan_set(plan.handle, idp.IDP_KEY_DST_SHAPE, 3) == idp.IDP_EINVAL


# d = 1 (section 5): phi* by the sine series, g at the two ends, and the
# straight line through them; every panel-count family and the largest size
ONE_D = [
    ("1d_17_bump", w.scaled_bump((17,), centre=(0.1,), eps=0.6, p=10)),
    ("1d_65_gauss", w.Problem("o1", (65,), (0.0,), (2.0,), "gauss", dict(seed=5))),
    ("1d_97_random", w.Problem("o2", (97,), (-1.0,), (0.5,), "random", dict(seed=9))),
    ("1d_129_points", w.Problem("o3", (129,), (0.0,), (1.0,), "points", dict(seed=13, count=3))),
    ("1d_385_gauss", w.Problem("o4", (385,), (-3.0,), (1.0,), "gauss", dict(seed=21))),
    ("1d_513_random", w.Problem("o5", (513,), (0.0,), (4.0,), "random", dict(seed=4))),
]


@pytest.mark.parametrize("name,prob", ONE_D, ids=[c[0] for c in ONE_D])
def test_one_dimensional_solve_matches_oracle(idp, name, prob):
    rho = prob.rho()
    parts = {}
    ref = osolve.solve(rho, prob.h, 6, parts=parts)
    line = ref - parts["phistar"]          # the oracle's straight line, g at the ends
    plan = idp.create_plan(1, prob.n, prob.h, 6)
    r = to_dev(rho)
    g = run_stage(idp, plan, idp.IDP_STAGE_BOUNDARY, r, prob.n)
    assert rel_max(g[[0, -1]], parts["g"][[0, -1]]) < TOL
    assert np.all(g[1:-1] == 0)
    ps = run_stage(idp, plan, idp.IDP_STAGE_PHISTAR, r, prob.n)
    assert rel_max(ps, parts["phistar"]) < TOL
    assert ps[0] == 0 and ps[-1] == 0
    u1 = run_stage(idp, plan, idp.IDP_STAGE_U1, r, prob.n)
    assert rel_max(u1, line) < TOL
    phi = run_stage(idp, plan, idp.IDP_STAGE_PHI, r, prob.n)
    assert rel_max(phi, ref) < TOL
    out = to_dev(np.zeros(prob.n))
    idp.solve(plan, r, out)
    idp.plan_status(plan)
    assert np.array_equal(out.cpu().numpy(), phi)
    # order has no effect in 1-D
    plan4 = idp.create_plan(1, prob.n, prob.h, 4)
    out4 = to_dev(np.zeros(prob.n))
    idp.solve(plan4, r, out4)
    idp.plan_status(plan4)
    assert np.array_equal(out4.cpu().numpy(), phi)


def test_one_dimensional_edge_cases(idp):
    n, h = (65,), (0.03,)
    plan = idp.create_plan(1, n, h, 6)
    # zero density, and values only on the two boundary entries (ignored): phi = 0
    for rho in (np.zeros(n), np.array([3.0] + [0.0] * 63 + [-2.0])):
        out = to_dev(np.full(n, 7.0))
        idp.solve(plan, to_dev(rho), out)
        idp.plan_status(plan)
        assert np.all(out.cpu().numpy() == 0)
    # stages without a 1-D meaning, and reduced precision, are refused
    r = to_dev(w.random_interior(n, seed=3))
    for stage in (idp.IDP_STAGE_GTILDE, idp.IDP_STAGE_R):
        with pytest.raises(idp.IdpError) as e:
            run_stage(idp, plan, stage, r, (63,))
        assert e.value.code == idp.IDP_ESUPPORT
    for prec in (idp.IDP_PRECISION_DF32, idp.IDP_PRECISION_MIXED_BF16X3):
        with pytest.raises(idp.IdpError) as e:
            idp.plan_set(plan, idp.IDP_KEY_PRECISION, prec)
        assert e.value.code == idp.IDP_ESUPPORT
    idp.plan_set(plan, idp.IDP_KEY_AUTOTUNE, 1)


def test_one_dimensional_host_and_batched_give_the_device_bits(idp):
    import torch
    p1 = w.Problem("o6", (257,), (-1.0,), (1.0,), "gauss", dict(seed=8))
    p3 = w.c2_3d(33)
    plans = [idp.create_plan(1, p1.n, p1.h, 6), idp.create_plan(3, p3.n, p3.h, 6)]
    rhos = [to_dev(p1.rho()), to_dev(p3.rho())]
    refs = []
    for pl, r, pr in zip(plans, rhos, (p1, p3)):
        o = to_dev(np.zeros(pr.n))
        idp.solve(pl, r, o)
        idp.plan_status(pl)
        refs.append(o.cpu().numpy())
    outs = [to_dev(np.zeros(p1.n)), to_dev(np.zeros(p3.n))]
    idp.solve_batched(plans, rhos, outs)
    torch.cuda.synchronize()
    for pl in plans:
        idp.plan_status(pl)
    for o, ref in zip(outs, refs):
        assert np.array_equal(o.cpu().numpy(), ref)
    rho_p = torch.from_numpy(p1.rho()).pin_memory()
    phi_p = torch.zeros(p1.n, dtype=torch.float64).pin_memory()
    for _ in range(2):
        phi_p.zero_()
        idp.solve_host(plans[0], rho_p.data_ptr(), phi_p.data_ptr())
        idp.plan_status(plans[0])
        assert np.array_equal(phi_p.numpy(), refs[0])


# Automatic padding (section 2: a panel count the transforms do not take is met
# by extending the domain by a few panels, h unchanged)
PADDED = [
    ("3d_41x50x37", w.Problem("p1", (41, 50, 37), (-1.0, -1.2, -0.9), (1.0, 1.25, 0.9), "bump",
                              dict(centre=(0.05, 0.0, 0.02), eps=0.6, p=10))),
    ("2d_70x45", w.Problem("p2", (70, 45), (-1.0, -0.7), (1.2, 0.7), "bump",
                           dict(centre=(0.1, 0.0), eps=0.55, p=8))),
    ("1d_100", w.Problem("p3", (100,), (-1.0,), (1.0,), "bump", dict(centre=(0.1,), eps=0.6, p=10))),
    ("3d_20x129x33", w.Problem("p4", (20, 129, 33), (0.0, 0.0, 0.0), (0.6, 4.0, 1.0), "gauss",
                               dict(seed=17))),
]
SUPPORTED = (16, 32, 48, 64, 96, 128, 192, 256, 384, 512)


def _embed(rho, n_solved, off):
    """The padded rho the library builds: the caller's interior values at their
    nodes of the larger grid, zero elsewhere."""
    out = np.zeros(n_solved)
    inner = tuple(slice(1, k - 1) for k in rho.shape)
    dst = tuple(slice(o + 1, o + k - 1) for o, k in zip(off, rho.shape))
    out[dst] = rho[inner]
    return out


def _restrict(phi, n, off):
    return phi[tuple(slice(o, o + k) for o, k in zip(off, n))]


@pytest.mark.parametrize("name,prob", PADDED, ids=[c[0] for c in PADDED])
def test_padded_plan_matches_the_oracle_on_the_padded_grid(idp, name, prob):
    rho = prob.rho()
    plan = idp.create_plan(prob.d, prob.n, prob.h, 6)
    n_solved, off = idp.plan_grid(plan)
    for k, m, o in zip(prob.n, n_solved, off):
        M = k - 1
        assert m - 1 == min(s for s in SUPPORTED if s >= M) and o == (m - 1 - M) // 2
    assert idp.plan_info(plan)["nodes"] == int(np.prod(prob.n))
    out = to_dev(np.zeros(prob.n))
    idp.solve(plan, to_dev(rho), out)
    idp.plan_status(plan)
    ref = _restrict(osolve.solve(_embed(rho, n_solved, off), prob.h, 6,
                                 boundary="convolution" if prob.d > 1 else "direct"), prob.n, off)
    assert rel_max(out.cpu().numpy(), ref) < TOL
    # the caller's boundary entries of rho are not used, as in an unpadded solve
    rho_b = rho.copy()
    for s in range(prob.d):
        idx = [slice(None)] * prob.d
        idx[s] = 0
        rho_b[tuple(idx)] = 5.0
    out_b = to_dev(np.zeros(prob.n))
    idp.solve(plan, to_dev(rho_b), out_b)
    idp.plan_status(plan)
    assert np.array_equal(out_b.cpu().numpy(), out.cpu().numpy())
    # full solves only
    with pytest.raises(idp.IdpError) as e:
        run_stage(idp, plan, idp.IDP_STAGE_BOUNDARY, to_dev(rho), prob.n)
    assert e.value.code == idp.IDP_ESUPPORT


@pytest.mark.parametrize("name,prob", PADDED[:3], ids=[c[0] for c in PADDED[:3]])
def test_padded_solve_is_as_accurate_as_the_unpadded_method(idp, name, prob):
    # against the exact free-space potential of the bump: the padded GPU solve
    # and the oracle on the caller's own (unpadded) grid have errors of the same size
    from oracle import closed_form
    from tests.test_oracle_full import _bump_potential_1d
    rho = prob.rho()
    if prob.d == 1:
        ex = _bump_potential_1d(prob.coords()[0], prob.params["centre"][0], prob.params["eps"], prob.params["p"])
    else:
        ex = closed_form.bump_potential_on_grid(prob)
    plan = idp.create_plan(prob.d, prob.n, prob.h, 6)
    out = to_dev(np.zeros(prob.n))
    idp.solve(plan, to_dev(rho), out)
    idp.plan_status(plan)
    err_pad = rel_max(out.cpu().numpy(), ex)
    err_own = rel_max(osolve.solve(rho, prob.h, 6, boundary="convolution" if prob.d > 1 else "direct"), ex)
    print("padding", name, err_pad, err_own)
    assert err_pad < 3 * err_own + 1e-13


def test_padded_host_and_batched_give_the_device_bits(idp):
    import torch
    probs = [PADDED[0][1], w.c2_3d(33), PADDED[2][1]]
    plans = [idp.create_plan(p.d, p.n, p.h, 6) for p in probs]
    rhos = [to_dev(p.rho()) for p in probs]
    refs = []
    for pl, r, pr in zip(plans, rhos, probs):
        o = to_dev(np.zeros(pr.n))
        idp.solve(pl, r, o)
        idp.plan_status(pl)
        refs.append(o.cpu().numpy())
    outs = [to_dev(np.zeros(p.n)) for p in probs]
    idp.solve_batched(plans, rhos, outs)
    torch.cuda.synchronize()
    for pl in plans:
        idp.plan_status(pl)
    for o, ref in zip(outs, refs):
        assert np.array_equal(o.cpu().numpy(), ref)
    for k in (0, 2):
        rho_p = torch.from_numpy(probs[k].rho()).pin_memory()
        phi_p = torch.zeros(probs[k].n, dtype=torch.float64).pin_memory()
        for _ in range(2):
            phi_p.zero_()
            idp.solve_host(plans[k], rho_p.data_ptr(), phi_p.data_ptr())
            idp.plan_status(plans[k])
            assert np.array_equal(phi_p.numpy(), refs[k])


def _status(idp, plan):
    try:
        idp.plan_status(plan)
        return idp.IDP_OK
    except idp.IdpError as e:
        return e.code


def test_validation_mode_reports_bad_densities(idp):
    # IDP_KEY_VALIDATE = k: NaN/inf in rho -> IDP_EINVAL, non-zero rho on a node
    # within k layers of the boundary -> IDP_ESUPPORT, each reported once by
    # idp_plan_status; the boundary entries of rho are not checked (not used)
    import torch
    prob = w.c2_3d(33)
    rho = prob.rho()
    plan = idp.create_plan(3, prob.n, prob.h, 6)
    ref = to_dev(np.zeros(prob.n))
    idp.solve(plan, to_dev(rho), ref)
    idp.plan_status(plan)
    idp.plan_set(plan, idp.IDP_KEY_VALIDATE, 3)

    def run(r, pl=plan, shape=prob.n):
        out = to_dev(np.zeros(shape))
        idp.solve(pl, to_dev(r), out)
        return _status(idp, pl), out

    code, out = run(rho)
    assert code == idp.IDP_OK and np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
    near = rho.copy()
    near[2, 16, 16] = 1.0                       # 2 layers from the face i0 = 0
    assert run(near)[0] == idp.IDP_ESUPPORT
    assert _status(idp, plan) == idp.IDP_OK     # reported once
    far = rho.copy()
    far[3, 16, 16] = 1.0                        # 3 layers: allowed with k = 3
    assert run(far)[0] == idp.IDP_OK
    bad = rho.copy()
    bad[16, 16, 16] = np.nan
    assert run(bad)[0] == idp.IDP_EINVAL
    both = near.copy()
    both[16, 16, 31] = np.inf
    assert run(both)[0] == idp.IDP_EINVAL       # NaN/inf is reported first
    edge = rho.copy()
    edge[0, 16, 16] = 5.0                       # a boundary entry: not used, not checked
    assert run(edge)[0] == idp.IDP_OK
    idp.plan_set(plan, idp.IDP_KEY_VALIDATE, 0)
    assert run(near)[0] == idp.IDP_OK           # validation off
    # host buffers, a 2-D, a 1-D and a padded plan check the caller's grid too
    idp.plan_set(plan, idp.IDP_KEY_VALIDATE, 3)
    rp = torch.from_numpy(near).pin_memory()
    pp = torch.zeros(prob.n, dtype=torch.float64).pin_memory()
    idp.solve_host(plan, rp.data_ptr(), pp.data_ptr())
    assert _status(idp, plan) == idp.IDP_ESUPPORT
    for n in ((33, 65), (129,), (41, 50, 37)):
        p2 = w.random_interior(n, seed=5, margin=4)
        pl = idp.create_plan(len(n), n, (0.01,) * len(n), 6)
        idp.plan_set(pl, idp.IDP_KEY_VALIDATE, 4)
        assert run(p2, pl, n)[0] == idp.IDP_OK
        q = p2.copy()
        q[(1,) * len(n)] = 0.5                  # the corner-most interior node
        assert run(q, pl, n)[0] == idp.IDP_ESUPPORT
    with pytest.raises(idp.IdpError) as e:
        idp.plan_set(plan, idp.IDP_KEY_VALIDATE, -1)
    assert e.value.code == idp.IDP_EINVAL


@pytest.mark.parametrize("d", [2, 3])
def test_zero_and_single_point_densities(idp, d):
    # the degenerate inputs: rho = 0 gives phi = 0 exactly (every line and slice is
    # skipped), and a single non-zero node (one line, one slice per axis) matches
    # the oracle; values on the boundary entries of rho are not used
    n = (33, 17, 49)[:d] if d == 3 else (33, 49)
    h = (0.05, 0.07, 0.03)[:d]
    plan = idp.create_plan(d, n, h, 6)
    out = to_dev(np.full(n, 3.0))
    idp.solve(plan, to_dev(np.zeros(n)), out)
    idp.plan_status(plan)
    assert np.all(out.cpu().numpy() == 0)
    rho = np.zeros(n)
    rho[tuple(k // 2 for k in n)] = 1.0
    rho[(0,) * d] = 7.0                       # a boundary entry: ignored
    out = to_dev(np.zeros(n))
    idp.solve(plan, to_dev(rho), out)
    idp.plan_status(plan)
    rho0 = rho.copy()
    rho0[(0,) * d] = 0.0
    ref = osolve.solve(rho0, h, 6, boundary="convolution")
    assert rel_max(out.cpu().numpy(), ref) < TOL


@pytest.mark.parametrize("n", [(3,), (3, 3), (3, 3, 3), (3, 18, 5)])
def test_smallest_grids(idp, n):
    # n = 3 nodes per axis (one interior node): padded to 16 panels (section 2),
    # phi at the caller's nodes equals the oracle's on the padded grid
    d = len(n)
    h = (0.1, 0.13, 0.07)[:d]
    rho = np.zeros(n)
    rho[tuple(1 if k == 3 else k // 2 for k in n)] = 1.0
    plan = idp.create_plan(d, n, h, 6)
    n_solved, off = idp.plan_grid(plan)
    out = to_dev(np.zeros(n))
    idp.solve(plan, to_dev(rho), out)
    idp.plan_status(plan)
    ref = _restrict(osolve.solve(_embed(rho, n_solved, off), h, 6,
                                 boundary="convolution" if d > 1 else "direct"), n, off)
    assert rel_max(out.cpu().numpy(), ref) < TOL
