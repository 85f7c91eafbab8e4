"""Throughput of the infinite-domain Poisson solve (grid points / s at 6th order).

Headline workload (the largest single-GPU configuration): 513^3 nodes on
[0,2]x[0,1]x[0,1] (anisotropic h), rho = a sum of 6 seeded Gaussians tapered to
zero near the edges, order 6, FP64.  Inputs are synthetic, generated on the
host and resident in HBM before timing.  One step = one complete solve
phi = phi* + phi_H (boundary convolutions, sine solves, 6th-order correction)
through the C ABI.  The same JSON line also carries the mixed-precision and
double-float variants of that workload, the 129^3 bump workload, the precision
sweep at 257^3 with every variant's error against the oracle, the 96-problem
batched workload, and two CPU baselines.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large|bump|sweep|sweep_long] [--n N] [--headline-only]

--impl reference times the CPU oracle on the host cores (the reference arm of
this comparison: there is no runnable reference implementation, only the
paper).  One JSON line is printed by rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

METRIC = "grid points/s at 6th order, FP64 vs mixed-precision at stated max error"
UNIT = "grid points/s"
L2_FLUSH_BYTES = 512 << 20          # > 129 MB of L2
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 4 FP64 flop/clk x 2.07 GHz
FP64_PROBE_TFLOPS = 1.198           # FMA-chain probe on this GPU model, 1995 MHz
KERNEL_NAMES = {1: "dst_pass", 2: "rfft", 3: "face", 4: "face_invb", 5: "face_c2r", 6: "gtilde_layers",
                7: "rhs6_w", 8: "rhs6_core", 9: "rhs6_extrap", 10: "gtilde_expand", 11: "dst_pass_layers",
                12: "mixed_pass", 13: "support_flags", 14: "rhs6_expand", 15: "line1d", 16: "pad",
                17: "validate"}
# DRAM bytes (read + write) per full-volume launch of the FP64 sine pass, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum over the 8 passes of one solve,
# averaged); a grid not listed reports null
# (profiles/dst_pass_fp64_257cube_traffic.md: 248.5 MB per launch at 257^3, scaled by the
# interior points to 513^3)
DST_TRAFFIC = {(257, 257, 257): 248.5e6, (513, 513, 513): 2.00e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None,
                    help="nodes per axis (default: 513 large, 129 bump, 257 sweep)")
    ap.add_argument("--workload", default="large", choices=["large", "bump", "sweep", "sweep_long"],
                    help="large: 6-Gaussian sum on [0,2]x[0,1]^2 (the headline); bump: 3-D bump on "
                         "[-1,1]^3; sweep / sweep_long: Gaussian sum on [0,1]^3 with (n-2)^3 / "
                         "(1.5(n-1)-1)x(n-2)^2 interior nodes")
    ap.add_argument("--order", type=int, default=6)
    ap.add_argument("--fp64-only", action="store_true", help="skip the reduced-precision variants")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the 129^3, sweep and batched workloads and the CPU baselines")
    ap.add_argument("--dst-shape", type=int, default=None, choices=[0, 8, -8, 32, 16, 4],
                    help="block shape of the FP64 sine passes (IDP_KEY_DST_SHAPE) instead of the "
                         "autotuner's: profiled runs, whose timings the profiler perturbs, then run "
                         "the shape of the plain run")
    ap.add_argument("--profile-window", type=int, default=0,
                    help="after the timed steps, run this many more solves between "
                         "cudaProfilerStart and cudaProfilerStop (for ncu --profile-from-start off)")
    ap.add_argument("--profile-precision", default="FP64",
                    choices=["FP64", "DF32", "MIXED_BF16X3", "MIXED_TF32X3"],
                    help="precision mode of the solves in the profiler window (an autotuned plan of "
                         "its own unless FP64)")
    ap.add_argument("--nvtx", action="store_true",
                    help="the solves in the profiler window with NVTX ranges around their launches and "
                         "stages (IDP_KEY_NVTX; plain launches)")
    ap.add_argument("--batched", action="store_true",
                    help="only the 96-problem batched workload (uneven sizes)")
    return ap.parse_args()


DEFAULT_N = {"bump": 129, "large": 513, "sweep": 257, "sweep_long": 257}


def workload(kind, n=None):
    n = n or DEFAULT_N[kind]
    if kind == "bump":
        return w.c2_3d(n)
    if kind == "large":
        return w.c3_large(n)
    if kind == "sweep":
        return w.c4_sweep((n - 2,) * 3)
    return w.c4_sweep((3 * (n - 1) // 2 - 1, n - 2, n - 2))


def describe(prob, order):
    dims = "x".join(str(k) for k in prob.n)
    box = "x".join("[%g,%g]" % (a, b) for a, b in zip(prob.lo, prob.hi))
    if prob.density == "bump":
        dens = "bump (1-r^2/0.49)^10, r<0.7, centre (0.05,0.1,-0.08)"
    else:
        dens = "6 Gaussians (seed 2108, centres in [0.3,0.7] box-relative, sigma U[0.04,0.1], " \
               "amplitudes U[-1,1]), tapered to zero within 0.15 of each edge"
    return "3-D FP64 order-%d solve, %s nodes on %s, %s" % (order, dims, box, dens)


def config_of(prob, order, extra=None):
    c = {"workload": describe(prob, order),
         "nodes": prob.points, "order": order, "grid": list(prob.n), "h": list(prob.h),
         "l2": "flushed between timed steps (512 MiB write)" + (
             "; inputs and workspace also exceed L2" if prob.points * 8 > (129 << 20) else "")}
    if extra:
        c.update(extra)
    return c


# ----------------------------------------------------------------------------- multi-rank helpers
def shard(items, rank, world):
    """Problems of rank `rank`: a size-balanced greedy split (largest problem first,
    each to the rank with the fewest nodes so far, ties to the lower rank), which
    every rank computes alike, so the batched workload needs no collective.  The
    problems keep their order within a rank."""
    load = [0] * world
    owner = [0] * len(items)
    for i in sorted(range(len(items)), key=lambda i: (-items[i].points, i)):
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += items[i].points
    return [it for it, o in zip(items, owner) if o == rank]


def max_over_ranks(value, world, device=None):
    """Largest `value` over all ranks (the job time is the slowest rank's)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU legs
def oracle_step(rho, h, order):
    from oracle import solve as osolve
    t = time.perf_counter()
    osolve.solve(rho, h, order, boundary="convolution")
    return time.perf_counter() - t


def reference_sample(prob, kind):
    """The oracle's bounded sample of a workload: the workload itself up to 129^3,
    else the same density family at 129^3 (the oracle's direct sine sums grow as n^4)."""
    return prob if max(prob.n) <= 129 else workload(kind, 129)


def cpu_baseline(prob, order, kind, budget_s=10.0):
    """Complete oracle solves of a bounded sample of the workload, repeated for
    about `budget_s` seconds (at least 2)."""
    sample = reference_sample(prob, kind)
    rho = sample.rho()
    ts = [oracle_step(rho, sample.h, order)]
    while len(ts) < 2 or sum(ts) < budget_s:
        ts.append(oracle_step(rho, sample.h, order))
    t = statistics.mean(ts)
    what = "the same" if sample is prob else "a 129^3-node sample (same domain and density family) of the"
    return {"value": sample.points / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d complete oracle solves (convolution form of the boundary sum, numpy BLAS sine "
                      "sums) of %s %s-node workload, %.2f s each" % (len(ts), what,
                                                                    "x".join(map(str, prob.n)), t)}


def cpu_paper_method(prob, order, kind):
    """The method with fast transforms on the host cores (scipy's multithreaded
    DST-I and FFT convolutions, the paper's FFTW setup of section 6), one solve
    of the workload, or of a 257^3 sample of it above 257^3."""
    try:
        from oracle import fft_baseline
    except ImportError as e:   # scipy missing on the host
        return {"value": None, "unit": UNIT, "unavailable": str(e)}
    sample = prob if max(prob.n) <= 257 else workload(kind, 257)
    rho = sample.rho()
    t = time.perf_counter()
    fft_baseline.solve(rho, sample.h, order, workers=os.cpu_count())
    t = time.perf_counter() - t
    what = "the" if sample is prob else "a 257^3-node sample (same domain and density family) of the"
    return {"value": sample.points / t, "unit": UNIT, "cores": os.cpu_count(),
            "kind": "fast transforms: scipy.fft DST-I and FFT convolutions, all host cores",
            "sample": "one solve of %s %s-node workload, %.2f s" % (what, "x".join(map(str, prob.n)), t)}


def run_reference(args, rank, world):
    prob = workload(args.workload, args.n)
    if rank != 0:
        return
    sample = reference_sample(prob, args.workload)
    rho = sample.rho()
    for _ in range(args.warmup):
        oracle_step(rho, sample.h, args.order)
    ts = [oracle_step(rho, sample.h, args.order) for _ in range(args.steps)]
    t = sum(ts)
    value = sample.points * args.steps / t
    what = "the workload" if sample is prob else "a 129^3-node sample (same domain and density family) " \
                                                 "of the workload"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_of(prob, args.order),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "%d complete oracle solves of %s" % (args.steps, what)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def dst_flops_per_launch(prob):
    """Algorithmic FP64 flops of one sine-transform pass, averaged over the three
    axes: 2.5 log2(2 M_s) per interior point."""
    lg = np.mean([np.log2(2 * (k - 1)) for k in prob.n])
    return 2.5 * lg * float(np.prod([k - 2 for k in prob.n]))


class Gpu:
    """Device, stream, L2 flush buffer and the timing helpers of the GPU arm."""

    def __init__(self, world):
        import torch
        import paper_2108_11871_gb300 as idp
        self.torch, self.idp, self.world = torch, idp, world
        self.local = int(os.environ.get("LOCAL_RANK", 0))
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.stream = torch.cuda.current_stream(self.dev)
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=self.dev)

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def plan(self, prob, order, prec=None, shape=None, bdd=False, exact=False):
        idp = self.idp
        plan = idp.create_plan(prob.d, prob.n, prob.h, order, exact=exact)
        if prec is not None:
            idp.plan_set(plan, idp.IDP_KEY_PRECISION, prec)
        if bdd:
            idp.plan_set(plan, idp.IDP_KEY_MIXED_BOUNDARY_DF32, 1)
        idp.plan_set(plan, idp.IDP_KEY_AUTOTUNE, 1)
        if shape is not None:
            idp.plan_set(plan, idp.IDP_KEY_DST_SHAPE, shape)
        return plan

    def timed(self, fn, steps, warmup):
        """Per-step ms of `fn()` by CUDA events on the launch stream, the L2
        flushed before each step (outside the events)."""
        torch = self.torch
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = []
        for i in range(steps):
            self.flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            fn()
            b.record(self.stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    def kernels(self, plan, rho, phi, reps=3):
        """Per-kernel durations of `reps` solves with plain launches (CUDA events on
        the launch stream): {family: [ms of each launch]}."""
        import ctypes
        idp = self.idp
        cap = 256
        kinds = (ctypes.c_int * cap)()
        ms = (ctypes.c_float * cap)()
        out = {}
        for i in range(reps):
            self.flush.fill_(float(i))
            n = idp.library().idp_profile_solve(plan.handle, ctypes.c_void_p(rho.data_ptr()),
                                                ctypes.c_void_p(phi.data_ptr()),
                                                ctypes.c_void_p(self.stream.cuda_stream), cap, kinds, ms)
            if n < 0:
                raise RuntimeError("idp_profile_solve: %s" % idp.strerror(n))
            for j in range(n):
                out.setdefault(KERNEL_NAMES.get(kinds[j], str(kinds[j])), []).append(ms[j])
        return out

    def launches(self, plan):
        import ctypes
        v = ctypes.c_int64()
        self.idp.library().idp_plan_launches(plan.handle, ctypes.byref(v))
        return int(v.value)


def rel(a, b):
    return float((a - b).abs().max().item() / b.abs().max().item())


def variant_record(g, prob, order, prec, label, rho, phi_ref, steps, warmup, bdd=False, exact=False):
    """A reduced-precision variant of the workload: throughput, per-kernel times and
    its max difference from the FP64 result (or from phi_ref)."""
    idp = g.idp
    plan = g.plan(prob, order, prec, bdd=bdd, exact=exact)
    phi = g.torch.empty_like(rho)
    ms = g.timed(lambda: idp.solve(plan, rho, phi, g.stream), steps, warmup)
    idp.plan_status(plan)
    t = max_over_ranks(sum(ms), g.world, g.dev)
    ks = g.kernels(plan, rho, phi)
    rec = {"variant": label, "tuning": idp.plan_tuning(plan),
           "value": g.world * prob.points * steps / (t / 1e3), "unit": UNIT, "ms_per_step": t / steps,
           "max_rel_error_vs_fp64": rel(phi, phi_ref) if phi_ref is not None else None,
           "kernel_ms_per_step": {k: sum(v) / 3 for k, v in ks.items()}}
    for fam in ("mixed_pass", "dst_pass"):
        if fam in ks:
            rec[fam + "_avg_ms"] = statistics.mean(ks[fam])
    del plan
    return phi, rec


VARIANTS = (("mixed_precision", "MIXED_BF16X3",
             "bf16x3 pieces, fp32 accumulate, tcgen05 (rho, R and final transforms)"),
            ("mixed_tf32x3", "MIXED_TF32X3",
             "tf32x3: two tf32 pieces, products hi*hi + hi*lo + lo*hi, fp32 accumulate, tcgen05 "
             "kind::tf32 (rho, R and final transforms)"),
            ("df32", "DF32", "double-float (FP32 pairs) FFT arithmetic"),
            ("mixed_df32_boundary", "MIXED_BF16X3",
             "bf16x3 tensor-core transforms as mixed_precision, with the 3-D boundary convolutions in "
             "double-float arithmetic (IDP_KEY_MIXED_BOUNDARY_DF32)"))


def run_headline(g, args, prob):
    """The workload's FP64 solve (the line's value), its variants, e2e and roofline."""
    idp, torch = g.idp, g.torch
    plan = g.plan(prob, args.order, shape=args.dst_shape)
    rho_h = prob.rho()
    rho = torch.from_numpy(rho_h).to(g.dev)
    phi = torch.empty_like(rho)
    g.barrier()
    with ClockSampler(g.local) as clk:
        ms = g.timed(lambda: idp.solve(plan, rho, phi, g.stream), args.steps, args.warmup)
    g.barrier()
    idp.plan_status(plan)
    total_ms = max_over_ranks(sum(ms), g.world, g.dev)
    out = {"value": g.world * prob.points * args.steps / (total_ms / 1e3),
           "ms_per_step": total_ms / args.steps, "clocks": clk.summary(),
           "gpu_launches": g.launches(plan) * args.steps}

    ks = g.kernels(plan, rho, phi, reps=max(3, min(args.steps, 10)))
    reps = max(3, min(args.steps, 10))
    out["kernel_ms_per_step"] = {k: sum(v) / reps for k, v in ks.items()}
    out["dominant_kernel"] = max(ks, key=lambda k: sum(ks[k]))
    dst_ms = statistics.mean(ks["dst_pass"])
    achieved = dst_flops_per_launch(prob) / (dst_ms / 1e3) / 1e12
    out["roofline"] = {"bound": "alu", "kernel": "dst_pass (FP64 sine-transform pass)",
                       "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": achieved / FP64_PEAK_TFLOPS,
                       "peak_note": "FP64 derived: 152 SMs x 4 flop/clk x 2.07 GHz; "
                                    "FMA-chain probe measured %.3f" % FP64_PROBE_TFLOPS,
                       "traffic": DST_TRAFFIC.get(tuple(prob.n)), "avg_launch_ms": dst_ms,
                       "flops_per_launch": dst_flops_per_launch(prob)}
    out["tuning"] = idp.plan_tuning(plan)
    # the boundary sums' share of the solve (the real FFTs, face passes and their
    # inverses: rows a3 of the method), and the phi* solve alone (rows a1 + a2:
    # forward DST of rho, eigenvalue division, inverse DST; IDP_STAGE_PHISTAR)
    kt = out["kernel_ms_per_step"]
    bnd = sum(kt.get(k, 0.0) for k in ("rfft", "face", "face_invb", "face_c2r"))
    out["boundary_share"] = bnd / sum(kt.values())
    # (into a buffer of its own: phi holds the solve, which the accuracy checks below read)
    phs = torch.empty_like(rho)
    psm = g.timed(lambda: idp.solve_stage(plan, idp.IDP_STAGE_PHISTAR, rho, phs, g.stream), args.steps, args.warmup)
    idp.plan_status(plan)
    del phs
    ps_ms = max_over_ranks(sum(psm), g.world, g.dev) / args.steps
    out["phi_star_solve"] = {"value": g.world * prob.points / (ps_ms / 1e3), "unit": UNIT, "ms_per_step": ps_ms,
                             "what": "phi* alone: forward DST of rho, eigenvalue division, inverse DST "
                                     "(idp_solve_stage IDP_STAGE_PHISTAR, plain launches)"}

    if args.profile_window > 0:
        # a window of solves for a profiler that starts collecting here
        wplan = plan if args.profile_precision == "FP64" else \
            g.plan(prob, args.order, getattr(idp, "IDP_PRECISION_" + args.profile_precision))
        wphi = torch.empty_like(rho)
        if args.nvtx:
            idp.plan_set(wplan, idp.IDP_KEY_NVTX, 1)
        idp.solve(wplan, rho, wphi, g.stream)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        for i in range(args.profile_window):
            g.flush.fill_(float(i))
            idp.solve(wplan, rho, wphi, g.stream)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        if args.nvtx:
            idp.plan_set(wplan, idp.IDP_KEY_NVTX, 0)
        del wplan, wphi

    # end to end through the host-buffer entry point (pinned host memory, both
    # copies inside the timed region)
    rho_pin = torch.from_numpy(rho_h).pin_memory()
    phi_pin = torch.empty_like(rho_pin).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    idp.solve_host(plan, rho_pin.data_ptr(), phi_pin.data_ptr(), g.stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        idp.solve_host(plan, rho_pin.data_ptr(), phi_pin.data_ptr(), g.stream)
    torch.cuda.synchronize()
    e2e_t = max_over_ranks((time.perf_counter() - t0) / e2e_steps, g.world, g.dev)
    out["e2e"] = {"value": g.world * prob.points / e2e_t, "unit": UNIT,
                  "h2d_bytes_per_step": 8 * prob.points, "d2h_bytes_per_step": 8 * prob.points}
    del rho_pin, phi_pin

    # FP64 accuracy evidence at full size: g against the direct trapezoid sum
    # (eq. TrapOrig2D) on sampled boundary nodes; the bump also against its exact
    # potential
    from oracle import greens as ogreens
    gstage = torch.empty_like(rho)
    idp.solve_stage(plan, idp.IDP_STAGE_BOUNDARY, rho, gstage, g.stream)
    idp.plan_status(plan)
    idx = ogreens.boundary_indices(prob.n)
    pick = idx[np.random.default_rng(7).choice(len(idx), 64 if prob.points > 3e7 else 512, replace=False)]
    gsamp = gstage.cpu().numpy()[tuple(pick.T)]
    gref = ogreens.boundary_direct(rho_h, prob.h, pick)
    prec = {"variant": "fp64", "g_vs_direct_sum": float(np.abs(gsamp - gref).max() / np.abs(gref).max()),
            "g_sample": "%d seeded boundary nodes" % len(pick)}
    del gstage
    if prob.density == "bump":
        from oracle import closed_form
        stride = 1 if prob.n[0] <= 129 else 4
        sub = w.Problem(prob.name, tuple(len(range(0, k, stride)) for k in prob.n), prob.lo,
                        tuple(lo + (len(range(0, k, stride)) - 1) * stride * hh
                              for lo, k, hh in zip(prob.lo, prob.n, prob.h)), prob.density, prob.params)
        exact = closed_form.bump_potential_on_grid(sub)
        o = phi[::stride, ::stride, ::stride].cpu().numpy()
        prec["max_rel_error_vs_exact_potential"] = float(np.abs(o - exact).max() / np.abs(exact).max())
    out["precision"] = prec
    del plan

    phis = {}
    if not args.fp64_only:
        for key, name, label in VARIANTS:
            ph, rec = variant_record(g, prob, args.order, getattr(idp, "IDP_PRECISION_" + name), label, rho, phi,
                                     args.steps, args.warmup, bdd=key == "mixed_df32_boundary")
            out[key] = rec
            phis[key] = ph
    return out, rho_h, phi, phis


def run_sweep(g, args):
    """The precision sweep at its nearest supported size (257^3 nodes, interior
    255^3): FP64 and every variant, each with its error against the oracle."""
    from oracle import solve as osolve
    prob = workload("sweep")
    head, rho_h, phi, phis = run_headline(g, argparse.Namespace(**{**vars(args), "profile_window": 0,
                                                                   "dst_shape": None}), prob)
    ref = osolve.solve(rho_h, prob.h, args.order, boundary="convolution")
    scale = np.abs(ref).max()
    rec = {"workload": describe(prob, args.order), "value": head["value"], "ms_per_step": head["ms_per_step"],
           "max_rel_error_vs_oracle": float(np.abs(phi.cpu().numpy() - ref).max() / scale)}
    for key, _, _ in VARIANTS:
        if key in head:
            rec[key] = {"value": head[key]["value"], "ms_per_step": head[key]["ms_per_step"],
                        "max_rel_error_vs_oracle": float(np.abs(phis[key].cpu().numpy() - ref).max() / scale)}
    return rec


def run_sweep_exact(g, args):
    """The precision sweep at its stated sizes, 256^3 and 384 x 256 x 256 interior
    points (M = 257 and 385: no FFT here), on plans that solve on the grid as given
    (idp_create_plan_exact): the tensor-core modes, whose sine-matrix products take
    any length, each against the oracle; FP64 on the ordinary (padded) plan."""
    import torch
    from oracle import solve as osolve
    idp = g.idp
    out = {}
    for key, interior in (("interior_256^3", (256, 256, 256)), ("interior_384x256x256", (384, 256, 256))):
        prob = w.c4_sweep(interior)
        rho_h = prob.rho()
        ref = osolve.solve(rho_h, prob.h, args.order, boundary="convolution")
        scale = np.abs(ref).max()
        rho = torch.from_numpy(rho_h).to(g.dev)
        rec = {"workload": describe(prob, args.order)}
        plan = g.plan(prob, args.order)   # padded FP64
        phi = torch.empty_like(rho)
        ms = g.timed(lambda: idp.solve(plan, rho, phi, g.stream), args.steps, args.warmup)
        idp.plan_status(plan)
        rec["fp64_padded"] = {"value": prob.points / (statistics.mean(ms) / 1e3), "ms_per_step": statistics.mean(ms),
                              "grid_solved": idp.plan_grid(plan)[0],
                              "max_rel_error_vs_oracle": float(np.abs(phi.cpu().numpy() - ref).max() / scale)}
        del plan
        for vk, name, bdd in (("mixed_precision", "MIXED_BF16X3", False), ("mixed_tf32x3", "MIXED_TF32X3", False),
                              ("mixed_df32_boundary", "MIXED_BF16X3", True)):
            ph, r = variant_record(g, prob, args.order, getattr(idp, "IDP_PRECISION_" + name), vk, rho, None,
                                   args.steps, args.warmup, bdd=bdd, exact=True)
            rec[vk] = {"value": r["value"], "ms_per_step": r["ms_per_step"], "exact_grid": True,
                       "max_rel_error_vs_oracle": float(np.abs(ph.cpu().numpy() - ref).max() / scale)}
            del ph
        out[key] = rec
        del rho, phi
        torch.cuda.empty_cache()
    return out


def run_bump(g, args):
    """The 129^3 bump workload (FP64): throughput and the error against its exact potential."""
    prob = workload("bump")
    ns = argparse.Namespace(**{**vars(args), "profile_window": 0, "dst_shape": None, "fp64_only": True})
    head, _, _, _ = run_headline(g, ns, prob)
    return {"workload": describe(prob, args.order), "value": head["value"], "ms_per_step": head["ms_per_step"],
            "max_rel_error_vs_exact_potential": head["precision"].get("max_rel_error_vs_exact_potential"),
            "roofline_frac": head["roofline"]["frac"], "dst_pass_avg_ms": head["roofline"]["avg_launch_ms"]}


def run_batched(g, args, rank):
    """96 independent problems, per-axis nodes from {33,65,97,129,193,257} (seed 21081),
    Gaussian-sum densities; one idp_solve_batched call per step."""
    idp, torch = g.idp, g.torch
    probs = w.c5_batch()
    mine = shard(probs, rank, g.world)
    total = sum(p.points for p in mine)
    t0 = time.perf_counter()
    plans = [g.plan(p, args.order) for p in mine]
    setup_s = time.perf_counter() - t0
    rhos = [torch.from_numpy(p.rho()).to(g.dev) for p in mine]
    phis = [torch.empty_like(r) for r in rhos]
    out = {}
    fp64 = None
    for label, prec, bdd in (("fp64", idp.IDP_PRECISION_FP64, 0), ("df32", idp.IDP_PRECISION_DF32, 0),
                             ("mixed_bf16x3", idp.IDP_PRECISION_MIXED_BF16X3, 0),
                             ("mixed_tf32x3", idp.IDP_PRECISION_MIXED_TF32X3, 0),
                             ("mixed_df32_boundary", idp.IDP_PRECISION_MIXED_BF16X3, 1)):
        if args.fp64_only and label != "fp64":
            continue
        for pl in plans:
            idp.plan_set(pl, idp.IDP_KEY_PRECISION, prec)
            idp.plan_set(pl, idp.IDP_KEY_MIXED_BOUNDARY_DF32, bdd)
            if prec != idp.IDP_PRECISION_FP64:
                idp.plan_set(pl, idp.IDP_KEY_AUTOTUNE, 1)
        ms = g.timed(lambda: idp.solve_batched(plans, rhos, phis, g.stream), args.steps, args.warmup)
        for pl in plans:
            idp.plan_status(pl)
        t = max_over_ranks(sum(ms) / args.steps, g.world, g.dev)
        # the same problems one after another (separate graph launches)
        seq = g.timed(lambda: [idp.solve(pl, r, ph, g.stream) for pl, r, ph in zip(plans, rhos, phis)], 2, 1)
        rec = {"value": g.world * total / (t / 1e3), "ms_per_step": t, "sequential_ms": statistics.mean(seq)}
        if label == "fp64":
            fp64 = [ph.clone() for ph in phis]
        else:
            rec["max_rel_error_vs_fp64"] = max(rel(a, b) for a, b in zip(phis, fp64))
        out[label] = rec
    return {"workload": "96 independent 3-D order-%d problems, per-axis nodes from {33,65,97,129,193,257} "
                        "(seed 21081), Gaussian sums (seed 2108+i), one idp_solve_batched call per step"
                        % args.order,
            "nodes": total * g.world, "problems": len(probs), "plan_setup_s": setup_s,
            "value": out["fp64"]["value"], "ms_per_step": out["fp64"]["ms_per_step"], "variants": out}


def run_ours(args, rank, world):
    g = Gpu(world)
    prob = workload(args.workload, args.n)
    head, rho_h, phi, phis = run_headline(g, args, prob)
    del phi, phis
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(prob, args.order, {"parallelism": "replicas" if world > 1 else "single"})}
    for k in ("precision", "mixed_precision", "mixed_tf32x3", "df32", "mixed_df32_boundary", "e2e", "gpu_launches",
              "roofline",
              "kernel_ms_per_step", "dominant_kernel", "tuning", "clocks", "boundary_share", "phi_star_solve"):
        if k in head:
            line[k] = head[k]
    if not args.headline_only:
        g.torch.cuda.empty_cache()
        line["bump_129"] = run_bump(g, args)
        line["sweep_257"] = run_sweep(g, args)
        g.torch.cuda.empty_cache()
        line["sweep_exact"] = run_sweep_exact(g, args)
        g.torch.cuda.empty_cache()
        line["batched"] = run_batched(g, args, rank)
    if rank != 0:
        return
    if world == 1 and not args.headline_only:
        line["cpu_baseline"] = cpu_baseline(prob, args.order, args.workload)
        line["cpu_paper_method"] = cpu_paper_method(prob, args.order, args.workload)
    elif world == 1:
        line["cpu_baseline"] = cpu_baseline(prob, args.order, args.workload, budget_s=1.0)
    print(json.dumps(line), flush=True)


def run_batched_only(args, rank, world):
    g = Gpu(world)
    rec = run_batched(g, args, rank)
    if rank != 0:
        return
    line = {"metric": METRIC + " (batched)", "value": rec["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": rec["workload"], "nodes": rec["nodes"],
                                            "problems": rec["problems"], "plan_setup_s": rec["plan_setup_s"]},
            "variants": rec["variants"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.batched:
        run_batched_only(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
