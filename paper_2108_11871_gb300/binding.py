"""ctypes binding of libidp.so (include/idp.h), one Python function per C entry point.

Only argument marshalling happens here: device arrays are passed as raw
pointers (torch tensors are accepted and their ``data_ptr()`` is used), and the
CUDA stream as a ``cudaStream_t`` handle.  There is no fallback: if the
library is missing or fails to load, every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

IDP_OK, IDP_EINVAL, IDP_ENOMEM, IDP_ECUDA, IDP_EALIAS, IDP_ESUPPORT, IDP_ESCRATCH = 0, -1, -2, -3, -4, -5, -6
IDP_EGUARD = -8
IDP_RHS6_NOALLOC_MAX_NODES = 524288
IDP_KEY_USE_GRAPH = 1
IDP_KEY_PRECISION = 2
IDP_KEY_STALL_TEST = 3
IDP_KEY_AUTOTUNE = 4
IDP_KEY_DST_SHAPE = 5
IDP_KEY_VALIDATE = 6
IDP_KEY_GUARD_TEST = 7
IDP_KEY_MIXED_BOUNDARY_DF32 = 8
IDP_KEY_NVTX = 9
IDP_PRECISION_FP64, IDP_PRECISION_MIXED_BF16X3, IDP_PRECISION_DF32, IDP_PRECISION_MIXED_TF32X3 = 0, 1, 2, 3
IDP_ETIMEOUT = -7
(IDP_STAGE_BOUNDARY, IDP_STAGE_GTILDE, IDP_STAGE_PHISTAR, IDP_STAGE_U1, IDP_STAGE_R,
 IDP_STAGE_PHI) = range(1, 7)

_lib = None
_vp, _i64, _int, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double


class IdpError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = "%s failed: %s (%d)" % (what, strerror(code), code)
        if code == IDP_ECUDA:
            msg += ": " + library().idp_last_cuda_error().decode()
        super().__init__(msg)


def library(path: str = None):
    """Load libidp.so (default: next to this file).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("IDP_LIBRARY") or _build.LIB
    if not os.path.exists(path):
        raise ImportError("libidp.so not found at %s: build it first "
                          "(python -m paper_2108_11871_gb300.build)" % path)
    lib = ctypes.CDLL(path)
    sig = {
        "idp_create_plan": (_int, [ctypes.POINTER(_vp), _int, ctypes.POINTER(_i64),
                                   ctypes.POINTER(_dbl), _int]),
        "idp_create_plan_exact": (_int, [ctypes.POINTER(_vp), _int, ctypes.POINTER(_i64),
                                         ctypes.POINTER(_dbl), _int]),
        "idp_plan_set": (_int, [_vp, _int, _i64]),
        "idp_solve": (_int, [_vp, _vp, _vp, _vp]),
        "idp_solve_host": (_int, [_vp, _vp, _vp, _vp]),
        "idp_solve_batched": (_int, [_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                     ctypes.POINTER(_vp), _vp]),
        "idp_solve_stage": (_int, [_vp, _int, _vp, _vp, _vp]),
        "idp_plan_status": (_int, [_vp]),
        "idp_plan_info": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                 ctypes.POINTER(_i64)]),
        "idp_destroy_plan": (_int, [_vp]),
        "idp_strerror": (ctypes.c_char_p, [_int]),
        "idp_last_cuda_error": (ctypes.c_char_p, []),
        "idp_plan_tuning": (_int, [_vp, ctypes.POINTER(_i64)]),
        "idp_profile_solve": (_int, [_vp, _vp, _vp, _vp, _int, ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_float)]),
        "idp_plan_launches": (_int, [_vp, ctypes.POINTER(_i64)]),
        "idp_plan_grid": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
        "idp_plan_check_guards": (_int, [_vp]),
        "idp_rhs6_noalloc": (_int, [_int, ctypes.POINTER(_i64), ctypes.POINTER(_dbl), _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return library().idp_strerror(int(code)).decode()


def _check(rc, what):
    if rc != IDP_OK:
        raise IdpError(rc, what)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("expected a device pointer, tensor or array, got %r" % type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Plan:
    """Owns one idp_plan handle."""

    def __init__(self, handle, d, n, h, order):
        self.handle = handle
        self.d, self.n, self.h, self.order = d, tuple(n), tuple(h), order

    def __del__(self):
        try:
            if self.handle:
                destroy_plan(self)
        except Exception:
            pass


def create_plan(d, n, h, order=6, exact=False) -> Plan:
    """idp_create_plan, or idp_create_plan_exact (exact=True: the grid as given)."""
    n = [int(v) for v in n]
    h = [float(v) for v in h]
    if len(n) != d or len(h) != d:
        raise ValueError("n and h need d entries")
    out = _vp()
    fn = library().idp_create_plan_exact if exact else library().idp_create_plan
    rc = fn(ctypes.byref(out), int(d), (_i64 * d)(*n), (_dbl * d)(*h), int(order))
    _check(rc, "idp_create_plan_exact" if exact else "idp_create_plan")
    return Plan(out.value, d, n, h, order)


def plan_set(plan: Plan, key: int, value: int):
    _check(library().idp_plan_set(plan.handle, int(key), int(value)), "idp_plan_set")


def solve(plan: Plan, rho, phi, stream=None):
    _check(library().idp_solve(plan.handle, _ptr(rho), _ptr(phi), _stream(stream)), "idp_solve")


def solve_host(plan: Plan, rho_host, phi_host, stream=None):
    _check(library().idp_solve_host(plan.handle, _ptr(rho_host), _ptr(phi_host), _stream(stream)),
           "idp_solve_host")


def solve_batched(plans, rhos, phis, stream=None):
    k = len(plans)
    hs = (_vp * k)(*[p.handle for p in plans])
    rs = (_vp * k)(*[_ptr(r) for r in rhos])
    ps = (_vp * k)(*[_ptr(p) for p in phis])
    _check(library().idp_solve_batched(k, hs, rs, ps, _stream(stream)), "idp_solve_batched")


def solve_stage(plan: Plan, stage: int, rho, out, stream=None):
    _check(library().idp_solve_stage(plan.handle, int(stage), _ptr(rho), _ptr(out),
                                     _stream(stream)), "idp_solve_stage")


def plan_status(plan: Plan):
    _check(library().idp_plan_status(plan.handle), "idp_plan_status")


def plan_info(plan: Plan):
    a, b, c = _i64(), _i64(), _i64()
    _check(library().idp_plan_info(plan.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "idp_plan_info")
    return dict(nodes=a.value, interior=b.value, workspace_bytes=c.value)


def plan_check_guards(plan: Plan):
    """Raise IdpError(IDP_EGUARD) if a kernel wrote outside one of the plan's buffers."""
    _check(library().idp_plan_check_guards(plan.handle), "idp_plan_check_guards")


def plan_grid(plan: Plan):
    """(node counts of the grid solved on, offset of the caller's node 0 in it)."""
    n = (_i64 * plan.d)()
    off = (_i64 * plan.d)()
    _check(library().idp_plan_grid(plan.handle, n, off), "idp_plan_grid")
    return [int(v) for v in n], [int(v) for v in off]


def plan_tuning(plan: Plan):
    out = (_i64 * 9)()
    _check(library().idp_plan_tuning(plan.handle, out), "idp_plan_tuning")
    return dict(tuned=bool(out[0]), mixed_path=("df32_fft" if out[1] else "tensor_matrix"),
                face_chunks=list(out[2:5]), slices_per_chunk=list(out[5:8]), dst_lines=int(out[8]))


def destroy_plan(plan: Plan):
    if plan.handle:
        h, plan.handle = plan.handle, None
        _check(library().idp_destroy_plan(h), "idp_destroy_plan")


def rhs6_noalloc(d, n, h, u1, R, stream=None):
    """6th-order right-hand side R from u1 without any device allocation (fixed
    12 MiB library scratch; at most IDP_RHS6_NOALLOC_MAX_NODES nodes).  For
    callers whose memory is fully owned by their own allocator or whose loop
    cannot pay cudaMalloc's synchronisation.  Concurrent calls race on the
    shared scratch."""
    n = [int(v) for v in n]
    h = [float(v) for v in h]
    rc = library().idp_rhs6_noalloc(int(d), (_i64 * d)(*n), (_dbl * d)(*h), _ptr(u1), _ptr(R),
                                    _stream(stream))
    _check(rc, "idp_rhs6_noalloc")
