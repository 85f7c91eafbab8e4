"""The C ABI library loads and exports what include/idp.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "idp.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(idp_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_11871_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ("idp_create_plan", "idp_solve", "idp_solve_batched", "idp_destroy_plan",
              "idp_plan_status", "idp_strerror"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_argument_errors_need_no_gpu():
    import paper_2108_11871_gb300 as idp
    lib = idp.library()
    out = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(33, 33, 33)
    h = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    assert lib.idp_create_plan(ctypes.byref(out), 4, n, h, 6) == idp.IDP_EINVAL
    assert lib.idp_create_plan(ctypes.byref(out), 0, n, h, 6) == idp.IDP_EINVAL
    one = (ctypes.c_int64 * 1)(2)       # d = 1 with fewer than 3 nodes
    assert lib.idp_create_plan(ctypes.byref(out), 1, one, h, 6) == idp.IDP_EINVAL
    one = (ctypes.c_int64 * 1)(600)     # d = 1, M = 599 panels
    assert lib.idp_create_plan(ctypes.byref(out), 1, one, h, 6) == idp.IDP_ESUPPORT
    assert lib.idp_create_plan(ctypes.byref(out), 3, n, h, 5) == idp.IDP_EINVAL
    # panel counts above 512 have no padded size (smaller unsupported counts are
    # padded, which needs the GPU)
    for bad_n in ((33, 34, 1026), (514, 33, 33), (33, 33, 1025)):   # M = 1025, 513, 1024
        bad = (ctypes.c_int64 * 3)(*bad_n)
        assert lib.idp_create_plan(ctypes.byref(out), 3, bad, h, 6) == idp.IDP_ESUPPORT
    assert lib.idp_solve(None, None, None, None) == idp.IDP_EINVAL
    assert idp.strerror(idp.IDP_EALIAS) == "input and output overlap"


def test_binding_constants_match_the_header():
    # every IDP_* constant the binding defines has the header's value
    import paper_2108_11871_gb300.binding as b
    text = open(HEADER).read()
    declared = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(IDP_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    mine = {k: v for k, v in vars(b).items() if k.startswith("IDP_") and isinstance(v, int)}
    assert mine, "binding defines no constants"
    for k, v in mine.items():
        if k in declared:
            assert declared[k] == v, k
    for k in ("IDP_KEY_DST_SHAPE", "IDP_KEY_AUTOTUNE", "IDP_STAGE_R", "IDP_PRECISION_DF32", "IDP_KEY_NVTX"):
        assert k in mine and k in declared, k


def test_package_exports_every_binding_constant():
    import paper_2108_11871_gb300 as pkg
    import paper_2108_11871_gb300.binding as b
    for k, v in vars(b).items():
        if k.startswith("IDP_") and isinstance(v, int):
            assert getattr(pkg, k, None) == v, k
