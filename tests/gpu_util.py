"""Helpers for the GPU parity tests (device arrays via torch, oracle on the host)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def device():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch.device("cuda:0")


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device())


def rel_max(a, b, ref=None):
    """max|a - b| / max|ref| (ref defaults to b)."""
    a = np.asarray(a)
    b = np.asarray(b)
    ref = b if ref is None else np.asarray(ref)
    return float(np.abs(a - b).max() / np.abs(ref).max())


def run_stage(idp, plan, stage, rho_dev, shape):
    out = torch.empty(shape, dtype=torch.float64, device=rho_dev.device)
    idp.solve_stage(plan, stage, rho_dev, out)
    torch.cuda.synchronize()
    idp.plan_status(plan)
    return out.cpu().numpy()


def r_amplification(h):
    """A = sum over ordered pairs s != r of c_sr * 64 / (h_s^4 h_r^2): the largest
    factor by which the 6th-order right-hand side R (a sixth difference of u1,
    section 5) can amplify a perturbation of u1 in the max norm (each D2 stencil
    has absolute weight sum 4 / h^2)."""
    d = len(h)
    a = 0.0
    for s in range(d):
        for r in range(d):
            if r != s:
                c = h[s] ** 4 / 240 + h[s] ** 2 * h[r] ** 2 / 144
                a += c * 64 / (h[s] ** 4 * h[r] ** 2)
    return a
