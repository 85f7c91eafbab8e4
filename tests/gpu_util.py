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
