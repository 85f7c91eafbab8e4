"""Green's function and the boundary values g of the harmonic correction (section 4).

Two evaluations of the same trapezoid sum:
  * ``boundary_direct``: eq. TrapOrig2D (and its 3-D analogue) one boundary
    node at a time, summing over the non-zero interior values of rho;
  * ``boundary_convolution``: the rearrangement of eqs. Trap2D,
    Trap2Dconvolution and convolution -- for each face, a sum over the slices
    parallel to it of (d-1)-dimensional aperiodic convolutions of the rho
    slice with G(sqrt(dist^2 + |.|^2)), each done with a zero-padded FFT.
Boundary nodes of rho do not contribute (the integrand vanishes there).
"""
import numpy as np

from . import _build


def green(r, d: int):
    """G(r): |r|/2 (1-D), log(r)/(2 pi) (2-D), -1/(4 pi r) (3-D); section 1."""
    r = np.asarray(r, dtype=np.float64)
    if d == 1:
        return 0.5 * np.abs(r)
    if d == 2:
        return np.log(r) / (2.0 * np.pi)
    if d == 3:
        return -1.0 / (4.0 * np.pi * r)
    raise ValueError(d)


def boundary_mask(n) -> np.ndarray:
    """True on every node with some index equal to 0 or M_s."""
    m = np.zeros(n, dtype=bool)
    for s in range(len(n)):
        idx = [slice(None)] * len(n)
        idx[s] = 0
        m[tuple(idx)] = True
        idx[s] = n[s] - 1
        m[tuple(idx)] = True
    return m


def boundary_indices(n) -> np.ndarray:
    """(nb, d) int32 node indices of all boundary nodes, C order."""
    return np.argwhere(boundary_mask(n)).astype(np.int32)


def boundary_direct(rho: np.ndarray, h, targets=None) -> np.ndarray:
    """g at the target nodes (default: all boundary nodes, C order) by the
    direct trapezoid sum over non-zero interior rho (eq. TrapOrig2D)."""
    d = rho.ndim
    inner = np.zeros(rho.shape, dtype=bool)
    inner[tuple(slice(1, n - 1) for n in rho.shape)] = True
    src_mask = inner & (rho != 0.0)
    src_idx = np.ascontiguousarray(np.argwhere(src_mask).astype(np.int32))
    src_val = np.ascontiguousarray(rho[src_mask].astype(np.float64))
    if targets is None:
        targets = boundary_indices(rho.shape)
    tgt = np.ascontiguousarray(np.asarray(targets, dtype=np.int32).reshape(-1, d))
    out = np.zeros(tgt.shape[0], dtype=np.float64)
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    _build.lib().oracle_boundary_direct(
        d, hh.ctypes.data, src_idx.shape[0], src_idx.ctypes.data,
        src_val.ctypes.data, tgt.shape[0], tgt.ctypes.data, out.ctypes.data)
    return out


def boundary_direct_nodes(rho: np.ndarray, h) -> np.ndarray:
    """Node array holding g on the boundary (direct sum) and 0 inside."""
    out = np.zeros(rho.shape, dtype=np.float64)
    idx = boundary_indices(rho.shape)
    out[tuple(idx.T)] = boundary_direct(rho, h, idx)
    return out


def _cyclic_kernel_1d(M: int, h: float):
    """Offsets of a length-2M cyclic kernel: t -> min(t, 2M - t) * h.

    Outputs j = 0..M and inputs q = 1..M-1 have |j - q| <= M - 1, so a cyclic
    convolution of length 2M reproduces the aperiodic one without wrap-around
    (the entry t = M is never used)."""
    t = np.arange(2 * M)
    return np.minimum(t, 2 * M - t).astype(np.float64) * h


def boundary_convolution(rho: np.ndarray, h, chunk: int = 16) -> np.ndarray:
    """Node array holding g on the boundary and 0 inside, by the convolution
    rearrangement of section 4 (eqs. Trap2D, Trap2Dconvolution, convolution).

    For axis a and its two faces (i_a = 0 and i_a = M_a):
      g_face(j) = h_a * sum_{p=1}^{M_a-1} (w_p)(j),
      (w_p)(j)  = sum_q G(sqrt(dist_p^2 + |(j - q) h|^2)) rho(p, q) prod_{b != a} h_b,
    with dist_p = p h_a for the face i_a = 0 and (M_a - p) h_a for i_a = M_a;
    q runs over the interior nodes of the slice.  Each w_p is a zero-padded
    cyclic FFT convolution of length 2 M_b per remaining axis b.  Nodes shared
    by several faces get the value of the last face that writes them.
    """
    d = rho.ndim
    n = rho.shape
    M = [k - 1 for k in n]
    out = np.zeros(n, dtype=np.float64)
    if d == 1:
        raise ValueError("use the 1-D sum directly")
    for a in range(d):
        others = [b for b in range(d) if b != a]
        # slab of interior slices p = 1..M_a-1 with the remaining axes padded to 2M_b
        r = np.moveaxis(rho, a, 0)[1:M[a]]
        inner = tuple(slice(1, n[b] - 1) for b in others)
        pad = np.zeros((M[a] - 1,) + tuple(2 * M[b] for b in others))
        pad[(slice(None),) + inner] = r[(slice(None),) + inner]
        axes = tuple(range(1, d))
        R = np.fft.rfftn(pad, axes=axes)
        # squared offsets of the (d-1)-dim cyclic kernel
        off2 = 0.0
        for j, b in enumerate(others):
            o = _cyclic_kernel_1d(M[b], h[b])
            shape = [1] * (d - 1)
            shape[j] = 2 * M[b]
            off2 = off2 + (o ** 2).reshape(shape)
        acc_lo = 0.0
        acc_hi = 0.0
        for p0 in range(1, M[a], chunk):
            ps = np.arange(p0, min(M[a], p0 + chunk))
            dist_lo = (ps * h[a]).reshape((-1,) + (1,) * (d - 1))
            dist_hi = ((M[a] - ps) * h[a]).reshape((-1,) + (1,) * (d - 1))
            K_lo = np.fft.rfftn(green(np.sqrt(dist_lo ** 2 + off2), d), axes=axes)
            K_hi = np.fft.rfftn(green(np.sqrt(dist_hi ** 2 + off2), d), axes=axes)
            Rp = R[ps - 1]
            acc_lo = acc_lo + (Rp * K_lo).sum(axis=0)
            acc_hi = acc_hi + (Rp * K_hi).sum(axis=0)
        shape2 = tuple(2 * M[b] for b in others)
        w_lo = np.fft.irfftn(acc_lo, s=shape2, axes=tuple(range(d - 1)))
        w_hi = np.fft.irfftn(acc_hi, s=shape2, axes=tuple(range(d - 1)))
        keep = tuple(slice(0, n[b]) for b in others)
        scale = float(np.prod(h))
        face = np.moveaxis(out, a, 0)
        face[0] = w_lo[keep] * scale
        face[M[a]] = w_hi[keep] * scale
    return out
