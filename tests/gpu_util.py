"""Helpers of the GPU tests: moving canonical fields between numpy and torch CUDA tensors,
allocating native buffers, and error measures."""
import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover
    torch = None


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def native_fine(V, nrhs, prec):
    """Native fine spinor buffer: 12 V complex per rhs (complex128 or complex64)."""
    dt = torch.complex128 if prec == 0 else torch.complex64
    return torch.zeros(nrhs * 12 * V, dtype=dt, device="cuda")


def coarse_buf(n, nrhs, prec):
    dt = torch.complex128 if prec == 0 else torch.complex64
    return torch.zeros(nrhs * n, dtype=dt, device="cuda")


def rel_err(got, want):
    got = np.asarray(got).ravel()
    want = np.asarray(want).ravel()
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


# tolerances of the operator parity tests (relative to the largest entry)
TOL = {0: 1e-12, 1: 1e-5}
