"""Helpers for the GPU parity tests: build/load libtopo, move numpy arrays to the device."""
import numpy as np


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2004_05756_gb300 import build
    build.build()
    return torch


def dev(x, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def cols(M, dtype=None):
    """N x m numpy block -> (m, N) contiguous CUDA tensor (column-major N x m, ld = N)."""
    M = np.asarray(M)
    if M.ndim == 1:
        M = M[:, None]
    return dev(np.ascontiguousarray(M.T), dtype)


def host_cols(t):
    """(m, ld) tensor -> N x m numpy block."""
    return t.detach().cpu().numpy().T.copy()


def relerr(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))
