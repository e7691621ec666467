"""Helpers for the GPU parity tests: device tensors from numpy and back."""

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2102_05054_gb300 import floquet
    floquet.lib()  # raises if libfloquet.so is missing
    return torch


def to_dev(x, dtype=None):
    import torch
    x = np.asarray(x)
    t = torch.from_numpy(np.ascontiguousarray(x.T if x.ndim == 2 else x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def from_dev(t, d=None):
    a = t.detach().cpu().numpy()
    if d is not None and a.size != d:
        a = a.reshape(-1, d).T  # column-major block d x n
    return a.astype(np.complex128)
