"""Helpers for the GPU tests: build/load libst.so, move numpy arrays to and
from device memory (torch is used only to own device buffers)."""

import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def library():
    from paper_2311_17500_gb300 import build
    build.build()
    import paper_2311_17500_gb300 as P
    P.load()
    return P


def dev(a, dtype=None):
    torch = torch_cuda()
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.astype(dtype or a.dtype)).cuda()
    return t


def empty(n, dtype="float64"):
    torch = torch_cuda()
    return torch.zeros(int(n), dtype=getattr(torch, dtype), device="cuda")


def host(t):
    torch = torch_cuda()
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def ptr(t):
    return t.data_ptr()


def stream():
    torch = torch_cuda()
    return torch.cuda.current_stream().cuda_stream


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)
