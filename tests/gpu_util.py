"""Shared fixtures for the GPU parity tests (device transfers only, no arithmetic)."""
import numpy as np
import pytest


def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_f(torch, a):
    """Column-major (Fortran) numpy block -> CUDA tensor with the same values."""
    return torch.from_numpy(np.asarray(a)).cuda()
