"""Helpers shared by the GPU tests: device buffers from torch, binding context."""
import pytest

torch = pytest.importorskip("torch")


def ctx():
    from paper_2609_20536_b300 import hotrg as H
    return H.Context()


def dev_f64(n):
    return torch.empty(n, dtype=torch.float64, device="cuda")


def dev_i32(n):
    return torch.empty(n, dtype=torch.int32, device="cuda")


def to_dev(a, dtype=None):
    import numpy as np
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()
