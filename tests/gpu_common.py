"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the CPU oracle)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

SQ2 = math.sqrt(2.0)
SQ3 = math.sqrt(3.0)


def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch.device("cuda:0")


def lib():
    import paper_2511_03909_gb300 as P

    P._build.build()
    P.load()
    return P


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def grid_dims(arr):
    return list(reversed(arr.shape))
