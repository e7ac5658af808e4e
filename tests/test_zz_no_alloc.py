"""The allocation-free entry point, wect_cubical_compute_static.

It exists for callers that cannot allocate device memory. Examples: code running while a CUDA
graph is captured, hosts whose allocator owns every device byte, and services that must not
allocate after start-up. Instead of allocating, it keeps its scratch in a static device array
held for the life of the process.

Each call goes through the C ABI and its output must equal, element for element, the output of
the allocating entry point wect_compute on the same inputs. The test runs two calls in a row, so
the second call also shows that the shared scratch is cleared correctly between calls. This
file is collected last, so a run that stops at the first failure has already run every other
test.
"""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib, torch

pytestmark = pytest.mark.gpu


def test_static_entry_matches_wect_compute_two_calls_in_a_row():
    dev()
    P = lib()
    cases = [
        # (grid dims axis 0 first, directions, T, lo, hi, weight seed)
        ([41, 33, 29], S.fibonacci_directions(150), 77, -math.sqrt(3), math.sqrt(3), 11),
        ([128, 128, 128], S.fibonacci_directions(256), 128, math.nan, math.nan, 2),   # default range
    ]
    for dims, dirs, T, lo, hi, seed in cases:
        w = cuda(S.uniform_u8_grid(dims, seed=seed))
        dt = cuda(dirs)
        ref = P.CubicalComplex(w).wect(dt, T, lo, hi)          # allocating entry point
        out = torch.full((len(dirs), T), -7, dtype=torch.int64, device=dt.device)
        got = P.cubical_wect_static(w, dt, T, lo, hi, out=out)  # allocation-free entry point
        torch.cuda.synchronize()
        assert got.data_ptr() == out.data_ptr()
        assert torch.equal(got, ref)


def test_static_entry_rejects_sizes_beyond_its_limits():
    dev()
    P = lib()
    dirs = cuda(S.fibonacci_directions(8))
    too_big = torch.zeros((129, 128, 128), dtype=torch.uint8, device=dirs.device)   # > 2^21 vertices
    with pytest.raises(P.WectError) as ei:
        P.cubical_wect_static(too_big, dirs, 16, -1.0, 1.0)
    assert ei.value.name == "INVALID_ARG" and "2^21" in str(ei.value)
    small = torch.zeros((4, 4, 4), dtype=torch.uint8, device=dirs.device)
    with pytest.raises(P.WectError) as ei:
        P.cubical_wect_static(small, dirs, 5000, -1.0, 1.0)                          # T > 4096
    assert ei.value.name == "INVALID_ARG"
