"""The allocation-free entry point, wect_cubical_compute_static.

Some callers cannot allocate device memory: frameworks and inference servers whose caching
allocator owns every device byte, real-time and embedded services that fix their memory at
start-up, and plugin hosts that give a plugin no allocator.  For them the library keeps this
entry point's scratch in a static device array held for the life of the process.

Each call goes through the C ABI with a caller-allocated output, and its output must equal,
element for element, the output of the allocating entry point wect_compute on the same inputs
(and the oracle's, on the small grids).  Every grid is computed by two calls in a row, and a
large grid runs before the small ones, so that scratch state left by an earlier call would show.
This file is collected last, so a run that stops at the first failure has already run every
other test.
"""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib, torch

pytestmark = pytest.mark.gpu

SQ2, SQ3 = math.sqrt(2.0), math.sqrt(3.0)


def _dirs(n, d):
    if n == 1:
        return np.array([[1.0], [-1.0], [0.5], [-0.25], [0.0]] * (d // 5 + 1))[:d]
    return S.circle_directions(d) if n == 2 else S.fibonacci_directions(d)


CASES = [
    # (dims axis 0 first, d, T, lo, hi, weighted, seed, compare with the oracle)
    ([128, 128, 128], 256, 128, math.nan, math.nan, True, 2, False),    # default range, full size
    ([41, 33, 29], 150, 77, -SQ3, SQ3, True, 11, True),
    ([300], 23, 40, -1.0, 1.0, True, 12, True),                          # n = 1
    ([70, 45], 64, 64, -SQ2, SQ2, True, 13, True),                       # n = 2
    ([37, 29], 40, 33, -SQ2, SQ2, False, 14, True),                      # unweighted (WECT_W_ONE)
    ([9, 8, 7], 33, 17, -0.4, 0.3, True, 15, True),                      # narrow range
    ([23, 19, 7], 50, 4096, -SQ3, SQ3, True, 16, True),                  # T beyond the shared histogram
]


def test_static_entry_matches_wect_compute_two_calls_in_a_row(oracle):
    dev()
    P = lib()
    for dims, d, T, lo, hi, weighted, seed, check_oracle in CASES:
        n = len(dims)
        g = S.uniform_u8_grid(dims, seed=seed) if weighted else None
        w = cuda(g) if weighted else None
        dirs = _dirs(n, d)
        dt = cuda(dirs)
        cx = P.CubicalComplex(w, dims=dims)
        ref = cx.wect(dt, T, lo, hi)                                     # allocating entry point
        for call in range(2):
            out = torch.full((d, T), -7 - call, dtype=torch.int64, device=dt.device)
            got = P.cubical_wect_static(w, dt, T, lo, hi, out=out, dims=dims)   # allocation-free
            P.cubical_static_status()
            assert got.data_ptr() == out.data_ptr()
            assert torch.equal(got, ref), (dims, call)
        if check_oracle:
            vw = g.ravel() if weighted else np.zeros(int(np.prod(dims)), dtype=np.int64)
            assert np.array_equal(ref.cpu().numpy(), oracle.wect_cubical(dims, vw, dirs, T, lo, hi, weighted=weighted))


def test_static_entry_reports_a_non_finite_direction():
    dev()
    P = lib()
    w = cuda(S.uniform_u8_grid([20, 18], seed=3))
    dirs = S.circle_directions(8)
    bad = dirs.copy()
    bad[5, 1] = math.nan
    P.cubical_wect_static(w, cuda(bad), 16, -SQ2, SQ2)
    with pytest.raises(P.WectError) as ei:
        P.cubical_static_status()
    assert ei.value.name == "INVALID_ARG"
    P.cubical_static_status()                       # the status word was cleared by the read
    got = P.cubical_wect_static(w, cuda(dirs), 16, -SQ2, SQ2)
    P.cubical_static_status()
    assert torch.equal(got, P.CubicalComplex(w).wect(cuda(dirs), 16, -SQ2, SQ2))


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
