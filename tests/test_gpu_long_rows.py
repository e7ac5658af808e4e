"""Grids whose axis-0 rows are longer than the stencil kernel's shared row buffers: the forward
walks them in segments of 512 vertices (each with its own row of octant contributions, the
neighbours across a segment boundary read from the grid).  Transform, ECF-free paths, the
global-histogram variant, batches and the adjoint against the oracle, bit for bit."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib, torch

pytestmark = pytest.mark.gpu

SQ2, SQ3 = math.sqrt(2.0), math.sqrt(3.0)


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


def _grid(dims, seed, kind="u8"):
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(dims))
    if kind == "u8":
        return rng.integers(0, 256, shape).astype(np.uint8)
    if kind == "flat":                     # long runs of equal weights: ties across segment ends
        return (rng.integers(0, 3, shape) * 100).astype(np.uint8)
    return rng.uniform(0.0, 4.0, shape).astype(np.float32)


def _dirs(n, d, seed):
    if n == 1:
        return np.array([[1.0], [-1.0], [0.75], [-0.3]])[:d]
    if n == 2:
        return S.circle_directions(d)
    return S.fibonacci_directions(d)


@pytest.mark.parametrize("dims,d,T,kind", [
    ([5000], 4, 40, "u8"),
    ([2100, 23], 40, 50, "u8"),
    ([1537, 11], 24, 33, "f32"),
    ([1030, 6, 5], 33, 64, "u8"),
    ([1025, 7], 16, 20, "flat"),
])
def test_long_rows_forward(P, oracle, dims, d, T, kind):
    w = _grid(dims, sum(dims), kind)
    n = len(dims)
    dirs = _dirs(n, d, 1)
    fb = 20 if kind == "f32" else 0
    cx = P.CubicalComplex(cuda(w), frac_bits=fb)
    vw = oracle.to_fixed(w, fb)
    for lo, hi in ((-math.sqrt(n), math.sqrt(n)), (math.nan, math.nan), (-0.3, 0.45)):
        got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
        ref = oracle.wect_cubical(dims, vw, dirs, T, lo, hi)
        assert np.array_equal(got, ref), (dims, lo, hi)
    cx.device_status()


def test_long_rows_unweighted_and_variants(P, oracle):
    """The unweighted complex, and the per-vertex kernel forced through the selection hook (the
    run-based kernel does not take segmented grids)."""
    dims = [1800, 9]
    dirs = S.circle_directions(30)
    T = 45
    cx = P.CubicalComplex(None, dims=dims)
    ref = oracle.wect_cubical(dims, np.ones(int(np.prod(dims)), dtype=np.int64), dirs, T, -SQ2, SQ2, weighted=False)
    for variant in (0, 1, 2, 3):
        P.stencil_variant(variant)
        try:
            got = cx.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()
            assert P.last_stencil_kernel() == "cubical_fwd_kernel"
        finally:
            P.stencil_variant(0)
        assert np.array_equal(got, ref), variant


def test_long_rows_large_T_global_histogram(P, oracle):
    """T beyond the shared histogram: the global-histogram variant walks the segments too."""
    dims = [1100, 9]
    w = _grid(dims, 77)
    dirs = S.circle_directions(20)
    T = 5000
    cx = P.CubicalComplex(cuda(w))
    got = cx.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()
    assert np.array_equal(got, oracle.wect_cubical(dims, w.ravel().astype(np.int64), dirs, T, -SQ2, SQ2))


def test_long_rows_in_a_batch(P, oracle):
    """A batch mixing segmented and whole-row grids: graph replay, the per-grid loop and the
    autotuned shape all equal the oracle."""
    dims_list = [[1300, 5], [40, 30], [700, 3], [17, 60]]
    grids = [_grid(dm, 90 + i) for i, dm in enumerate(dims_list)]
    dirs = S.circle_directions(48)
    T, lo, hi = 40, -SQ2, SQ2
    b = P.CubicalBatch([cuda(g) for g in grids])
    refs = [oracle.wect_cubical(dm, g.ravel().astype(np.int64), dirs, T, lo, hi) for dm, g in zip(dims_list, grids)]
    for loop in (False, True):
        out = b.wect(cuda(dirs), T, lo, hi, loop=loop).cpu().numpy()
        for i, ref in enumerate(refs):
            assert np.array_equal(out[i], ref), (loop, i)
    b.autotune(cuda(dirs), T, lo, hi)
    shape = b.tuned_shape(48, T)
    assert shape is not None and not shape[2]
    out = b.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    for i, ref in enumerate(refs):
        assert np.array_equal(out[i], ref), i


def test_long_rows_adjoint(P, oracle):
    dims = [1500, 7]
    w = _grid(dims, 55)
    dirs = S.circle_directions(24)
    T = 32
    cx = P.CubicalComplex(cuda(w))
    G = np.random.default_rng(56).integers(-3000, 3000, (len(dirs), T)).astype(np.int64)
    g = cx.backward(cuda(dirs), T, -SQ2, SQ2, cuda(G), 0.25).cpu().numpy()
    ref = oracle.wect_backward_cubical(dims, w.ravel().astype(np.int64), dirs, T, -SQ2, SQ2, G, 0.25)
    assert np.array_equal(g.reshape(-1), ref.reshape(-1))
