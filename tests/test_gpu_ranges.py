"""Threshold ranges much narrower than the spread of the heights.

With a step of about 1e-7, the scaled heights (h - lo) / step reach tens of millions. That is
beyond the range in which the float32 filter's magic-constant ceiling is exact, so every bin must
then take the exact float64 path. At a step near 1e-6 the filter still applies, with bins far
outside [0, T-1] on both sides. Forward and adjoint, on cubical and simplicial complexes, are
compared element by element with the oracle.
"""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib

pytestmark = pytest.mark.gpu

# (lo, hi, T): scaled heights of about +-1.8e7 (exact path only), +-1e6 (filter, far clamps),
# and a range of width 2^-30 around an off-centre threshold
RANGES = [(0.0, 15 * 9.4e-8, 16), (0.0, 8 * 1.7e-6, 9), (0.3, 0.3 + 2.0 ** -30, 5)]


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


@pytest.mark.parametrize("r", range(len(RANGES)))
def test_cubical_forward_and_adjoint_narrow_ranges(P, oracle, r):
    lo, hi, T = RANGES[r]
    dims = [11, 9, 7]
    w = S.uniform_u8_grid(dims, seed=40 + r)
    dirs = S.fibonacci_directions(24)
    cx = P.CubicalComplex(cuda(w))
    got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    ref = oracle.wect_cubical(dims, w.ravel(), dirs, T, lo, hi)
    assert np.array_equal(got, ref)
    G = np.random.default_rng(r).integers(-(1 << 30), 1 << 30, (len(dirs), T)).astype(np.int64)
    g = cx.backward(cuda(dirs), T, lo, hi, cuda(G), 2.0 ** -30).cpu().numpy()
    gref = oracle.wect_backward_cubical(dims, w.ravel().astype(np.int64), dirs, T, lo, hi, G, 2.0 ** -30)
    assert np.array_equal(g, gref)


@pytest.mark.parametrize("r", range(len(RANGES)))
def test_simplicial_forward_and_adjoint_narrow_ranges(P, oracle, r):
    lo, hi, T = RANGES[r]
    cx = S.random_simplicial(200, 3, 600, 300, seed=50 + r)
    dirs = S.random_directions(40, 3, 60 + r)
    vw = cx.weights.astype(np.int64)
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(cx.weights))
    got = h.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
    assert np.array_equal(got, ref)
    G = np.random.default_rng(r).integers(-(1 << 30), 1 << 30, (len(dirs), T)).astype(np.int64)
    g = h.backward(cuda(dirs), T, lo, hi, cuda(G), 2.0 ** -30).cpu().numpy()
    gref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, T, lo, hi, G, 2.0 ** -30)
    assert np.array_equal(g, gref)


def test_long_threshold_rows(P, oracle):
    """T = 1500: the prefix scan over thresholds takes one block per row."""
    dims = [45, 38]
    w = S.uniform_u8_grid(dims, seed=51)
    dirs = S.circle_directions(20)
    cx = P.CubicalComplex(cuda(w))
    got = cx.wect(cuda(dirs), 1500, -1.5, 1.5).cpu().numpy()
    ref = oracle.wect_cubical(dims, w.ravel(), dirs, 1500, -1.5, 1.5)
    assert np.array_equal(got, ref)
    sc = S.random_simplicial(150, 2, 400, 200, seed=52)
    h = P.SimplicialComplex(cuda(sc.coords), [cuda(x) for x in sc.simplices], cuda(sc.weights))
    got = h.wect(cuda(dirs), 1500, -1.5, 1.5).cpu().numpy()
    vw = sc.weights.astype(np.int64)
    ref = oracle.wect_simplicial(sc.coords, sc.simplices, oracle.simplicial_weights(sc.simplices, vw), dirs, 1500, -1.5, 1.5)
    assert np.array_equal(got, ref)


def _chain_complex(X):
    """Vertices X with edges between consecutive points (a path)."""
    nv = X.shape[0]
    edges = np.stack([np.arange(nv - 1), np.arange(1, nv)], axis=1).astype(np.int32)
    return [edges]


@pytest.mark.parametrize("case", ["circle", "origin", "outliers3d"])
def test_simplicial_default_range_candidates(P, oracle, case):
    """The default range M = max |h| over all vertices and directions: every vertex of a circle is
    a candidate, a complex at the origin has M = 0, and far outliers leave a few candidates."""
    rng = np.random.default_rng(61)
    if case == "circle":
        t = rng.uniform(0, 2 * np.pi, 3000)
        X = np.stack([np.cos(t), np.sin(t)], axis=1)
        dirs = S.random_directions(300, 2, 62)
    elif case == "origin":
        X = np.zeros((50, 2))
        dirs = S.circle_directions(16)
    else:
        X = rng.uniform(-1, 1, (5000, 3))
        X[[7, 123, 4000]] = [[9.0, -3.0, 2.0], [-8.5, 4.0, -4.0], [3.0, 9.25, 1.0]]
        dirs = S.fibonacci_directions(200)
    lists = _chain_complex(X)
    w = rng.integers(0, 256, X.shape[0]).astype(np.uint8)
    h = P.SimplicialComplex(cuda(X), [cuda(x) for x in lists], cuda(w))
    got = h.wect(cuda(dirs), 33).cpu().numpy()
    ref = oracle.wect_simplicial(X, lists, oracle.simplicial_weights(lists, w.astype(np.int64)), dirs, 33)
    assert np.array_equal(got, ref)
