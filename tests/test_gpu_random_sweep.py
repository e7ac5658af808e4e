"""Seeded random sweep of the CUDA path against the oracle, element by element: random grid
shapes (axes of length 1 and 2 included), dimensions 1-3, direction sets with exact zeros and
dyadic components (ties between vertex heights), thresholds from 2 to 300, default, wide, narrow
and degenerate ranges, every weight type; the transform, the ECF, the adjoint, simplex lists
and batches."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


def _dirs(rng, n, d):
    kind = rng.integers(0, 3)
    if kind == 0:
        X = rng.normal(size=(d, n))
        X /= np.linalg.norm(X, axis=1, keepdims=True)
    elif kind == 1:                       # dyadic components, many exact zeros: ties
        X = rng.integers(-4, 5, size=(d, n)) / 4.0
        X[np.all(X == 0, axis=1), 0] = 1.0
    else:                                 # axis-aligned and diagonal directions mixed with random ones
        X = rng.normal(size=(d, n))
        for i in range(0, d, 3):
            X[i] = 0.0
            X[i, rng.integers(0, n)] = rng.choice([-1.0, 1.0])
        if n >= 2 and d > 1:
            X[1] = np.full(n, 1.0 / math.sqrt(n))
    return np.ascontiguousarray(X)


def _range(rng, R):
    kind = rng.integers(0, 4)
    if kind == 0:
        return math.nan, math.nan
    if kind == 1:
        return -R, R
    if kind == 2:                         # narrow, off-centre: many heights outside
        a = rng.uniform(-0.5, 0.3) * R
        return a, a + rng.uniform(0.01, 0.4) * R
    a = float(rng.uniform(-0.3, 0.3))     # degenerate
    return a, a


def _weights(rng, shape, kind):
    if kind == "u8":
        return rng.integers(0, 256, shape, dtype=np.uint8), 0
    if kind == "f32":
        return rng.random(shape, dtype=np.float32) * 4, 24
    if kind == "i64":
        return rng.integers(-(1 << 22), 1 << 22, shape).astype(np.int64), 0
    return None, 0


def _fixed(oracle, w, fb, shape):
    if w is None:
        return np.ones(int(np.prod(shape)), dtype=np.int64)
    if w.dtype == np.float32:
        return oracle.to_fixed(w, fb).ravel()
    return w.astype(np.int64).ravel()


@pytest.mark.parametrize("seed", range(60))
def test_random_cubical(P, oracle, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 4))
    dims = [int(rng.choice([1, 2, 3, 7, 16, 33, 40])) for _ in range(n)]
    if n == 1:
        dims[0] = int(rng.integers(1, 300))
    shape = tuple(reversed(dims))
    d = int(rng.integers(1, 70))
    T = int(rng.choice([2, 3, 17, 64, 129, 300]))
    wk = ["u8", "f32", "i64", "one"][seed % 4]
    w, fb = _weights(rng, shape, wk)
    dirs = _dirs(rng, n, d)
    lo, hi = _range(rng, math.sqrt(n))
    cx = P.CubicalComplex(None if w is None else cuda(w), frac_bits=fb, dims=dims if w is None else None)
    vw = _fixed(oracle, w, fb, shape)
    got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    ref = oracle.wect_cubical(dims, vw, dirs, T, lo, hi)
    assert np.array_equal(got, ref), (dims, d, T, wk, lo, hi)
    # the ECF of a random filter with many exact ties, weighted and not
    f = np.round(rng.normal(size=int(np.prod(dims))) * 3) / 3
    for weighted in (False, True):
        e = cx.ecf(cuda(f), T, -1.0, 1.0, weighted=weighted).cpu().numpy()
        eref = oracle.wecf_cubical(dims, vw, f, T, -1.0, 1.0, weighted=weighted)[0]
        assert np.array_equal(e, eref), ("ecf", weighted)
    # the exact adjoint for an integer upstream gradient (explicit range)
    if not (lo == lo):
        lo, hi = -math.sqrt(n), math.sqrt(n)
    G = rng.integers(-(1 << 20), 1 << 20, (d, T)).astype(np.int64)
    g = cx.backward(cuda(dirs), T, lo, hi, cuda(G), 0.25).cpu().numpy()
    gref = oracle.wect_backward_cubical(dims, vw, dirs, T, lo, hi, G, 0.25)
    assert np.array_equal(g, gref), "adjoint"


@pytest.mark.parametrize("seed", range(30))
def test_random_simplicial(P, oracle, seed):
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(2, 4))
    nv = int(rng.integers(3, 400))
    cx = S.random_simplicial(nv, n, int(rng.integers(1, 900)), int(rng.integers(1, 600)), seed=3000 + seed,
                             coord_bits=None if seed % 2 else 6)
    d = int(rng.integers(1, 90))
    T = int(rng.choice([2, 5, 33, 100, 257]))
    dirs = _dirs(rng, n, d)
    lo, hi = _range(rng, 1.8)
    simp = cx.simplices
    wk = seed % 3
    if wk == 0:
        w, fb, vw = cx.weights, 0, cx.weights.astype(np.int64)
    elif wk == 1:
        wf = rng.random(nv, dtype=np.float32) * 3
        w, fb, vw = wf, 24, oracle.to_fixed(wf, 24)
    else:
        w, fb, vw = None, 0, np.ones(nv, dtype=np.int64)
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(x) for x in simp], None if w is None else cuda(w), frac_bits=fb)
    got = h.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    ref = oracle.wect_simplicial(cx.coords, simp, oracle.simplicial_weights(simp, vw), dirs, T, lo, hi)
    assert np.array_equal(got, ref), (nv, n, d, T, lo, hi, wk)
    if lo == lo:
        G = rng.integers(-(1 << 20), 1 << 20, (d, T)).astype(np.int64)
        g = h.backward(cuda(dirs), T, lo, hi, cuda(G), 0.5).cpu().numpy()
        gref = oracle.wect_backward_simplicial(cx.coords, vw, simp, dirs, T, lo, hi, G, 0.5)
        assert np.array_equal(g, gref), "adjoint"


@pytest.mark.parametrize("seed", range(10))
def test_random_batch(P, oracle, seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(2, 4))
    count = int(rng.integers(1, 40))
    wk = ["u8", "f32", "i64"][seed % 3]
    grids, fbs = [], 0
    for _ in range(count):
        dims = [int(rng.integers(1, 30)) for _ in range(n)]
        w, fbs = _weights(rng, tuple(reversed(dims)), wk)
        grids.append(w)
    d = int(rng.integers(1, 80))
    T = int(rng.choice([2, 9, 64, 200]))
    dirs = _dirs(rng, n, d)
    lo, hi = -math.sqrt(n), math.sqrt(n) * float(rng.uniform(0.2, 1.0))
    b = P.CubicalBatch([cuda(x) for x in grids], frac_bits=fbs)
    got = b.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    loop = b.wect(cuda(dirs), T, lo, hi, loop=True).cpu().numpy()
    assert np.array_equal(got, loop)
    for i, x in enumerate(grids):
        dims = list(reversed(x.shape))
        ref = oracle.wect_cubical(dims, _fixed(oracle, x, fbs, x.shape), dirs, T, lo, hi)
        assert np.array_equal(got[i], ref), i
