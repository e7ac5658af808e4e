"""GPU parity of the multi-filter WECF (wecf_compute, Algorithm 1 with m arbitrary vertex
filters) against the CPU oracle: cubical grids and simplicial complexes, weighted and
unweighted, default and explicit ranges."""
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


def _filters(nv, m, seed):
    rng = np.random.default_rng(seed)
    f = rng.normal(0.0, 1.0, size=(m, nv))
    f[0] = np.round(f[0] * 4) / 4          # many exact ties and values on thresholds
    return f


@pytest.mark.parametrize("dims", [[37, 29], [13, 11, 9], [50]])
def test_wecf_cubical(P, oracle, dims):
    nv = int(np.prod(dims))
    w = S.uniform_u8_grid(dims, seed=31)
    f = _filters(nv, 6, seed=32)
    cx = P.CubicalComplex(cuda(w))
    for weighted, T, lo, hi in ((True, 41, math.nan, math.nan), (False, 17, -2.0, 2.5), (True, 2, -1.0, 1.0)):
        got = cx.wecf(cuda(f), T, lo, hi, weighted=weighted).cpu().numpy()
        ref = oracle.wecf_cubical(dims, w.ravel(), f, T, lo, hi, weighted=weighted)
        assert np.array_equal(got, ref), (weighted, T)


def test_wecf_simplicial(P, oracle):
    for cx in (S.random_simplicial(400, 2, 1200, 700, seed=33), S.tetra_grid(7, seed=34)):
        f = _filters(cx.nv, 5, seed=35)
        vw = cx.weights.astype(np.int64)
        h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(cx.weights))
        for weighted, T, lo, hi in ((True, 33, math.nan, math.nan), (False, 64, -1.5, 1.5)):
            got = h.wecf(cuda(f), T, lo, hi, weighted=weighted).cpu().numpy()
            sw = oracle.simplicial_weights(cx.simplices, vw, "max" if weighted else "one")
            ref = oracle.wecf_simplicial(f, cx.simplices, sw, T, lo, hi)
            assert np.array_equal(got, ref), (weighted, T)
        h.device_status()


def test_wecf_one_filter_equals_ecf(P, oracle):
    dims = [33, 21]
    w = S.uniform_u8_grid(dims, seed=36)
    f = _filters(33 * 21, 1, seed=37)
    cx = P.CubicalComplex(cuda(w))
    a = cx.wecf(cuda(f), 50, -2.0, 2.0, weighted=True).cpu().numpy()[0]
    b = cx.ecf(cuda(f[0]), 50, -2.0, 2.0, weighted=True).cpu().numpy()
    assert np.array_equal(a, b)
