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


def _hard_values(nv, T, lo, hi, oracle, seed):
    """Filter values on and next to every threshold, signed zeros, subnormals, huge values and
    values beyond the range, shuffled into random values."""
    rng = np.random.default_rng(seed)
    beta = oracle.beta(T, lo, hi)
    picks = [beta, np.nextafter(beta, -np.inf), np.nextafter(beta, np.inf),
             np.array([0.0, -0.0, 5e-324, -5e-324, 1e-310, -1e-310, 1e300, -1e300, lo - 1.0, hi + 1.0])]
    special = rng.permutation(np.concatenate(picks))
    f = rng.uniform(lo - 0.25, hi + 0.25, nv)
    idx = rng.choice(nv, size=min(nv, special.size), replace=False)
    f[idx] = special[: idx.size]
    return f


@pytest.mark.parametrize("T", [3, 64, 1000, 30000, 60000])
def test_ecf_bins_at_thresholds_and_large_T(P, oracle, T):
    """Exact bins for values on, just below and just above every threshold, and large T: the
    threshold keys leave shared memory above T = 28,000 or so and the weighted (int64) histogram
    does too; the unweighted one (int32) leaves it above T = 57,000."""
    dims = [97, 89]
    nv = int(np.prod(dims))
    w = S.uniform_u8_grid(dims, seed=33)
    cx = P.CubicalComplex(cuda(w))
    lo, hi = -0.75, 1.25
    f = _hard_values(nv, T, lo, hi, oracle, seed=T)
    for weighted in (False, True):
        got = cx.ecf(cuda(f), T, lo, hi, weighted=weighted).cpu().numpy()
        ref = oracle.wecf_cubical(dims, w.ravel(), f, T, lo, hi, weighted=weighted)[0]
        assert np.array_equal(got, ref), (T, weighted)


def test_ecf_degenerate_range(P, oracle):
    """lo == hi: every threshold is lo; values <= lo land in bin 0, the others in T - 1."""
    dims = [9, 8, 7]
    nv = int(np.prod(dims))
    w = S.uniform_u8_grid(dims, seed=34)
    f = np.random.default_rng(35).choice([-1.0, 0.5, 0.5 + 2**-40, 0.5 - 2**-40, 2.0], size=nv)
    cx = P.CubicalComplex(cuda(w))
    for weighted in (False, True):
        got = cx.ecf(cuda(f), 9, 0.5, 0.5, weighted=weighted).cpu().numpy()
        ref = oracle.wecf_cubical(dims, w.ravel(), f, 9, 0.5, 0.5, weighted=weighted)[0]
        assert np.array_equal(got, ref)


def test_wecf_many_filters_3d(P, oracle):
    """m = 40 filters on a 3D grid (blocks spread over the filters), weighted and unweighted."""
    dims = [21, 17, 19]
    nv = int(np.prod(dims))
    w = S.uniform_u8_grid(dims, seed=36)
    f = _filters(nv, 40, seed=37)
    cx = P.CubicalComplex(cuda(w))
    for weighted in (False, True):
        got = cx.wecf(cuda(f), 97, -2.5, 2.5, weighted=weighted).cpu().numpy()
        ref = oracle.wecf_cubical(dims, w.ravel(), f, 97, -2.5, 2.5, weighted=weighted)
        assert np.array_equal(got, ref), weighted
