"""GPU parity of simplicial complexes in R^4 with simplices up to dimension 4 (the method holds
in any R^n, Section 2): the transform, the ECF, the adjoint and large T, against the oracle."""
import math
from itertools import combinations

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


def _make(P, cx, w, fb=0):
    return P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(w), frac_bits=fb)


def _random_pentachora(nv, k4, seed):
    """Random points in [-1, 1]^4 and k4 random 4-simplices with all their faces (the lists of a
    complex without locality: the gather reads global memory for most chunks)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (nv, 4))
    top = np.array([rng.choice(nv, 5, replace=False) for _ in range(k4)], dtype=np.int64)
    cx = S.closure_from_top(X, top)
    cx.weights = rng.integers(0, 256, nv, dtype=np.uint8)
    return cx


@pytest.mark.parametrize("case", range(4))
def test_four_dimensional_complexes(P, oracle, case):
    if case < 2:
        cx = S.freudenthal_mesh([5, 4, 4, 3] if case == 0 else [3, 3, 2, 7], seed=70 + case)
    else:
        cx = _random_pentachora(300, 500, seed=70 + case)
    dirs = S.random_directions(45, 4, seed=80 + case)
    T, lo, hi = [(33, -2.0, 2.0), (64, math.nan, math.nan), (200, -1.5, 1.2), (17, math.nan, math.nan)][case]
    rng = np.random.default_rng(90 + case)
    if case % 2:
        w, fb = rng.random(cx.nv, dtype=np.float32) * 3, 24
        vw = oracle.to_fixed(w, 24)
    else:
        w, fb = cx.weights, 0
        vw = w.astype(np.int64)
    h = _make(P, cx, w, fb)
    assert h.cell_counts() == [cx.nv] + [len(s) for s in cx.simplices]
    got = h.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    h.device_status()
    ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
    assert np.array_equal(got, ref)
    # ECF of one filter, weighted and not
    f = rng.standard_normal(cx.nv)
    for weighted in (False, True):
        e = h.ecf(cuda(f), 40, -2.5, 2.5, weighted=weighted).cpu().numpy()
        ws = oracle.simplicial_weights(cx.simplices, vw, "max" if weighted else "one")
        assert np.array_equal(e, oracle.wecf_simplicial(f, cx.simplices, ws, 40, -2.5, 2.5)[0])


def test_four_sphere_euler_characteristic(P, oracle):
    """The boundary of a 5-simplex in R^4 is a 4-sphere: chi = 2 in the top column."""
    rng = np.random.default_rng(75)
    X = rng.uniform(-1, 1, (6, 4))
    cx = S.closure_from_top(X, np.array(list(combinations(range(6), 5)), dtype=np.int64))
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], None)
    W = h.wect(cuda(S.random_directions(9, 4, seed=76)), 11).cpu().numpy()
    assert np.all(W[:, -1] == 2)


def test_four_dimensional_adjoint_and_large_T(P, oracle):
    cx = S.freudenthal_mesh([4, 3, 3, 3], seed=77)
    rng = np.random.default_rng(78)
    vw = rng.integers(0, 1 << 20, cx.nv).astype(np.int64)
    dirs = S.random_directions(40, 4, seed=79)
    h = _make(P, cx, vw)
    for T in (30, 5000):
        G = rng.integers(-1000, 1000, (40, T)).astype(np.int64)
        g = h.backward(cuda(dirs), T, -2.0, 2.0, cuda(G), 0.5).cpu().numpy()
        ref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, T, -2.0, 2.0, G, 0.5)
        assert np.array_equal(g, ref), T
        got = h.wect(cuda(dirs), T, -2.0, 2.0).cpu().numpy()
        ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T,
                                     -2.0, 2.0)
        assert np.array_equal(got, ref), T
