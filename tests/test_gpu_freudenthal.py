"""GPU parity of the device-built Freudenthal triangulation (wect_complex_create_freudenthal):
its cell counts, forward transform and adjoint against the oracle on the same triangulation
built on the CPU."""
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


@pytest.mark.parametrize("dims", [[40], [23, 17], [9, 8, 7], [1, 6, 5]])
def test_freudenthal_forward_and_adjoint(P, oracle, dims):
    n = len(dims)
    w = S.uniform_u8_grid(dims, seed=41)
    lists = S.freudenthal_lists(dims)
    X = oracle.grid_coords(dims)
    cx = P.FreudenthalComplex(cuda(w))
    assert cx.cell_counts()[: n + 1] == [X.shape[0]] + [len(l) for l in lists]
    dirs = S.fibonacci_directions(37) if n == 3 else (S.circle_directions(37) if n == 2 else np.array([[1.0], [-1.0], [0.3]]))
    vw = w.ravel().astype(np.int64)
    sw = oracle.simplicial_weights(lists, vw)
    for T, lo, hi in ((29, math.nan, math.nan), (64, -math.sqrt(n), math.sqrt(n))):
        got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
        ref = oracle.wect_simplicial(X, lists, sw, dirs, T, lo, hi)
        assert np.array_equal(got, ref), T
    G = np.random.default_rng(42).integers(-3000, 3000, (len(dirs), 31)).astype(np.int64)
    g = cx.backward(cuda(dirs), 31, -1.8, 1.8, cuda(G), 0.125).cpu().numpy()
    ref = oracle.wect_backward_simplicial(X, vw, lists, dirs, 31, -1.8, 1.8, G, 0.125)
    assert np.array_equal(g, ref)
    cx.device_status()


def test_freudenthal_f32_weights_and_unweighted(P, oracle):
    dims = [30, 26]
    rng = np.random.default_rng(43)
    w = rng.random((26, 30), dtype=np.float32)
    lists = S.freudenthal_lists(dims)
    X = oracle.grid_coords(dims)
    dirs = S.circle_directions(24)
    cx = P.FreudenthalComplex(cuda(w), frac_bits=24)
    got = cx.wect(cuda(dirs), 50, -1.5, 1.5).cpu().numpy()
    vw = oracle.fixed_from_f32(w.ravel(), 24)
    assert np.array_equal(got, oracle.wect_simplicial(X, lists, oracle.simplicial_weights(lists, vw), dirs, 50, -1.5, 1.5))
    cu = P.FreudenthalComplex(None, dims=dims)
    got = cu.wect(cuda(dirs), 50, -1.5, 1.5).cpu().numpy()
    one = oracle.simplicial_weights(lists, np.ones(X.shape[0], dtype=np.int64), "one")
    ref = oracle.wect_simplicial(X, lists, one, dirs, 50, -1.5, 1.5)
    assert np.array_equal(got, ref)
    assert np.all(got[:, -1] == 1)
