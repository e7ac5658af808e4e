"""GPU parity at large T and large d x T, where the shared-memory histograms and the adjoint's
shared suffix table no longer fit: the forward kernels then add every update to the int64
difference table in global memory, and the adjoint sums its octant sums over direction chunks.
Results must stay bit-exact against the oracle."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import SQ2, SQ3, cuda, dev, lib, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


def _weights(dims, kind, rng):
    shape = tuple(reversed(dims))
    if kind == "u8":
        return rng.integers(0, 256, shape, dtype=np.uint8), 0
    if kind == "f32":
        return rng.random(shape, dtype=np.float32), 24
    return rng.integers(-(1 << 27), 1 << 27, shape).astype(np.int64), 0


def _dirs(n, d, seed):
    if n == 1:
        return np.array([[1.0], [-1.0], [0.5], [-0.25], [0.0]] * (d // 5 + 1))[:d]
    base = S.circle_directions(d) if n == 2 else S.fibonacci_directions(d)
    if d >= 4:                                       # axis-aligned directions: heights on thresholds
        base[0] = [1.0] + [0.0] * (n - 1)
        base[1] = [0.0] * (n - 1) + [-1.0]
    return base


@pytest.mark.parametrize("T", [4096, 10000])
@pytest.mark.parametrize("dims,kind", [([301], "u8"), ([37, 29], "f32"), ([17, 13, 11], "u8"), ([12, 9, 10], "i64")])
def test_cubical_forward_large_T(P, oracle, dims, kind, T):
    rng = np.random.default_rng(T + len(dims))
    w, fb = _weights(dims, kind, rng)
    n = len(dims)
    dirs = _dirs(n, 40, T)
    lo, hi = -math.sqrt(n), math.sqrt(n)
    cx = P.CubicalComplex(cuda(w), frac_bits=fb)
    got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    cx.device_status()
    ref = oracle.wect_cubical(dims, oracle.to_fixed(w, fb), dirs, T, lo, hi)
    assert np.array_equal(got, ref)
    got = cx.wect(cuda(dirs), T).cpu().numpy()                 # default range
    assert np.array_equal(got, oracle.wect_cubical(dims, oracle.to_fixed(w, fb), dirs, T))


def test_batch_forward_large_T(P, oracle):
    imgs = S.blob_images(12, seed=21, side_lo=5, side_hi=40)
    dirs = S.circle_directions(36)
    T = 5000
    b = P.CubicalBatch([cuda(x) for x in imgs])
    got = b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()
    again = b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()
    loop = b.wect(cuda(dirs), T, -SQ2, SQ2, loop=True).cpu().numpy()
    assert np.array_equal(got, again) and np.array_equal(got, loop)
    b.autotune(cuda(dirs), T, -SQ2, SQ2)              # no shared-histogram shape fits: keeps the global one
    assert np.array_equal(b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy(), got)
    for i, x in enumerate(imgs):
        ref = oracle.wect_cubical(list(reversed(x.shape)), x.ravel(), dirs, T, -SQ2, SQ2)
        assert np.array_equal(got[i], ref), i


@pytest.mark.parametrize("T", [4096, 10000])
@pytest.mark.parametrize("kind", ["u8", "f32"])
def test_simplicial_forward_large_T(P, oracle, kind, T):
    cx = S.random_simplicial(400, 3, 1200, 900, seed=T % 97)
    rng = np.random.default_rng(T)
    w = cx.weights if kind == "u8" else rng.random(cx.nv, dtype=np.float32) * 5
    fb = 24 if kind == "f32" else 0
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(w), frac_bits=fb)
    dirs = S.random_directions(45, 3, T)
    got = h.wect(cuda(dirs), T, -1.5, 1.5).cpu().numpy()
    h.device_status()
    vw = oracle.to_fixed(w, fb) if kind == "f32" else w.astype(np.int64)
    ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, -1.5, 1.5)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dims,d,T", [([9, 8, 7], 12, 4096), ([30, 11], 7, 10000), ([50], 5, 10000),
                                      ([13, 12, 11], 256, 128), ([10, 9, 8], 300, 300)])
def test_cubical_adjoint_direction_chunks(P, oracle, dims, d, T):
    """d x T beyond the shared suffix table: the octant sums are accumulated over direction chunks."""
    rng = np.random.default_rng(d * T)
    w = rng.random(tuple(reversed(dims)), dtype=np.float32)
    n = len(dims)
    dirs = _dirs(n, d, d)
    lo, hi = -math.sqrt(n), math.sqrt(n)
    G = rng.integers(-(1 << 20), 1 << 20, (d, T)).astype(np.int64)
    cx = P.CubicalComplex(cuda(w), frac_bits=24)
    g = cx.backward(cuda(dirs), T, lo, hi, cuda(G), 2.0 ** -30).cpu().numpy()
    cx.device_status()
    ref = oracle.wect_backward_cubical(dims, oracle.to_fixed(w, 24), dirs, T, lo, hi, G, 2.0 ** -30)
    assert np.array_equal(g, ref)


def test_batch_adjoint_direction_chunks(P, oracle):
    """A batch of volumes with d = 256, T = 128 (the 128^3 workload's d and T): two chunks."""
    count, dims, d, T = 3, [11, 10, 9], 256, 128
    vols = S.uniform_f32_grids(count, dims, seed=41)
    dirs = S.fibonacci_directions(d)
    rng = np.random.default_rng(42)
    G = rng.integers(-(1 << 16), 1 << 16, (count, d, T)).astype(np.int64)
    b = P.CubicalBatch([cuda(x) for x in vols], frac_bits=24)
    g = b.backward(cuda(dirs), T, -SQ3, SQ3, cuda(G), 2.0 ** -20).cpu().numpy().reshape(count, -1)
    for i in range(count):
        ref = oracle.wect_backward_cubical(dims, oracle.to_fixed(vols[i], 24), dirs, T, -SQ3, SQ3, G[i], 2.0 ** -20)
        assert np.array_equal(g[i], ref), i


def test_simplicial_adjoint_large_T(P, oracle):
    cx = S.random_simplicial(200, 2, 500, 300, seed=44)
    rng = np.random.default_rng(44)
    vw = rng.integers(0, 1 << 20, cx.nv).astype(np.int64)
    dirs = S.circle_directions(20)
    T = 10000
    G = rng.integers(-1000, 1000, (20, T)).astype(np.int64)
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(vw))
    g = h.backward(cuda(dirs), T, -1.5, 1.5, cuda(G), 0.25).cpu().numpy()
    ref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, T, -1.5, 1.5, G, 0.25)
    assert np.array_equal(g, ref)
