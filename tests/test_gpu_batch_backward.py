"""GPU parity of the batched persistent launch (graph-captured) and of the exact adjoint."""
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


def test_batch_images_small(P, oracle):
    imgs = S.blob_images(60, seed=4, side_lo=5, side_hi=70)
    dirs = S.circle_directions(64)
    T = 64
    b = P.CubicalBatch([cuda(x) for x in imgs])
    got = b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()
    again = b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()          # graph replay
    loop = b.wect(cuda(dirs), T, -SQ2, SQ2, loop=True).cpu().numpy()
    assert np.array_equal(got, again) and np.array_equal(got, loop)
    for i, x in enumerate(imgs):
        ref = oracle.wect_cubical(list(reversed(x.shape)), x.ravel(), dirs, T, -SQ2, SQ2)
        assert np.array_equal(got[i], ref), i


def test_batch_autotune_keeps_results(P, oracle):
    imgs = S.blob_images(40, seed=11, side_lo=20, side_hi=90)
    dirs = S.circle_directions(64)
    b = P.CubicalBatch([cuda(x) for x in imgs])
    before = b.wect(cuda(dirs), 64, -SQ2, SQ2).cpu().numpy()
    b.autotune(cuda(dirs), 64, -SQ2, SQ2)
    after = b.wect(cuda(dirs), 64, -SQ2, SQ2).cpu().numpy()
    assert np.array_equal(before, after)


def test_backward_cubical_matches_oracle(P, oracle):
    rng = np.random.default_rng(5)
    for dims, d, T in (([9, 8, 7], 16, 16), ([30, 20], 24, 33), ([40], 5, 9), ([13, 12, 11], 128, 128)):
        w = rng.random(tuple(reversed(dims)), dtype=np.float32)
        n = len(dims)
        dirs = S.fibonacci_directions(d) if n == 3 else (S.circle_directions(d) if n == 2 else
                                                         np.array([[1.0], [-1.0], [0.3], [-0.7], [0.0]]))
        lo, hi = -math.sqrt(n), math.sqrt(n)
        G = rng.integers(-(1 << 30), 1 << 30, (len(dirs), T)).astype(np.int64)
        cx = P.CubicalComplex(cuda(w), frac_bits=24)
        g = cx.backward(cuda(dirs), T, lo, hi, cuda(G), 2.0 ** -40).cpu().numpy()
        ref = oracle.wect_backward_cubical(dims, oracle.to_fixed(w, 24), dirs, T, lo, hi, G, 2.0 ** -40)
        assert np.array_equal(g, ref), dims


def test_backward_ties_and_u8(P, oracle):
    """Integer weights with many ties: the heaviest vertex with the lowest index takes the gradient."""
    rng = np.random.default_rng(6)
    dims = [12, 11, 10]
    w = rng.integers(0, 4, tuple(reversed(dims)), dtype=np.uint8)
    dirs = S.fibonacci_directions(20)
    G = rng.integers(-50, 50, (20, 24)).astype(np.int64)
    cx = P.CubicalComplex(cuda(w))
    g = cx.backward(cuda(dirs), 24, -SQ3, SQ3, cuda(G), 1.0).cpu().numpy()
    ref = oracle.wect_backward_cubical(dims, w.ravel().astype(np.int64), dirs, 24, -SQ3, SQ3, G, 1.0)
    assert np.array_equal(g, ref)


def test_backward_simplicial_matches_oracle(P, oracle):
    cx = S.random_simplicial(150, 2, 400, 200, seed=8)
    rng = np.random.default_rng(8)
    vw = rng.integers(0, 1 << 20, cx.nv).astype(np.int64)
    dirs = S.circle_directions(40)
    G = rng.integers(-1000, 1000, (40, 30)).astype(np.int64)
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(vw))
    g = h.backward(cuda(dirs), 30, -1.5, 1.5, cuda(G), 0.25).cpu().numpy()
    ref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, 30, -1.5, 1.5, G, 0.25)
    assert np.array_equal(g, ref)


def test_autograd_mse_small(P, oracle):
    """Volumes with f32 weights, loss = MSE(WECT(w), WECT(target)): the autograd gradient equals
    the oracle's exact adjoint of the loss, bit for bit.  N = count * d * T is a power of two, so
    the upstream 2 (W - B) 2^-24 / N is exact in float64 and its quantisation loses nothing."""
    count, side, d, T = 4, 9, 16, 32
    a = S.uniform_f32_grids(count, [side] * 3, seed=5)
    t = S.uniform_f32_grids(count, [side] * 3, seed=6)
    dirs = S.fibonacci_directions(d)
    bt = P.CubicalBatch([cuda(x) for x in t], frac_bits=24)
    B = bt.wect(cuda(dirs), T, -SQ3, SQ3).to(torch.float64) * 2.0 ** -24
    b = P.CubicalBatch([cuda(x) for x in a], frac_bits=24)
    w = cuda(a.reshape(-1)).requires_grad_(True)
    W = P.WECTFunction.apply(b, w, cuda(dirs), T, -SQ3, SQ3)
    loss = ((W - B) ** 2).mean()
    loss.backward()
    g = w.grad.detach().cpu().numpy().reshape(count, -1)
    N = count * d * T
    for i in range(count):
        vw = oracle.to_fixed(a[i], 24)
        Wi = oracle.wect_cubical([side] * 3, vw, dirs, T, -SQ3, SQ3)
        Bi = oracle.wect_cubical([side] * 3, oracle.to_fixed(t[i], 24), dirs, T, -SQ3, SQ3)
        ref = oracle.wect_backward_cubical([side] * 3, vw, dirs, T, -SQ3, SQ3, Wi - Bi, 2.0 ** -23 / N)
        assert np.array_equal(g[i], ref), i
