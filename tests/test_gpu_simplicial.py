"""GPU parity of the simplicial (gather) path against the CPU oracle."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import cuda, dev, lib, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


def _make(P, cx, weights, fb=0, explicit=None):
    sim = [cuda(s) for s in cx.simplices]
    w = None if weights is None else cuda(weights)
    sw = None if explicit is None else [cuda(e) for e in explicit]
    return P.SimplicialComplex(cuda(cx.coords), sim, w, frac_bits=fb, simplex_weights=sw)


@pytest.mark.parametrize("seed", range(4))
def test_random_complexes(P, oracle, seed):
    n = 2 + seed % 2
    cx = S.random_simplicial(300 + 37 * seed, n, 900, 500, seed=seed)
    dirs = S.random_directions(45, n, seed + 10)
    T, lo, hi = [(33, -1.5, 1.5), (64, math.nan, math.nan), (2, -1.0, 1.0), (200, -0.3, 0.2)][seed]
    h = _make(P, cx, cx.weights)
    got = h.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    vw = cx.weights.astype(np.int64)
    ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
    assert np.array_equal(got, ref)
    h.device_status()


def test_closed_surfaces_and_explicit_weights(P, oracle):
    tor = S.torus_mesh(12, 9)
    h = _make(P, tor, None)
    dirs = S.fibonacci_directions(33)
    got = h.wect(cuda(dirs), 40).cpu().numpy()
    ref = oracle.wect_simplicial(tor.coords, tor.simplices,
                                 oracle.simplicial_weights(tor.simplices, np.ones(tor.nv, np.int64), "one"), dirs, 40)
    assert np.array_equal(got, ref)
    assert np.all(got[:, -1] == 0)
    rng = np.random.default_rng(3)
    ex = [rng.integers(-1000, 1000, tor.nv).astype(np.int64)] + \
         [rng.integers(-1000, 1000, len(s)).astype(np.int64) for s in tor.simplices]
    h2 = _make(P, tor, None, explicit=ex)
    got = h2.wect(cuda(dirs), 40, -3.0, 3.0).cpu().numpy()
    ref = oracle.wect_simplicial(tor.coords, tor.simplices, ex, dirs, 40, -3.0, 3.0)
    assert np.array_equal(got, ref)


def test_vertex_only_and_point(P, oracle):
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (500, 2))
    w = rng.integers(0, 256, 500, dtype=np.uint8)
    cx = S.Simplicial(coords=X, simplices=[], weights=w)
    h = _make(P, cx, w)
    dirs = S.circle_directions(40)
    got = h.wect(cuda(dirs), 25, -1.2, 1.2).cpu().numpy()
    ref = oracle.wect_simplicial(X, [], [w.astype(np.int64)], dirs, 25, -1.2, 1.2)
    assert np.array_equal(got, ref)
    pt = S.Simplicial(coords=np.zeros((1, 3)), simplices=[], weights=np.array([1], np.uint8))
    got = _make(P, pt, pt.weights).wect(cuda(S.fibonacci_directions(4)), 5).cpu().numpy()
    assert np.all(got == 1)


def test_mesh_small_lognormal_fixed_point(P, oracle):
    """Jittered 96x96 mesh with f32 lognormal weights at 2^-24 (the 1024^2 workload's recipe,
    smaller), default range."""
    cx = S.jittered_grid_mesh(96, seed=3)
    dirs = S.circle_directions(100)
    h = _make(P, cx, cx.weights, fb=24)
    got = h.wect(cuda(dirs), 512).cpu().numpy()
    vw = oracle.fixed_from_f32(cx.weights, 24)
    ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, 512)
    assert np.array_equal(got, ref)


def test_ecf_simplicial(P, oracle):
    cx = S.random_simplicial(200, 2, 500, 300, seed=7)
    rng = np.random.default_rng(7)
    f = rng.standard_normal(cx.nv)
    h = _make(P, cx, cx.weights)
    for weighted in (False, True):
        got = h.ecf(cuda(f), 40, -2.0, 2.0, weighted=weighted).cpu().numpy()
        vw = cx.weights.astype(np.int64)
        ws = oracle.simplicial_weights(cx.simplices, vw, "max" if weighted else "one")
        ref = oracle.wecf_simplicial(f, cx.simplices, ws, 40, -2.0, 2.0)[0]
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("T", [2, 1000, 30000, 60000])
def test_ecf_simplicial_histogram_modes(P, oracle, T):
    """Per-block int32 histograms, int64 ones (f32 weights at 2^-24), and global atomics once T
    no longer fits shared memory; values on the thresholds."""
    cx = S.random_simplicial(300, 3, 900, 700, seed=17)
    rng = np.random.default_rng(T)
    beta = oracle.beta(T, -1.5, 1.5)
    f = rng.uniform(-1.7, 1.7, cx.nv)
    f[: min(cx.nv, T) // 2] = rng.choice(beta, size=min(cx.nv, T) // 2)
    for kind in ("u8", "f32"):
        w = cx.weights if kind == "u8" else rng.random(cx.nv, dtype=np.float32) * 3
        h = P.SimplicialComplex(cuda(cx.coords), [cuda(x) for x in cx.simplices], cuda(w),
                                frac_bits=24 if kind == "f32" else 0)
        vw = w.astype(np.int64) if kind == "u8" else oracle.to_fixed(w, 24)
        for weighted in (False, True):
            got = h.ecf(cuda(f), T, -1.5, 1.5, weighted=weighted).cpu().numpy()
            ws = oracle.simplicial_weights(cx.simplices, vw, "max" if weighted else "one")
            ref = oracle.wecf_simplicial(f, cx.simplices, ws, T, -1.5, 1.5)[0]
            assert np.array_equal(got, ref), (kind, weighted)


def test_bad_indices_rejected(P):
    X = np.zeros((4, 2))
    E = np.array([[0, 1], [2, 7]], dtype=np.int32)
    cx = S.Simplicial(coords=X, simplices=[E], weights=np.ones(4, np.uint8))
    with pytest.raises(P.WectError) as ei:
        _make(P, cx, cx.weights)
    assert ei.value.name == "INVALID_ARG"
    X2 = X.copy()
    X2[1, 0] = np.nan
    cx2 = S.Simplicial(coords=X2, simplices=[E[:1]], weights=np.ones(4, np.uint8))
    with pytest.raises(P.WectError):
        _make(P, cx2, cx2.weights)


def test_staged_and_direct_chunks(P, oracle):
    """Lists are cut into chunks. A chunk that references at most a shared-memory window of
    distinct vertices is staged through shared memory; a larger one reads global memory. The
    complexes here mix both kinds: a 160^2 mesh whose triangle list is shuffled in its second
    half, and a random complex on 20000 vertices, where every chunk reads global memory."""
    cx = S.jittered_grid_mesh(160, seed=11)
    tri = cx.simplices[1].copy()
    half = len(tri) // 2
    tri[half:] = tri[half:][np.random.default_rng(12).permutation(len(tri) - half)]
    mixed = S.Simplicial(cx.coords, [cx.simplices[0], tri], cx.weights)
    rnd = S.random_simplicial(20000, 2, 6000, 4000, seed=13)
    dirs = S.circle_directions(40)
    for c, fb, rng_ in ((mixed, 24, (-1.5, 1.5)), (mixed, 24, (math.nan, math.nan)), (rnd, 0, (-1.2, 1.3))):
        h = _make(P, c, c.weights, fb=fb)
        got = h.wect(cuda(dirs), 64, *rng_).cpu().numpy()
        vw = oracle.fixed_from_f32(c.weights, fb) if fb else c.weights.astype(np.int64)
        ref = oracle.wect_simplicial(c.coords, c.simplices, oracle.simplicial_weights(c.simplices, vw), dirs, 64, *rng_)
        assert np.array_equal(got, ref)
        h.device_status()


def test_tetrahedral_grid_forward_and_adjoint(P, oracle):
    """A 12^3 solid cube cut into tetrahedra (lists of dim 1, 2 and 3), u8 weights: the forward
    with the default and a fixed range, and the adjoint, against the oracle."""
    cx = S.tetra_grid(12, seed=22)
    dirs = S.fibonacci_directions(70)
    vw = cx.weights.astype(np.int64)
    h = _make(P, cx, cx.weights)
    for T, lo, hi in ((64, math.nan, math.nan), (97, -1.5, 1.6)):
        got = h.wect(cuda(dirs), T, lo, hi).cpu().numpy()
        ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
        assert np.array_equal(got, ref)
    G = np.random.default_rng(23).integers(-5000, 5000, (len(dirs), 40)).astype(np.int64)
    g = h.backward(cuda(dirs), 40, -1.5, 1.6, cuda(G), 0.5).cpu().numpy()
    ref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, 40, -1.5, 1.6, G, 0.5)
    assert np.array_equal(g, ref)
    h.device_status()
