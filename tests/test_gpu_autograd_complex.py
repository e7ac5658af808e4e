"""The autograd function of one complex (grid or simplicial), through wect_backward_f64, against
the oracle's exact adjoint: loss = MSE(WECT(w), WECT(target)) with f32 weights at 2^-24 fixed
point.  d * T is a power of two, so the upstream 2 (W - B) 2^-24 / (d T) is exact in float64, its
quantisation loses nothing, and the gradient must equal the oracle's bit for bit."""
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


def _mse_grad(P, cx, w, B, dirs, T, lo, hi):
    wt = cuda(w).requires_grad_(True)
    W = P.ComplexWECTFunction.apply(cx, wt, cuda(dirs), T, lo, hi)
    loss = ((W - B) ** 2).mean()
    loss.backward()
    return wt.grad.detach().cpu().numpy(), W.detach().cpu().numpy()


@pytest.mark.parametrize("side,seed", [(24, 31), (41, 32)])
def test_simplicial_mesh_mse(P, oracle, side, seed):
    """Jittered triangulated mesh (vertices, edges, triangles), lognormal f32 weights."""
    cx = S.jittered_grid_mesh(side, seed=seed)
    tgt = S.jittered_grid_mesh(side, seed=seed + 100).weights
    dirs = S.circle_directions(16)
    T, lo, hi = 64, -1.5, 1.5
    sims = [cuda(s) for s in cx.simplices]
    h = P.SimplicialComplex(cuda(cx.coords), sims, cuda(cx.weights), frac_bits=24)
    ht = P.SimplicialComplex(cuda(cx.coords), sims, cuda(tgt), frac_bits=24)
    B = ht.wect(cuda(dirs), T, lo, hi).to(torch.float64) * 2.0 ** -24
    g, W = _mse_grad(P, h, cx.weights, B, dirs, T, lo, hi)
    vw = oracle.fixed_from_f32(cx.weights, 24)
    Wi = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
    vt = oracle.fixed_from_f32(tgt, 24)
    Bi = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vt), dirs, T, lo, hi)
    assert np.array_equal(W, Wi.astype(np.float64) * 2.0 ** -24)
    N = len(dirs) * T
    ref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, T, lo, hi, Wi - Bi, 2.0 ** -23 / N)
    assert np.array_equal(g, ref)
    h.device_status()


def test_simplicial_tetrahedra_mse(P, oracle):
    """A solid cube cut into tetrahedra (lists of dim 1, 2, 3), f32 weights, 3-D directions."""
    cx = S.tetra_grid(9, seed=33)
    rng = np.random.default_rng(34)
    w = rng.uniform(0.0, 1.0, len(cx.coords)).astype(np.float32)
    t = rng.uniform(0.0, 1.0, len(cx.coords)).astype(np.float32)
    dirs = S.fibonacci_directions(32)
    T, lo, hi = 32, -SQ3, SQ3
    sims = [cuda(s) for s in cx.simplices]
    h = P.SimplicialComplex(cuda(cx.coords), sims, cuda(w), frac_bits=24)
    ht = P.SimplicialComplex(cuda(cx.coords), sims, cuda(t), frac_bits=24)
    B = ht.wect(cuda(dirs), T, lo, hi).to(torch.float64) * 2.0 ** -24
    g, _ = _mse_grad(P, h, w, B, dirs, T, lo, hi)
    vw, vt = oracle.fixed_from_f32(w, 24), oracle.fixed_from_f32(t, 24)
    Wi = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
    Bi = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vt), dirs, T, lo, hi)
    N = len(dirs) * T
    ref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, T, lo, hi, Wi - Bi, 2.0 ** -23 / N)
    assert np.array_equal(g, ref)


@pytest.mark.parametrize("dims", [[23, 17], [11, 9, 7]])
def test_cubical_complex_mse(P, oracle, dims):
    """One grid (not a batch) through the same autograd function."""
    rng = np.random.default_rng(35)
    shape = tuple(reversed(dims))
    w = rng.uniform(0.0, 1.0, shape).astype(np.float32)
    t = rng.uniform(0.0, 1.0, shape).astype(np.float32)
    n = len(dims)
    dirs = S.circle_directions(32) if n == 2 else S.fibonacci_directions(32)
    T = 64
    lo, hi = (-SQ2, SQ2) if n == 2 else (-SQ3, SQ3)
    h = P.CubicalComplex(cuda(w), frac_bits=24)
    ht = P.CubicalComplex(cuda(t), frac_bits=24)
    B = ht.wect(cuda(dirs), T, lo, hi).to(torch.float64) * 2.0 ** -24
    g, _ = _mse_grad(P, h, w, B, dirs, T, lo, hi)
    vw, vt = oracle.to_fixed(w, 24), oracle.to_fixed(t, 24)
    Wi = oracle.wect_cubical(dims, vw, dirs, T, lo, hi)
    Bi = oracle.wect_cubical(dims, vt, dirs, T, lo, hi)
    N = len(dirs) * T
    ref = oracle.wect_backward_cubical(dims, vw, dirs, T, lo, hi, Wi - Bi, 2.0 ** -23 / N)
    assert np.array_equal(g.reshape(-1), ref.reshape(-1))


def test_backward_f64_default_range_and_nonfinite_upstream(P, oracle):
    """The default range resolves as in the forward; a NaN in the upstream counts as zero and is
    reported by the device status."""
    cx = S.jittered_grid_mesh(17, seed=36)
    dirs = S.circle_directions(8)
    T = 16
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(cx.weights), frac_bits=24)
    G = np.random.default_rng(37).integers(-64, 64, (len(dirs), T)).astype(np.float64) * 2.0 ** -10
    g = h.backward_f64(cuda(dirs), T, math.nan, math.nan, cuda(G)).cpu().numpy()
    vw = oracle.fixed_from_f32(cx.weights, 24)
    lo, hi = oracle.default_range_simplicial(cx.coords, dirs)
    ref = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, T, lo, hi,
                                          (G * 2.0 ** 10).astype(np.int64), 2.0 ** -10)
    assert np.array_equal(g, ref)
    h.device_status()
    G2 = G.copy()
    G2[3, 5] = math.nan
    h.backward_f64(cuda(dirs), T, -1.5, 1.5, cuda(G2))
    with pytest.raises(P.WectError):
        h.device_status()
    h.device_status()                  # cleared by the read


def test_simplicial_gradient_matches_central_differences(P):
    """Central differences (h = 2^-10 ~ 1e-3) of an MSE loss through ComplexWECTFunction on a
    triangulated mesh, at vertices whose weight differs from every neighbour's by more than 2h
    (away from ties the transform is linear in the weight, so the difference quotient is exact
    up to float64 rounding): within 1e-6 relative of the autograd gradient."""
    cx = S.jittered_grid_mesh(20, seed=38)
    rng = np.random.default_rng(39)
    # dyadic weights (multiples of 2^-10), so w +- h is exact in float32 and in 2^-24 fixed point
    w = (np.floor(cx.weights.astype(np.float64) * 1024.0) / 1024.0).astype(np.float32)
    t = (np.floor(rng.lognormal(0.0, 1.0, w.size) * 1024.0) / 1024.0).astype(np.float32)
    dirs = S.circle_directions(16)
    T, lo, hi = 64, -1.5, 1.5
    sims = [cuda(s) for s in cx.simplices]
    h = P.SimplicialComplex(cuda(cx.coords), sims, cuda(w), frac_bits=24)
    ht = P.SimplicialComplex(cuda(cx.coords), sims, cuda(t), frac_bits=24)
    B = ht.wect(cuda(dirs), T, lo, hi).to(torch.float64) * 2.0 ** -24

    def loss_of(wv):
        W = P.ComplexWECTFunction.apply(h, cuda(wv), cuda(dirs), T, lo, hi)
        return float(((W - B) ** 2).mean())

    g, _ = _mse_grad(P, h, w, B, dirs, T, lo, hi)
    step = 2.0 ** -10
    nbr = [set() for _ in range(w.size)]
    for e in cx.simplices[0]:
        nbr[int(e[0])].add(int(e[1]))
        nbr[int(e[1])].add(int(e[0]))
    free = [v for v in range(w.size) if nbr[v] and all(abs(float(w[v]) - float(w[u])) > 2 * step for u in nbr[v])]
    assert len(free) >= 20
    picked = [free[i] for i in rng.choice(len(free), 20, replace=False)]
    checked = 0
    for v in picked:
        wp, wm = w.copy(), w.copy()
        wp[v] += np.float32(step)
        wm[v] -= np.float32(step)
        fd = (loss_of(wp) - loss_of(wm)) / (2 * step)
        if fd == 0.0 and g[v] == 0.0:
            continue
        assert abs(g[v] - fd) <= 1e-6 * max(abs(fd), abs(float(g[v]))), (v, g[v], fd)
        checked += 1
    assert checked >= 10
