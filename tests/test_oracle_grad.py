"""Pins of the oracle's exact adjoint (no GPU): central finite differences of the oracle's own
forward transform, which are exact here because the loss is quadratic in the transform and the
transform is linear in each vertex weight away from ties of the per-simplex maximum."""
import math

import numpy as np

import synthetic as S


def _loss_int(W, B):
    """sum (W - B)^2 as an exact Python integer."""
    D = (W.astype(object) - B.astype(object)).ravel()
    return sum(int(x) * int(x) for x in D)


def _tie_free(vw_fix, dims, k, v):
    """True when no vertex sharing a cell with v has a fixed weight within k of v's."""
    n = len(dims)
    idx = []
    r = v
    for a in range(n):
        idx.append(r % dims[a])
        r //= dims[a]
    strides = [int(np.prod(dims[:a])) for a in range(n)]
    for off in np.ndindex(*([3] * n)):
        u = [idx[a] + off[a] - 1 for a in range(n)]
        if any(u[a] < 0 or u[a] >= dims[a] for a in range(n)) or all(o == 1 for o in off):
            continue
        uv = sum(u[a] * strides[a] for a in range(n))
        if abs(int(vw_fix[uv]) - int(vw_fix[v])) <= 2 * k:
            return False
    return True


def test_cubical_adjoint_equals_finite_differences(oracle):
    dims = [5, 4, 3]
    nv = int(np.prod(dims))
    rng = np.random.default_rng(31)
    w = rng.random(nv, dtype=np.float32)
    wt = rng.random(nv, dtype=np.float32)
    dirs = S.fibonacci_directions(7)
    T, lo, hi = 9, -math.sqrt(3), math.sqrt(3)
    frac = 24
    vw = oracle.fixed_from_f32(w, frac)
    B = oracle.wect_cubical(dims, oracle.fixed_from_f32(wt, frac), dirs, T, lo, hi)
    W = oracle.wect_cubical(dims, vw, dirs, T, lo, hi)
    N = W.size
    # exact adjoint of L = (1/N) sum (W_real - B_real)^2 with W_real = W * 2^-24
    g = oracle.wect_backward_cubical(dims, vw, dirs, T, lo, hi, W - B, 2.0 ** (1 - frac) / N)
    k = 1 << 14                                         # perturbation of the fixed weight (~1e-3)
    tested = 0
    for v in range(nv):
        if not _tie_free(vw, dims, k, v):
            continue
        vp, vm = vw.copy(), vw.copy()
        vp[v] += k
        vm[v] -= k
        Lp = _loss_int(oracle.wect_cubical(dims, vp, dirs, T, lo, hi), B)
        Lm = _loss_int(oracle.wect_cubical(dims, vm, dirs, T, lo, hi), B)
        # dL/dw = (Lp - Lm) * 2^-48 / N / (2 k 2^-24), computed exactly then rounded
        from fractions import Fraction

        fd = Fraction(Lp - Lm, 2 * k * N) * Fraction(1, 1 << 24)
        assert abs(float(fd) - float(g[v])) <= 1e-6 * max(abs(float(fd)), 1e-12)
        tested += 1
    assert tested >= 5


def test_simplicial_adjoint_equals_finite_differences(oracle):
    cx = S.random_simplicial(14, 2, 24, 12, seed=32)
    rng = np.random.default_rng(33)
    vw = rng.integers(0, 1 << 20, cx.nv).astype(np.int64)
    dirs = S.circle_directions(6)
    T, lo, hi = 10, -1.5, 1.5
    G = rng.integers(-1000, 1000, (6, T)).astype(np.int64)
    g = oracle.wect_backward_simplicial(cx.coords, vw, cx.simplices, dirs, T, lo, hi, G, 1.0)

    def lin(vv):  # <G, W(vv)>: linear in the weights, so its difference quotient is exact
        W = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vv), dirs, T, lo, hi)
        return int((W.astype(object) * G.astype(object)).sum())

    # dW[p][q]/dw = sum_{q'} ... ; the adjoint maps G to sum_{p,q} G[p,q] dW[p,q]/dw_v
    k = 3
    nbrs = {v: set() for v in range(cx.nv)}
    for lst in cx.simplices:
        for row in lst:
            for a in row:
                nbrs[int(a)].update(int(b) for b in row if b != a)
    tested = 0
    for v in range(cx.nv):
        if any(abs(int(vw[u]) - int(vw[v])) <= k for u in nbrs[v]):
            continue
        vp, vm = vw.copy(), vw.copy()
        vp[v] += k
        vm[v] -= k
        fd = (lin(vp) - lin(vm)) / (2 * k)
        assert float(g[v]) == float(np.float32(fd))
        tested += 1
    assert tested >= 5


def test_cubical_and_simplicial_adjoints_agree_on_a_path(oracle):
    L = 17
    rng = np.random.default_rng(34)
    vw = rng.integers(0, 1000, L).astype(np.int64)
    X = oracle.grid_coords([L])
    E = np.stack([np.arange(L - 1), np.arange(1, L)], 1).astype(np.int32)
    dirs = np.array([[1.0], [-1.0], [0.25]])
    G = rng.integers(-50, 50, (3, 8)).astype(np.int64)
    a = oracle.wect_backward_cubical([L], vw, dirs, 8, -1.0, 1.0, G, 0.5)
    b = oracle.wect_backward_simplicial(X, vw, [E], dirs, 8, -1.0, 1.0, G, 0.5)
    assert np.array_equal(a, b)


# Tie-break of the adjoint, worked by hand from its definition.  The path of 4 vertices at
# x = -1, -1/3, 1/3, 1 (a 1-D grid of length 4), weights w = (5, 9, 9, 2), direction s = (1),
# T = 3 over [-1, 1]: beta = (-1, 0, 1), and bin(h) = #{q <= 1 : beta[q] < h} gives the vertex
# bins (0, 1, 2, 2).  A cell's bin is that of its highest vertex: edges (0,1) -> 1, (1,2) -> 2,
# (2,3) -> 2.  Upstream G = (1, 10, 100), suffix sums S = (111, 110, 100).
#   vertices (sign +): I0 += S[0] = 111, I1 += S[1] = 110, I2 += S[2] = 100, I3 += S[2] = 100
#   edge (0,1), heaviest vertex 1:                 I1 -= S[1] -> I1 = 0
#   edge (1,2), weights 9 = 9, lowest index is 1:  I1 -= S[2] -> I1 = -100
#   edge (2,3), heaviest vertex 2:                 I2 -= S[2] -> I2 = 0
# so I = (111, -100, 0, 100).  Routing the tie to the highest index would give (111, 0, -100, 100).
_TIE_W = np.array([5, 9, 9, 2], dtype=np.int64)
_TIE_G = np.array([[1, 10, 100]], dtype=np.int64)
_TIE_I = np.array([111, -100, 0, 100], dtype=np.float32)


def test_adjoint_tie_break_cubical_by_hand(oracle):
    g = oracle.wect_backward_cubical([4], _TIE_W, np.array([[1.0]]), 3, -1.0, 1.0, _TIE_G, 1.0)
    assert np.array_equal(g, _TIE_I)


def test_adjoint_tie_break_simplicial_by_hand(oracle):
    """The same path as a simplicial complex, with the tied edge listed as (2, 1): the tie goes
    to the lower vertex index, not to the first vertex of the row."""
    X = np.array([[-1.0], [-1.0 / 3.0], [1.0 / 3.0], [1.0]])
    E = np.array([[0, 1], [2, 1], [2, 3]], dtype=np.int32)
    g = oracle.wect_backward_simplicial(X, _TIE_W, [E], np.array([[1.0]]), 3, -1.0, 1.0, _TIE_G, 1.0)
    assert np.array_equal(g, _TIE_I)
