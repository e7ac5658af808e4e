"""Pins of the CPU oracle to facts outside itself (no GPU).

Each test checks the oracle against something the paper or mathematics fixes: the
appendix's worked examples, exact rational arithmetic, closed-form Euler characteristics,
library routines for special cases, invariances, and brute-force enumeration of the
sublevel subcomplexes of tiny complexes.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------- helpers (exact)


def rn(x: Fraction) -> float:
    """Round a rational to the nearest float64 (ties to even): CPython's int/int division is
    correctly rounded, and Fraction.__float__ uses it."""
    return float(x)


def fma_exact(a: float, b: float, c: float) -> float:
    return rn(Fraction(a) * Fraction(b) + Fraction(c))


def height_reading(x, s) -> float:
    """Independent restatement of the height rounding rule: RN(x[n-1] s[n-1]), then fma from n-2 to 0."""
    n = len(x)
    h = rn(Fraction(x[n - 1]) * Fraction(s[n - 1]))
    for c in range(n - 2, -1, -1):
        h = fma_exact(x[c], s[c], h)
    return h


def face_dim(s, cubical=False):
    """Dimension of a simplex (vertices - 1) or of a cubical cell (log2 of its vertex count)."""
    return (len(s).bit_length() - 1) if cubical else len(s) - 1


def brute_wecf(nv, faces, weights, f, T, beta, cubical=False):
    """Brute force over sublevel subcomplexes: for each threshold q <= T-2 the subcomplex
    F(beta[q]) = {s : every vertex v of s has f(v) <= beta[q]} (Definition "Lower-Star
    Filtrations"), and W[q] = sum over F(beta[q]) of (-1)^dim(s) w(s); the top column is the
    sum over the whole complex.  faces: list of vertex tuples; weights: same order."""
    sign = [(-1) ** face_dim(s, cubical) for s in faces]
    W = []
    for q in range(T - 1):
        tot = 0
        for s, w, e in zip(faces, weights, sign):
            if all(f[v] <= beta[q] for v in s):
                tot += e * w
        W.append(tot)
    W.append(sum(e * w for w, e in zip(weights, sign)))
    return W


def cubical_cells(dims):
    """All boxes (corner, extent mask) of a grid as vertex tuples (axis 0 fastest)."""
    n = len(dims)
    strides = [int(np.prod(dims[:a])) for a in range(n)]
    cells = []
    for corner in itertools.product(*[range(L) for L in dims]):
        for e in itertools.product((0, 1), repeat=n):
            if any(corner[a] + e[a] > dims[a] - 1 for a in range(n)):
                continue
            verts = []
            for sub in itertools.product(*[(0, 1) if e[a] else (0,) for a in range(n)]):
                verts.append(sum((corner[a] + sub[a]) * strides[a] for a in range(n)))
            cells.append(tuple(verts))
    return cells


def simplicial_faces(cx, vw):
    """Flat face list and max-of-vertex weights of a Simplicial."""
    faces = [(v,) for v in range(cx.nv)]
    for lst in cx.simplices:
        faces += [tuple(int(x) for x in row) for row in lst]
    weights = [max(int(vw[v]) for v in s) for s in faces]
    return faces, weights


# ----------------------------------------------------------------------- appendix examples


def _golden_rows(key):
    with open(os.path.join(GOLDEN, "appendix_tensor_ops.txt")) as fh:
        for line in fh:
            if line.startswith(key + " "):
                body = line[len(key) + 1:]
                return np.array([[int(t) for t in r.split()] for r in body.split(";")], dtype=np.int64)
    raise KeyError(key)


def test_appendix_cumsum(oracle):
    T = np.array([[1, 2], [3, 4], [5, 6]], dtype=np.int64)
    assert np.array_equal(oracle.cumsum_rows(T), _golden_rows("cumsum"))


def test_appendix_rmax(oracle):
    T = np.array([[1, 2], [3, 4], [5, 6]], dtype=np.int64)
    assert np.array_equal(oracle.rmax_rows(T).reshape(-1, 1), _golden_rows("rmax"))


def test_appendix_scatter_add(oracle):
    Sm = np.array([[1, 3, 5], [2, 4, 6]], dtype=np.int64)
    U = np.array([[1], [2]], dtype=np.int64)
    V = np.array([5], dtype=np.int64)
    assert np.array_equal(oracle.scatter_add(Sm, U, V), _golden_rows("scatter_add"))


# ----------------------------------------------------------------------- arithmetic readings


def test_height_rounding_matches_exact_fma_reading(oracle):
    rng = np.random.default_rng(11)
    for n in (1, 2, 3, 4):
        for _ in range(400):
            x = rng.uniform(-1, 1, n) * (2.0 ** rng.integers(-3, 3, n))
            s = rng.standard_normal(n)
            assert oracle.height(x, s) == height_reading(list(x), list(s))


def test_height_order_is_not_symmetric(oracle):
    # A transposed fma order gives a different float on some inputs; the pin above would catch it.
    rng = np.random.default_rng(12)
    diff = 0
    for _ in range(2000):
        x = rng.uniform(-1, 1, 3)
        s = rng.standard_normal(3)
        rev = rn(Fraction(x[0]) * Fraction(s[0]))
        rev = fma_exact(x[1], s[1], rev)
        rev = fma_exact(x[2], s[2], rev)
        diff += oracle.height(x, s) != rev
    assert diff > 0


def test_beta_against_exact_rationals(oracle):
    for T, lo, hi in [(64, -math.sqrt(2), math.sqrt(2)), (128, -math.sqrt(3), math.sqrt(3)), (2, -1.0, 3.0),
                      (513, -0.7, 1.3), (17, -2.0, 2.0)]:
        b = oracle.beta(T, lo, hi)
        assert b[0] == lo
        assert np.all(np.diff(b) >= 0)
        for q in range(T):
            exact = Fraction(lo) + q * (Fraction(hi) - Fraction(lo)) / (T - 1)
            assert abs(Fraction(b[q]) - exact) <= Fraction(4 * T) * Fraction(2) ** -52 * (abs(Fraction(lo)) + abs(Fraction(hi)))
    # exact dyadic case: every beta is exact
    b = oracle.beta(17, -2.0, 2.0)
    assert list(b) == [-2.0 + 0.25 * q for q in range(17)]


def test_beta_degenerate_range(oracle):
    b = oracle.beta(8, 0.5, 0.5)
    assert np.all(b == 0.5)
    assert oracle.bin_of(0.5, b) == 0
    assert oracle.bin_of(np.nextafter(0.5, 1.0), b) == 7


def test_bin_galois_exhaustive(oracle):
    """Eq. "galois": bin(t) <= q  <=>  t <= beta[q], for q <= T-2, checked at every threshold and
    its float neighbours; values above hi clamp to T-1 and values below lo go to 0."""
    for T, lo, hi in [(64, -math.sqrt(2), math.sqrt(2)), (128, -math.sqrt(3), math.sqrt(3)), (7, -1.0, 1.0)]:
        b = oracle.beta(T, lo, hi)
        for q in range(T - 1):
            for t in (b[q], np.nextafter(b[q], -np.inf), np.nextafter(b[q], np.inf)):
                k = oracle.bin_of(t, b)
                for qq in range(T - 1):
                    assert (k <= qq) == (t <= b[qq])
        assert oracle.bin_of(hi + 1.0, b) == T - 1
        assert oracle.bin_of(lo - 1.0, b) == 0


def test_bin_matches_searchsorted(oracle):
    rng = np.random.default_rng(13)
    b = oracle.beta(100, -1.5, 1.5)
    ts = np.concatenate([rng.uniform(-2, 2, 500), b, np.nextafter(b, np.inf)])
    ref = np.searchsorted(b[:-1], ts, side="left")     # #{q <= T-2 : beta[q] < t}
    got = np.array([oracle.bin_of(t, b) for t in ts])
    assert np.array_equal(got, ref)


def test_grid_coords(oracle):
    for L in (1, 2, 3, 28, 64, 127, 128, 256):
        xs = [oracle.grid_coord(i, L) for i in range(L)]
        if L == 1:
            assert xs == [0.0]
            continue
        assert xs[0] == -1.0 and xs[-1] == 1.0
        for i in range(L):
            assert xs[i] == rn(Fraction(2 * i - (L - 1), L - 1))
            assert xs[i] == -xs[L - 1 - i]


def test_fixed_point_conversion(oracle):
    rng = np.random.default_rng(14)
    w = np.concatenate([rng.random(1000, dtype=np.float32), rng.lognormal(0, 1, 1000).astype(np.float32),
                        np.array([0.0, 1.0, 2.0 ** -25, 3 * 2.0 ** -25, -2.0 ** -25], dtype=np.float32)])
    got = oracle.fixed_from_f32(w, 24)
    ref = np.array([round(float(x) * 2 ** 24) for x in w], dtype=np.int64)    # round-half-even
    assert np.array_equal(got, ref)


def test_i128_to_double_rounding(oracle):
    rng = np.random.default_rng(15)
    vals = [0, 1, -1, 2 ** 53 + 1, 2 ** 53 + 3, -(2 ** 70) - 2 ** 17, (1 << 100) + (1 << 47), -(1 << 126)]
    vals += [int(rng.integers(-2 ** 62, 2 ** 62)) * int(rng.integers(1, 2 ** 40)) for _ in range(200)]
    for v in vals:
        assert oracle.i128_to_double(v) == float(v)


# ----------------------------------------------------------------------- special cases


def test_vertex_only_complex_is_weighted_histogram(oracle):
    """A complex with vertices only: W[p] = cumsum of the weighted histogram of bins."""
    rng = np.random.default_rng(16)
    X = rng.uniform(-1, 1, (300, 2))
    w = rng.integers(-50, 200, 300).astype(np.int64)
    dirs = S.random_directions(5, 2, seed=17)
    T, lo, hi = 33, -1.2, 1.2
    got = oracle.wect_simplicial(X, [], [w], dirs, T, lo, hi)
    b = oracle.beta(T, lo, hi)
    for p in range(5):
        h = np.array([oracle.height(X[v], dirs[p]) for v in range(300)])
        bins = np.searchsorted(b[:-1], h, side="left")
        ref = np.cumsum(np.bincount(bins, weights=w, minlength=T).astype(np.int64))
        assert np.array_equal(got[p], ref)


def test_max_of_bins_equals_bin_of_max(oracle):
    """Eq. "msi": alpha is order-preserving, so the bin of the max is the max of the bins."""
    rng = np.random.default_rng(18)
    b = oracle.beta(50, -1.0, 1.0)
    for _ in range(300):
        h = rng.uniform(-1.2, 1.2, rng.integers(1, 5))
        if rng.random() < 0.3:
            h[0] = b[rng.integers(0, 49)]
        assert oracle.bin_of(h.max(), b) == max(oracle.bin_of(t, b) for t in h)


# ----------------------------------------------------------------------- closed forms


def test_point_complex(oracle):
    out = oracle.wect_simplicial(np.zeros((1, 2)), [], [np.array([1], dtype=np.int64)], S.circle_directions(4), 5)
    # default range with M = 0: beta all 0, the point (height 0) is in bin 0 for every direction
    assert np.all(out == 1)


def test_closed_forms_top_column(oracle):
    # torus: chi = 0; octahedron surface (a 2-sphere): chi = 2
    tor = S.torus_mesh(6, 5)
    one = lambda cx: oracle.simplicial_weights(cx.simplices, np.ones(cx.nv, dtype=np.int64), "one")
    W = oracle.wect_simplicial(tor.coords, tor.simplices, one(tor), S.fibonacci_directions(7), 9)
    assert np.all(W[:, -1] == 0)
    octa = S.octahedron_surface()
    W = oracle.wect_simplicial(octa.coords, octa.simplices, one(octa), S.fibonacci_directions(7), 9)
    assert np.all(W[:, -1] == 2)
    # triangulated disc (jittered square mesh) and the solid square / cube grids: chi = 1
    disc = S.jittered_grid_mesh(6, seed=5)
    W = oracle.wect_simplicial(disc.coords, disc.simplices, one(disc), S.circle_directions(6), 9)
    assert np.all(W[:, -1] == 1)
    for dims in ([1], [5], [4, 3], [3, 4, 2]):
        n = len(dims)
        dirs = S.fibonacci_directions(5) if n == 3 else (S.circle_directions(5) if n == 2 else np.array([[1.0], [-1.0]]))
        W = oracle.wect_cubical(dims, np.zeros(int(np.prod(dims)), dtype=np.int64), dirs, 7,
                                -math.sqrt(n), math.sqrt(n), weighted=False)
        assert np.all(W[:, -1] == 1)


def test_full_grid_staircase(oracle):
    """The sublevel set of a full grid under a linear height is a down-set of the grid in the
    sign order, hence contractible: the unweighted ECF is 1 from min_v h on and 0 below."""
    rng = np.random.default_rng(19)
    for dims in ([6, 5], [4, 3, 5], [9], [7, 7]):
        n = len(dims)
        dirs = S.random_directions(6, n, seed=int(rng.integers(1 << 30)))
        T = 23
        lo, hi = -math.sqrt(n), math.sqrt(n)
        W = oracle.wect_cubical(dims, np.zeros(int(np.prod(dims)), dtype=np.int64), dirs, T, lo, hi, weighted=False)
        b = oracle.beta(T, lo, hi)
        X = oracle.grid_coords(dims)
        for p in range(len(dirs)):
            hmin = min(oracle.height(X[v], dirs[p]) for v in range(len(X)))
            ref = np.array([1 if (b[q] >= hmin or q == T - 1) else 0 for q in range(T)])
            assert np.array_equal(W[p], ref)


def test_grid2d_ecf_of_direction_x(oracle):
    """The unweighted ECF of the 64x64 grid for the filter f = x: ECF[q] = [beta[q] >= -1]."""
    dims = [64, 64]
    X = oracle.grid_coords(dims)
    T = 64
    lo, hi = -math.sqrt(2), math.sqrt(2)
    E = oracle.wecf_cubical(dims, np.zeros(64 * 64, dtype=np.int64), X[:, 0], T, lo, hi, weighted=False)[0]
    b = oracle.beta(T, lo, hi)
    assert np.array_equal(E, np.array([1 if (b[q] >= -1.0 or q == T - 1) else 0 for q in range(T)]))


# ----------------------------------------------------------------------- brute force


def test_brute_force_simplicial_exact_dyadic(oracle):
    """Tiny random complexes with dyadic coordinates and directions (all products, sums and
    thresholds exact): the oracle equals brute-force enumeration in rational arithmetic."""
    for seed in range(6):
        cx = S.random_simplicial(10, 2 + seed % 2, 14, 6, seed=100 + seed, coord_bits=3)
        rng = np.random.default_rng(200 + seed)
        dirs = rng.integers(-8, 9, size=(4, cx.n)).astype(np.float64) / 8.0
        T, lo, hi = 17, -2.0, 2.0
        vw = cx.weights.astype(np.int64)
        got = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
        faces, weights = simplicial_faces(cx, vw)
        beta = [Fraction(lo) + q * (Fraction(hi) - Fraction(lo)) / (T - 1) for q in range(T)]
        for p in range(len(dirs)):
            f = [sum(Fraction(cx.coords[v, a]) * Fraction(dirs[p, a]) for a in range(cx.n)) for v in range(cx.nv)]
            assert got[p].tolist() == brute_wecf(cx.nv, faces, weights, f, T, beta)


def test_brute_force_simplicial_rounding(oracle):
    """Non-dyadic inputs: brute force with float64 heights from the exact-fma restatement of
    the rounding rule and float64 thresholds."""
    for seed in range(4):
        cx = S.random_simplicial(11, 3, 16, 8, seed=300 + seed)
        dirs = S.random_directions(5, 3, seed=400 + seed)
        T, lo, hi = 12, -1.3, 1.1
        vw = cx.weights.astype(np.int64)
        got = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
        faces, weights = simplicial_faces(cx, vw)
        step = (hi - lo) / (T - 1)
        beta = [lo + q * step for q in range(T)]
        for p in range(len(dirs)):
            f = [height_reading(list(cx.coords[v]), list(dirs[p])) for v in range(cx.nv)]
            assert got[p].tolist() == brute_wecf(cx.nv, faces, weights, f, T, beta)


def test_freudenthal_triangulation_of_grids(oracle):
    """The Freudenthal triangulation of a full grid is a triangulated box: Euler characteristic
    1 at the top threshold in every direction."""
    for dims in ([6], [5, 4], [3, 4, 3]):
        n = len(dims)
        lists = S.freudenthal_lists(dims)
        X = oracle.grid_coords(dims)
        nv = X.shape[0]
        one = oracle.simplicial_weights(lists, np.ones(nv, dtype=np.int64), "one")
        dirs = S.fibonacci_directions(5) if n == 3 else (S.circle_directions(5) if n == 2 else np.array([[1.0], [-1.0]]))
        W = oracle.wect_simplicial(X, lists, one, dirs, 9)
        assert np.all(W[:, -1] == 1)


def test_tetrahedral_solid_cube(oracle):
    """Lists with tetrahedra: a triangulated solid cube (six tetrahedra per cell) has Euler
    characteristic 1, and brute-force enumeration of its sublevel subcomplexes (float64
    heights from the exact-fma restatement) equals the oracle, weights included."""
    cx = S.tetra_grid(3, seed=21)
    one = oracle.simplicial_weights(cx.simplices, np.ones(cx.nv, dtype=np.int64), "one")
    dirs = S.fibonacci_directions(6)
    W = oracle.wect_simplicial(cx.coords, cx.simplices, one, dirs, 11)
    assert np.all(W[:, -1] == 1)
    vw = cx.weights.astype(np.int64)
    T, lo, hi = 13, -1.6, 1.7
    got = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, lo, hi)
    faces, weights = simplicial_faces(cx, vw)
    step = (hi - lo) / (T - 1)
    beta = [lo + q * step for q in range(T)]
    for p in range(len(dirs)):
        f = [height_reading(list(cx.coords[v]), list(dirs[p])) for v in range(cx.nv)]
        assert got[p].tolist() == brute_wecf(cx.nv, faces, weights, f, T, beta)


@pytest.mark.parametrize("dims", [[5], [4, 3], [3, 2, 3], [2, 2, 2]])
def test_brute_force_cubical(oracle, dims):
    rng = np.random.default_rng(sum(dims))
    n = len(dims)
    nv = int(np.prod(dims))
    vw = rng.integers(-5, 30, nv).astype(np.int64)
    dirs = S.random_directions(4, n, seed=7 * n)
    T, lo, hi = 11, -math.sqrt(n), math.sqrt(n)
    got = oracle.wect_cubical(dims, vw, dirs, T, lo, hi)
    X = oracle.grid_coords(dims)
    cells = cubical_cells(dims)
    weights = [max(int(vw[v]) for v in c) for c in cells]
    step = (hi - lo) / (T - 1)
    beta = [lo + q * step for q in range(T)]
    for p in range(len(dirs)):
        f = [height_reading(list(X[v]), list(dirs[p])) for v in range(nv)]
        assert got[p].tolist() == brute_wecf(nv, cells, weights, f, T, beta, cubical=True)


def test_cubical_1d_equals_path_complex(oracle):
    """A 1D grid is the path graph: cubical and simplicial oracles agree."""
    L = 23
    rng = np.random.default_rng(21)
    vw = rng.integers(0, 256, L).astype(np.int64)
    X = oracle.grid_coords([L])
    E = np.stack([np.arange(L - 1), np.arange(1, L)], 1).astype(np.int32)
    dirs = np.array([[1.0], [-1.0], [0.3]])
    a = oracle.wect_cubical([L], vw, dirs, 13, -1.0, 1.0)
    b = oracle.wect_simplicial(X, [E], oracle.simplicial_weights([E], vw), dirs, 13, -1.0, 1.0)
    assert np.array_equal(a, b)


# ----------------------------------------------------------------------- invariances


def test_invariance_under_permutations(oracle):
    cx = S.random_simplicial(40, 2, 60, 30, seed=22)
    vw = cx.weights.astype(np.int64)
    dirs = S.circle_directions(8)
    T = 20
    ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, -1.5, 1.5)
    rng = np.random.default_rng(23)
    perm = rng.permutation(cx.nv)          # new id of old vertex v is inv[v]
    inv = np.argsort(perm)
    X2 = cx.coords[perm]
    vw2 = vw[perm]
    lists2 = []
    for lst in cx.simplices:
        l2 = inv[lst].astype(np.int32)
        l2 = l2[rng.permutation(len(l2))]                         # permute simplices
        l2 = np.array([r[rng.permutation(len(r))] for r in l2], dtype=np.int32)  # permute rows
        lists2.append(l2)
    got = oracle.wect_simplicial(X2, lists2, oracle.simplicial_weights(lists2, vw2), dirs, T, -1.5, 1.5)
    assert np.array_equal(got, ref)


def test_linearity_and_scaling(oracle):
    cx = S.random_simplicial(30, 2, 40, 20, seed=24)
    dirs = S.circle_directions(6)
    T = 15
    rng = np.random.default_rng(25)
    w1 = [rng.integers(-100, 100, cx.nv)] + [rng.integers(-100, 100, len(s)) for s in cx.simplices]
    w2 = [rng.integers(-100, 100, cx.nv)] + [rng.integers(-100, 100, len(s)) for s in cx.simplices]
    f = lambda w: oracle.wect_simplicial(cx.coords, cx.simplices, [np.asarray(a, dtype=np.int64) for a in w], dirs, T, -1.5, 1.5)
    assert np.array_equal(f([a + b for a, b in zip(w1, w2)]), f(w1) + f(w2))
    ones = oracle.simplicial_weights(cx.simplices, np.ones(cx.nv, dtype=np.int64), "one")
    assert np.array_equal(f([7 * a for a in ones]), 7 * f(ones))


def test_default_range_is_max_abs_height(oracle):
    cx = S.random_simplicial(20, 2, 10, 5, seed=26, coord_bits=4)
    dirs = np.array([[1.0, 0.0], [0.5, -0.5], [0.0, 1.0]])
    lo, hi = oracle.default_range_simplicial(cx.coords, dirs)
    M = max(abs(sum(Fraction(cx.coords[v, a]) * Fraction(dirs[p, a]) for a in range(2))) for v in range(cx.nv) for p in range(3))
    assert hi == float(M) and lo == -hi


def _grid_axis_coords(L):
    """Exact rational grid coordinates (2i - (L-1)) / (L-1) of one axis (0 when L = 1)."""
    return [Fraction(0) if L == 1 else Fraction(2 * i - (L - 1), L - 1) for i in range(L)]


@pytest.mark.parametrize("dims", [[9], [5, 17], [9, 3, 5]])
def test_grid_default_range_exact_dyadic(oracle, dims):
    """Default range [-M, M] of a grid (Section 3, the definition of M) against the exact rational
    max of |x(v) . s| over every vertex and direction.  L - 1 is a power of two and the direction
    components are dyadic, so every height is exact.  The data put the largest |h| in the last
    direction, with the last axis contributing: a skipped axis or a direction left out would each
    change M (the grid is symmetric about 0, so max h = -min h)."""
    n = len(dims)
    base = [[0.5, -0.25, 0.125], [-0.25, 0.5, 0.25], [-0.75, -0.5, -1.0]]
    if n == 1:
        base = [[0.5], [0.25], [-0.75]]
    dirs = np.array([row[:n] for row in base], dtype=np.float64)
    axes = [_grid_axis_coords(L) for L in dims]
    M = Fraction(0)
    for idx in itertools.product(*[range(L) for L in dims]):
        for s in dirs:
            M = max(M, abs(sum(axes[a][idx[a]] * Fraction(s[a]) for a in range(n))))
    lo, hi = oracle.default_range_grid(dims, dirs)
    assert hi == float(M) and lo == -hi
    # the same M once the last direction or the last axis is dropped is smaller
    assert oracle.default_range_grid(dims, dirs[:2])[1] < hi
    if n > 1:
        assert oracle.default_range_grid(dims[:-1], np.ascontiguousarray(dirs[:, :-1]))[1] < hi


@pytest.mark.parametrize("dims", [[7], [6, 11], [7, 6, 11]])
def test_grid_default_range_with_rounding(oracle, dims):
    """Non-dyadic grid coordinates and Fibonacci directions: M equals the max of |h| over every
    vertex, with h from the independent restatement of the height rounding rule (exact rational
    coordinates rounded once, then the fma chain)."""
    n = len(dims)
    dirs = S.fibonacci_directions(9)[:, :n] if n == 3 else S.random_directions(9, n, seed=41)
    axes = [[rn(c) for c in _grid_axis_coords(L)] for L in dims]
    M = 0.0
    for idx in itertools.product(*[range(L) for L in dims]):
        x = [axes[a][idx[a]] for a in range(n)]
        for s in dirs:
            M = max(M, abs(height_reading(x, list(s))))
    lo, hi = oracle.default_range_grid(dims, np.ascontiguousarray(dirs))
    assert hi == M and lo == -M


# ----------------------------------------------------------------------- four dimensions


def test_four_sphere_and_four_box_closed_forms(oracle):
    """R^4: the boundary of the 5-simplex (all 4-faces of 6 points in general position, and their
    faces) is a 4-sphere, Euler characteristic 1 - 1 + 1 - 1 + 1 ... = 2; the Freudenthal
    triangulation of a 3 x 2 x 2 x 2 grid is a triangulated box, Euler characteristic 1.  Both at
    the top threshold, in every direction."""
    rng = np.random.default_rng(61)
    pts = rng.uniform(-1, 1, (6, 4))
    from itertools import combinations

    top = np.array(list(combinations(range(6), 5)), dtype=np.int64)
    sphere = S.closure_from_top(pts, top)
    assert [len(s) for s in sphere.simplices] == [15, 20, 15, 6]
    dirs = S.random_directions(7, 4, seed=62)
    one = oracle.simplicial_weights(sphere.simplices, np.ones(6, dtype=np.int64), "one")
    assert np.all(oracle.wect_simplicial(pts, sphere.simplices, one, dirs, 9)[:, -1] == 2)
    dims = [3, 2, 2, 2]
    lists = S.freudenthal_lists(dims)
    assert len(lists) == 4 and lists[3].shape == (2 * 24, 5)
    X = oracle.grid_coords(dims)
    one = oracle.simplicial_weights(lists, np.ones(X.shape[0], dtype=np.int64), "one")
    assert np.all(oracle.wect_simplicial(X, lists, one, dirs, 9)[:, -1] == 1)


@pytest.mark.parametrize("dyadic", [True, False])
def test_brute_force_four_dimensional(oracle, dyadic):
    """A jittered 2^4 Freudenthal grid in R^4 (24 four-simplices and their faces), u8 weights:
    the oracle equals brute-force enumeration of the sublevel subcomplexes, in exact rational
    arithmetic for dyadic coordinates and directions, else with float64 heights from the
    independent restatement of the rounding rule."""
    dims = [2, 2, 2, 2]
    rng = np.random.default_rng(63 + dyadic)
    lists = S.freudenthal_lists(dims)
    base = oracle.grid_coords(dims)
    if dyadic:
        X = base + rng.integers(-2, 3, base.shape).astype(np.float64) / 16.0
        dirs = rng.integers(-8, 9, size=(5, 4)).astype(np.float64) / 8.0
    else:
        X = base + rng.uniform(-0.2, 0.2, base.shape)
        dirs = S.random_directions(5, 4, seed=64)
    nv = X.shape[0]
    vw = rng.integers(0, 256, nv).astype(np.int64)
    cx = S.Simplicial(coords=np.ascontiguousarray(X), simplices=lists, weights=vw.astype(np.uint8))
    T, lo, hi = 17, -2.0, 2.0                     # step 1/4: the float64 thresholds are exact too
    got = oracle.wect_simplicial(X, lists, oracle.simplicial_weights(lists, vw), dirs, T, lo, hi)
    faces, weights = simplicial_faces(cx, vw)
    if dyadic:
        beta = [Fraction(lo) + q * (Fraction(hi) - Fraction(lo)) / (T - 1) for q in range(T)]
    else:
        step = (hi - lo) / (T - 1)
        beta = [lo + q * step for q in range(T)]
    for p in range(len(dirs)):
        if dyadic:
            f = [sum(Fraction(X[v, a]) * Fraction(dirs[p, a]) for a in range(4)) for v in range(nv)]
        else:
            f = [height_reading(list(X[v]), list(dirs[p])) for v in range(nv)]
        assert got[p].tolist() == brute_wecf(nv, faces, weights, f, T, beta)


# ----------------------------------------------------------------------- arbitrary filters (Algorithm 1, m filters)


def test_wecf_simplicial_arbitrary_filters_brute_force(oracle):
    """Algorithm 1 with m caller filters that are not heights (dyadic values, many of them
    exactly on thresholds, repeated values, values outside the range): the oracle's WECF table
    equals brute-force enumeration of every sublevel subcomplex with rational thresholds."""
    for seed in range(4):
        cx = S.random_simplicial(11, 2 + seed % 2, 16, 7, seed=300 + seed, coord_bits=3)
        rng = np.random.default_rng(400 + seed)
        m, T, lo, hi = 5, 17, -2.0, 2.0
        f = rng.integers(-20, 21, size=(m, cx.nv)).astype(np.float64) / 8.0      # also beyond [lo, hi]
        vw = cx.weights.astype(np.int64)
        got = oracle.wecf_simplicial(f, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), T, lo, hi)
        faces, weights = simplicial_faces(cx, vw)
        beta = [Fraction(lo) + q * (Fraction(hi) - Fraction(lo)) / (T - 1) for q in range(T)]
        for p in range(m):
            fr = [Fraction(x) for x in f[p]]
            assert got[p].tolist() == brute_wecf(cx.nv, faces, weights, fr, T, beta)


@pytest.mark.parametrize("weighted", [True, False])
def test_wecf_cubical_arbitrary_filters_brute_force(oracle, weighted):
    """The grid WECF (and unweighted ECF) of caller filters against brute force over every box
    of the grid; the cell weight is the max of its vertex weights, or 1 unweighted."""
    for dims in ([5, 4], [3, 3, 2]):
        rng = np.random.default_rng(500 + len(dims))
        nv = int(np.prod(dims))
        vw = rng.integers(-3, 12, nv).astype(np.int64)
        m, T, lo, hi = 4, 9, -1.0, 1.0
        f = rng.integers(-10, 11, size=(m, nv)).astype(np.float64) / 8.0
        got = oracle.wecf_cubical(dims, vw, f, T, lo, hi, weighted=weighted)
        cells = cubical_cells(dims)
        weights = [max(int(vw[v]) for v in c) if weighted else 1 for c in cells]
        beta = [Fraction(lo) + q * (Fraction(hi) - Fraction(lo)) / (T - 1) for q in range(T)]
        for p in range(m):
            fr = [Fraction(x) for x in f[p]]
            assert got[p].tolist() == brute_wecf(nv, cells, weights, fr, T, beta, cubical=True)


def test_wecf_of_height_filters_is_the_wect(oracle):
    """Algorithm 1 fed the oracle's own float64 heights as filters gives the WECT table."""
    cx = S.random_simplicial(40, 3, 90, 60, seed=601)
    dirs = S.random_directions(6, 3, seed=602)
    vw = cx.weights.astype(np.int64)
    sw = oracle.simplicial_weights(cx.simplices, vw)
    T, lo, hi = 23, -1.7, 1.9
    f = np.array([[oracle.height(cx.coords[v], dirs[p]) for v in range(cx.nv)] for p in range(len(dirs))])
    assert np.array_equal(oracle.wecf_simplicial(f, cx.simplices, sw, T, lo, hi),
                          oracle.wect_simplicial(cx.coords, cx.simplices, sw, dirs, T, lo, hi))
