"""Seeded synthetic inputs for the weighted Euler characteristic transform (WECT).

This module only draws random numbers and lays out complexes; it holds none of the
method's arithmetic (no heights, no thresholds, no binning, no Euler sums).  Both the
CPU oracle tests and the CUDA path take their inputs from here.

Conventions shared by every generator:

* A cubical grid with axis lengths ``dims = [L0, L1, ...]`` stores its vertex values in
  a C-contiguous numpy array of shape ``(..., L1, L0)``: axis 0 is the fastest axis and
  the flat vertex index is ``i0 + L0 * (i1 + L1 * i2)``.
* A simplicial complex is ``(coords[nv, n] float64, [edges[k1, 2] int32,
  triangles[k2, 3] int32, ...], vertex_weights[nv])``.
* Direction sets are returned as float64 arrays ``[d, n]``; they are input data.

The workloads stand in for the paper's image, voxel and mesh datasets (Fashion-MNIST,
3D cubical complexes, ImageNet samples, Stanford meshes; Section 4), none of which is
used or reproduced here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------- directions


def circle_directions(d: int) -> np.ndarray:
    """d equally spaced unit vectors on S^1: (cos 2*pi*p/d, sin 2*pi*p/d), p = 0 is (1, 0)."""
    p = np.arange(d, dtype=np.float64)
    t = 2.0 * math.pi * p / d
    return np.ascontiguousarray(np.stack([np.cos(t), np.sin(t)], axis=1))


def fibonacci_directions(d: int) -> np.ndarray:
    """d Fibonacci-sphere points on S^2 (not renormalised).

    z = 1 - (2p+1)/d, r = sqrt(1 - z^2), phi = p * pi * (3 - sqrt 5), s = (r cos phi, r sin phi, z).
    """
    p = np.arange(d, dtype=np.float64)
    z = 1.0 - (2.0 * p + 1.0) / d
    r = np.sqrt(1.0 - z * z)
    phi = p * math.pi * (3.0 - math.sqrt(5.0))
    return np.ascontiguousarray(np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1))


def random_directions(d: int, n: int, seed: int) -> np.ndarray:
    """d random unit vectors in R^n (Gaussian, normalised in float64)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((d, n))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.ascontiguousarray(v)


# --------------------------------------------------------------------------- grids


def uniform_u8_grid(dims, seed: int) -> np.ndarray:
    """iid uniform integers 0..255 on a grid (shape reversed from dims, axis 0 fastest)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=tuple(reversed(dims)), dtype=np.uint8)


def smooth_u8_grid(dims, seed: int, sigma: float = 4.0) -> np.ndarray:
    """Gaussian random field: N(0,1) white noise, Gaussian blur (reflect), min-max, round to uint8."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(tuple(reversed(dims)))
    f = gaussian_filter(noise, sigma=sigma, mode="reflect")
    f = (f - f.min()) / (f.max() - f.min())
    return np.rint(f * 255.0).astype(np.uint8)


def uniform_f32_grids(count: int, dims, seed: int) -> np.ndarray:
    """count iid U[0,1) float32 volumes, array shape (count, *reversed(dims))."""
    rng = np.random.default_rng(seed)
    return rng.random((count,) + tuple(reversed(dims)), dtype=np.float32)


def blob_images(count: int, seed: int, side_lo: int = 28, side_hi: int = 256):
    """count 2D uint8 images with sides iid U{side_lo..side_hi}, each a sum of K ~ U{1..8}
    Gaussian blobs (centre uniform, sigma ~ U[2, min(H,W)/4] px, amplitude ~ U[0.2, 1]),
    normalised by its max, scaled by 255 and rounded.  Returns a list of (H, W) arrays
    (axis 0 of the complex = image column, the fastest axis)."""
    rng = np.random.default_rng(seed)
    hs = rng.integers(side_lo, side_hi + 1, size=count)
    ws = rng.integers(side_lo, side_hi + 1, size=count)
    out = []
    for k in range(count):
        H, W = int(hs[k]), int(ws[k])
        K = int(rng.integers(1, 9))
        yy = np.arange(H, dtype=np.float64)[:, None]
        xx = np.arange(W, dtype=np.float64)[None, :]
        img = np.zeros((H, W), dtype=np.float64)
        for _ in range(K):
            cy = rng.uniform(0, H - 1)
            cx = rng.uniform(0, W - 1)
            sg = rng.uniform(2.0, max(2.0, min(H, W) / 4.0))
            amp = rng.uniform(0.2, 1.0)
            img += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * sg * sg))
        img /= img.max()
        out.append(np.rint(img * 255.0).astype(np.uint8))
    return out


# --------------------------------------------------------------------------- simplicial


@dataclass
class Simplicial:
    coords: np.ndarray                      # [nv, n] float64
    simplices: list = field(default_factory=list)   # simplices[i-1] = int32 [k_i, i+1]
    weights: np.ndarray | None = None      # [nv] vertex weights (any dtype)

    @property
    def n(self) -> int:
        return int(self.coords.shape[1])

    @property
    def nv(self) -> int:
        return int(self.coords.shape[0])


def jittered_grid_mesh(side: int, seed: int, jitter: float = 0.3) -> Simplicial:
    """side x side jittered grid in [-1,1]^2, each cell cut into two triangles along a random
    diagonal.  Lists are int32 and ordered by their lowest-row/lowest-column vertex (row-major),
    so consecutive simplices touch nearby vertices.  Weights: float32 lognormal(0, 1)."""
    rng = np.random.default_rng(seed)
    L = side
    h = 2.0 / (L - 1)
    i = np.arange(L, dtype=np.float64)
    base = -1.0 + 2.0 * i / (L - 1)
    X, Y = np.meshgrid(base, base, indexing="xy")            # Y rows, X fastest
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    coords = coords + rng.uniform(-jitter * h, jitter * h, size=coords.shape)
    diag = rng.integers(0, 2, size=(L - 1, L - 1))           # per cell: 0 -> (00,11), 1 -> (10,01)
    w = rng.lognormal(0.0, 1.0, size=L * L).astype(np.float32)

    def vid(c, r):
        return r * L + c

    edges = []
    tris = []
    for r in range(L):
        cs = np.arange(L)
        # edges grouped by their lower-left vertex, row-major
        e_rows = []
        right = cs[:-1]
        e_rows.append(np.stack([vid(right, r), vid(right + 1, r)], axis=1))   # horizontal
        if r < L - 1:
            e_rows.append(np.stack([vid(cs, r), vid(cs, r + 1)], axis=1))     # vertical
            d = diag[r]
            c0 = cs[:-1]
            a = np.where(d == 0, vid(c0, r), vid(c0 + 1, r))
            b = np.where(d == 0, vid(c0 + 1, r + 1), vid(c0, r + 1))
            e_rows.append(np.stack([a, b], axis=1))                           # diagonal
            v00, v10, v01, v11 = vid(c0, r), vid(c0 + 1, r), vid(c0, r + 1), vid(c0 + 1, r + 1)
            t1 = np.where(d[:, None] == 0, np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
            t2 = np.where(d[:, None] == 0, np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
            tris.append(np.stack([t1, t2], axis=1).reshape(-1, 3))
        edges.append(np.concatenate(e_rows, axis=0))
    E = np.ascontiguousarray(np.concatenate(edges, axis=0).astype(np.int32))
    F = np.ascontiguousarray(np.concatenate(tris, axis=0).astype(np.int32))
    return Simplicial(coords=np.ascontiguousarray(coords), simplices=[E, F], weights=w)


def torus_mesh(nu: int, nv_: int, R: float = 2.0, r: float = 0.75) -> Simplicial:
    """Triangulated torus in R^3 (nu x nv_ quad grid with wrap-around, each quad cut in two)."""
    verts = []
    for a in range(nu):
        for b in range(nv_):
            u = 2 * math.pi * a / nu
            v = 2 * math.pi * b / nv_
            verts.append(((R + r * math.cos(v)) * math.cos(u), (R + r * math.cos(v)) * math.sin(u), r * math.sin(v)))
    idx = lambda a, b: (a % nu) * nv_ + (b % nv_)
    tris = []
    for a in range(nu):
        for b in range(nv_):
            tris.append((idx(a, b), idx(a + 1, b), idx(a + 1, b + 1)))
            tris.append((idx(a, b), idx(a + 1, b + 1), idx(a, b + 1)))
    return closure_from_top(np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int64))


def octahedron_surface() -> Simplicial:
    """Boundary of the octahedron (a 2-sphere): 6 vertices, 12 edges, 8 triangles."""
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    tris = []
    for x in (0, 1):
        for y in (2, 3):
            for z in (4, 5):
                tris.append((x, y, z))
    return closure_from_top(V, np.array(tris, dtype=np.int64))


def closure_from_top(coords: np.ndarray, top: np.ndarray) -> Simplicial:
    """All faces of the given top simplices (rows of vertex ids), as sorted int32 lists."""
    k = top.shape[1]
    faces = [set() for _ in range(k - 1)]        # faces[i-1]: i-simplices
    from itertools import combinations

    for row in top:
        row = tuple(sorted(int(x) for x in row))
        for i in range(1, k):
            for f in combinations(row, i + 1):
                faces[i - 1].add(f)
    lists = [np.ascontiguousarray(np.array(sorted(f), dtype=np.int32).reshape(-1, i + 2)) for i, f in enumerate(faces)]
    return Simplicial(coords=np.ascontiguousarray(coords), simplices=lists, weights=np.ones(coords.shape[0], dtype=np.uint8))


def freudenthal_lists(dims) -> list:
    """Index lists of the Freudenthal (Kuhn) triangulation of a full grid (axis 0 fastest): the
    k-simplices are {v + c_0, ..., v + c_k} for chains 0 = c_0 < ... < c_k of nested axis masks,
    wherever v + c_k is in the grid.  Lists [edges, triangles, ...] as int32 arrays."""
    n = len(dims)
    strides = [1] * n
    for a in range(1, n):
        strides[a] = strides[a - 1] * dims[a - 1]

    def chains(last, cur, out):
        if len(cur) > 1:
            out.setdefault(len(cur) - 1, []).append(list(cur))
        for nxt in range(1, 1 << n):
            if (nxt & last) == last and nxt != last:
                chains(nxt, cur + [nxt], out)

    by_dim = {}
    chains(0, [0], by_dim)
    lists = []
    for k in range(1, n + 1):
        rows = []
        for ch in by_dim.get(k, []):
            ext = [(ch[-1] >> a) & 1 for a in range(n)]
            ranges = [range(dims[a] - ext[a]) for a in range(n)]
            offs = [sum(strides[a] for a in range(n) if (c >> a) & 1) for c in ch]
            for idx in np.ndindex(*[len(r) for r in reversed(ranges)]):
                v = sum(i * strides[n - 1 - j] for j, i in enumerate(idx))
                rows.append([v + o for o in offs])
        lists.append(np.array(rows, dtype=np.int32).reshape(-1, k + 1))
    return lists


def freudenthal_mesh(dims, seed: int, jitter: float = 0.2) -> Simplicial:
    """The Freudenthal triangulation of a jittered full grid in R^n (any n): grid points at
    -1 + 2 i / (L - 1) per axis, each moved by U(+-jitter cell), with all simplices of
    freudenthal_lists(dims); u8 weights ~ U{0..255}."""
    rng = np.random.default_rng(seed)
    n = len(dims)
    axes = [(-1.0 + 2.0 * np.arange(L, dtype=np.float64) / (L - 1)) if L > 1 else np.zeros(1) for L in dims]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    X = np.stack([m.ravel() for m in reversed(mesh)], axis=1)
    cell = np.array([2.0 / (L - 1) if L > 1 else 0.0 for L in dims])
    X = X + rng.uniform(-jitter, jitter, X.shape) * cell
    w = rng.integers(0, 256, size=X.shape[0], dtype=np.uint8)
    return Simplicial(coords=np.ascontiguousarray(X), simplices=freudenthal_lists(dims), weights=w)


def tetra_grid(side: int, seed: int, jitter: float = 0.2) -> Simplicial:
    """Solid side^3 jittered grid in [-1,1]^3 cut into tetrahedra (six per cube cell, one per
    ordering of the axes: the path lower corner -> +e_a -> +e_a+e_b -> upper corner), with all
    their faces.  A triangulated solid cube: Euler characteristic 1.  u8 weights."""
    rng = np.random.default_rng(seed)
    L = side
    h = 2.0 / (L - 1)
    g = -1.0 + 2.0 * np.arange(L, dtype=np.float64) / (L - 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    coords = coords + rng.uniform(-jitter * h, jitter * h, size=coords.shape)
    from itertools import permutations

    def vid(x, y, z):
        return (z * L + y) * L + x

    tets = []
    for z in range(L - 1):
        for y in range(L - 1):
            for x in range(L - 1):
                for perm in permutations(range(3)):
                    p = [x, y, z]
                    path = [vid(*p)]
                    for a in perm:
                        p[a] += 1
                        path.append(vid(*p))
                    tets.append(path)
    cx = closure_from_top(coords, np.array(tets, dtype=np.int64))
    cx.weights = rng.integers(0, 256, size=coords.shape[0], dtype=np.uint8)
    return cx


def random_simplicial(nv: int, n: int, k1: int, k2: int, seed: int, coord_bits: int | None = None) -> Simplicial:
    """Random (not necessarily closed) complex: nv random points, k1 random edges, k2 random
    triangles, u8 weights.  With coord_bits, coordinates are multiples of 2^-coord_bits in
    [-1, 1] so that products and sums with short dyadic directions are exact in float64."""
    rng = np.random.default_rng(seed)
    if coord_bits is None:
        X = rng.uniform(-1, 1, size=(nv, n))
    else:
        s = 1 << coord_bits
        X = rng.integers(-s, s + 1, size=(nv, n)).astype(np.float64) / s
    E = np.array([rng.choice(nv, 2, replace=False) for _ in range(k1)], dtype=np.int32).reshape(-1, 2)
    F = np.array([rng.choice(nv, 3, replace=False) for _ in range(k2)], dtype=np.int32).reshape(-1, 3)
    w = rng.integers(0, 256, size=nv, dtype=np.uint8)
    return Simplicial(coords=np.ascontiguousarray(X), simplices=[E, F], weights=w)


# --------------------------------------------------------------------------- workloads


@dataclass
class Workload:
    """One named workload: its inputs plus the parameters of the transform."""
    name: str
    kind: str                  # "cubical", "simplicial", "batch", "diff"
    dirs: np.ndarray
    T: int
    lo: float
    hi: float
    dims: list | None = None
    grid: np.ndarray | None = None          # cubical vertex weights
    grids: list | None = None               # batch / diff vertex weights
    target: np.ndarray | None = None        # diff: second seeded batch
    complex: Simplicial | None = None
    frac_bits: int = 0
    extra: dict = field(default_factory=dict)


SQRT2 = math.sqrt(2.0)
SQRT3 = math.sqrt(3.0)


def grid2d_64(side: int = 64, d: int = 32, T: int = 64) -> Workload:
    """2D cubical complex of a 64x64 image, u8 weights ~ U{0..255} (seed 1), d directions on S^1,
    T thresholds over [-sqrt2, sqrt2]."""
    g = uniform_u8_grid([side, side], seed=1)
    return Workload("grid2d_64x64_d32_T64", "cubical", circle_directions(d), T, -SQRT2, SQRT2,
                    dims=[side, side], grid=g)


def voxel3d_128(side: int = 128, d: int = 256, T: int = 128) -> Workload:
    """3D cubical complex of a 128^3 smoothed Gaussian random field quantised to u8 (seed 2),
    d Fibonacci directions, T thresholds over [-sqrt3, sqrt3]."""
    g = smooth_u8_grid([side, side, side], seed=2)
    return Workload(f"voxel3d_{side}^3_d{d}_T{T}", "cubical", fibonacci_directions(d), T, -SQRT3, SQRT3,
                    dims=[side, side, side], grid=g)


def mesh2d_1024(side: int = 1024, d: int = 1024, T: int = 512) -> Workload:
    """2D simplicial complex: side^2 jittered grid cut into triangles (seed 3), f32 lognormal
    weights at 2^-24 fixed point, d directions on S^1, T thresholds over the default range."""
    cx = jittered_grid_mesh(side, seed=3)
    return Workload(f"mesh2d_{side}^2_d{d}_T{T}", "simplicial", circle_directions(d), T, math.nan, math.nan,
                    complex=cx, frac_bits=24)


def image_batch(count: int = 4096, d: int = 64, T: int = 64, side_lo: int = 28, side_hi: int = 256) -> Workload:
    """count 2D u8 blob images of independent random sides (seed 4), d directions, T over [-sqrt2, sqrt2]."""
    imgs = blob_images(count, seed=4, side_lo=side_lo, side_hi=side_hi)
    return Workload(f"images2d_{count}x[{side_lo}..{side_hi}]^2_d{d}_T{T}", "batch", circle_directions(d), T,
                    -SQRT2, SQRT2, grids=imgs)


def volume_batch_diff(count: int = 256, side: int = 64, d: int = 128, T: int = 128) -> Workload:
    """count 3D f32 U[0,1) volumes (seed 5) and a target batch (seed 6), d Fibonacci directions,
    T over [-sqrt3, sqrt3], 2^-24 fixed-point weights."""
    a = uniform_f32_grids(count, [side] * 3, seed=5)
    b = uniform_f32_grids(count, [side] * 3, seed=6)
    return Workload(f"volumes3d_{count}x{side}^3_d{d}_T{T}", "diff", fibonacci_directions(d), T, -SQRT3, SQRT3,
                    dims=[side] * 3, grids=a, target=b, frac_bits=24)
