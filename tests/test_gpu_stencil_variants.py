"""The stencil kernels of full cubical grids give identical integers: the per-vertex kernel with
and without TMA staging of the neighbouring rows, and the run-based kernel (bin boundaries along
the rows, prefix-sum differences), each forced through the wect_debug_stencil_variant hook,
against the oracle."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import SQ2, SQ3, cuda, dev, lib, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    dev()
    L = lib()
    yield L
    L.stencil_variant(0)


def _w(dims, kind, rng):
    shape = tuple(reversed(dims))
    if kind == "u8":
        return rng.integers(0, 256, shape, dtype=np.uint8), 0
    if kind == "i64":                        # narrow fixed-point weights: one histogram plane
        return rng.integers(-2000, 2000, shape).astype(np.int64), 0
    return None, 0


def _dirs(n, d, seed):
    rng = np.random.default_rng(seed)
    if n == 1:
        return np.array([[1.0], [-1.0], [0.5], [-0.25], [0.0], [-0.0], [3.0]] * (d // 7 + 1))[:d]
    D = S.random_directions(d, n, seed) if seed % 2 else (S.circle_directions(d) if n == 2 else S.fibonacci_directions(d))
    D = D.copy()
    D[0] = 0.0
    D[0, -1] = 1.0                                   # s_0 = 0: one run per row
    D[1] = 0.0
    D[1, 0] = -1.0                                   # axis direction: heights on thresholds
    if d > 3:
        D[2] = -D[2]
        D[3, 0] = -0.0
    return D


CASES = [
    # dims (axis 0 first), d, T, lo, hi, weights
    ([700], 14, 40, -1.0, 1.0, "u8"),
    ([64, 64], 32, 64, -SQ2, SQ2, "u8"),
    ([257, 9], 70, 33, -SQ2, SQ2, "one"),
    ([129, 7], 65, 2, -SQ2, SQ2, "u8"),
    ([31, 17, 9], 100, 128, -SQ3, SQ3, "u8"),
    ([128, 12, 11], 256, 128, -SQ3, SQ3, "u8"),
    ([40, 13, 10], 33, 17, -SQ3, SQ3, "i64"),
    ([90, 8, 7], 64, 300, -0.4, 0.3, "u8"),          # narrow range: heights outside [lo, hi]
    ([60, 11], 40, 50, 0.2, 0.2, "u8"),              # degenerate range lo == hi
    ([77, 9, 5], 48, 64, math.nan, math.nan, "u8"),  # default range
    ([1, 5, 6], 10, 20, -SQ3, SQ3, "u8"),            # rows of one vertex
    ([2, 3, 40], 16, 9, -SQ3, SQ3, "u8"),
    ([200, 30], 24, 1000, -SQ2, SQ2, "u8"),          # many thresholds per row (empty runs)
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_both_stencil_kernels_match_oracle(P, oracle, case):
    dims, d, T, lo, hi, kind = CASES[case]
    rng = np.random.default_rng(case + 500)
    w, fb = _w(dims, kind, rng)
    n = len(dims)
    dirs = _dirs(n, d, case)
    vw = np.zeros(int(np.prod(dims)), dtype=np.int64) if w is None else w.ravel().astype(np.int64)
    ref = oracle.wect_cubical(dims, vw, dirs, T, lo, hi, weighted=w is not None)
    for variant in (1, 2, 3, 0):
        P.stencil_variant(variant)
        cx = P.CubicalComplex(None if w is None else cuda(w), frac_bits=fb, dims=dims)
        got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
        cx.device_status()
        assert np.array_equal(got, ref), variant
    P.stencil_variant(0)


def test_tma_staging_on_volumes(P, oracle):
    """Grids with rows of 64 and 128 vertices (TMA staging applies) with u8, f32 and i64 weights,
    with and without the staging, and a batch of volumes whose tensor maps are per grid."""
    rng = np.random.default_rng(77)
    dirs = S.fibonacci_directions(96)
    for dims, kind in (([64, 20, 9], "u8"), ([128, 3, 5], "f32"), ([32, 7, 12], "i64"), ([48, 40], "u8")):
        shape = tuple(reversed(dims))
        if kind == "u8":
            w, fb = rng.integers(0, 256, shape, dtype=np.uint8), 0
        elif kind == "f32":
            w, fb = rng.random(shape, dtype=np.float32), 24
        else:
            w, fb = rng.integers(-(1 << 20), 1 << 20, shape).astype(np.int64), 0
        n = len(dims)
        D = dirs if n == 3 else S.circle_directions(96)
        lo, hi = -math.sqrt(n), math.sqrt(n)
        ref = oracle.wect_cubical(dims, oracle.to_fixed(w, fb), D, 77, lo, hi)
        for variant in (3, 1):
            P.stencil_variant(variant)
            cx = P.CubicalComplex(cuda(w), frac_bits=fb)
            got = cx.wect(cuda(D), 77, lo, hi).cpu().numpy()
            cx.device_status()
            assert np.array_equal(got, ref), (dims, variant)
    P.stencil_variant(0)
    vols = S.uniform_f32_grids(6, [16, 12, 10], seed=78)
    b = P.CubicalBatch([cuda(x) for x in vols], frac_bits=24)
    got = b.wect(cuda(dirs), 40, -SQ3, SQ3).cpu().numpy()
    for i in range(6):
        ref = oracle.wect_cubical([16, 12, 10], oracle.to_fixed(vols[i], 24), dirs, 40, -SQ3, SQ3)
        assert np.array_equal(got[i], ref), i


def test_run_kernel_voxel_field_sampled(P, oracle):
    """A smoothed 96^3 u8 field (the voxel workload's recipe, smaller) with 256 Fibonacci
    directions: both kernels equal on every direction, the oracle on a sample."""
    g = S.smooth_u8_grid([96, 96, 96], seed=9)
    dirs = S.fibonacci_directions(256)
    outs = []
    for variant in (1, 2):
        P.stencil_variant(variant)
        cx = P.CubicalComplex(cuda(g))
        outs.append(cx.wect(cuda(dirs), 128, -SQ3, SQ3).cpu().numpy())
    P.stencil_variant(0)
    assert np.array_equal(outs[0], outs[1])
    sample = [0, 1, 100, 201, 255]
    ref = oracle.wect_cubical([96, 96, 96], g.ravel(), dirs[sample], 128, -SQ3, SQ3)
    assert np.array_equal(outs[1][sample], ref)


def test_run_kernel_in_batches(P, oracle):
    """Batches of images: the graph-captured launch, the per-image loop and the autotuner with
    the run-based kernel forced, against the oracle."""
    imgs = S.blob_images(30, seed=31, side_lo=3, side_hi=120)
    dirs = S.circle_directions(64)
    T = 64
    P.stencil_variant(2)
    b = P.CubicalBatch([cuda(x) for x in imgs])
    got = b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()
    loop = b.wect(cuda(dirs), T, -SQ2, SQ2, loop=True).cpu().numpy()
    P.stencil_variant(0)
    assert np.array_equal(got, loop)
    for i, x in enumerate(imgs):
        ref = oracle.wect_cubical(list(reversed(x.shape)), x.ravel(), dirs, T, -SQ2, SQ2)
        assert np.array_equal(got[i], ref), i
    b.autotune(cuda(dirs), T, -SQ2, SQ2)
    assert np.array_equal(b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy(), got)
