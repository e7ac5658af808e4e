"""The stencil kernel on TMA-staged grids with the benchmark's tile shape (a 256-wide tile, two
directions per lane: 129-256 directions, rows of a multiple of 4 vertices): one and two
histogram planes, 2-D and 3-D grids, a batch, against the oracle bit for bit."""
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


@pytest.mark.parametrize("dims,d,kind", [
    ([64, 50], 200, "u8"),
    ([64, 37], 256, "f32"),
    ([16, 12, 9], 180, "u8"),
    ([20, 9, 7], 240, "f32"),
])
def test_tma_staged_256_wide_tile(P, oracle, dims, d, kind):
    rng = np.random.default_rng(sum(dims) + d)
    shape = tuple(reversed(dims))
    n = len(dims)
    if kind == "u8":
        w = rng.integers(0, 256, shape).astype(np.uint8)
        fb, vw = 0, w.ravel().astype(np.int64)
    else:
        w = rng.uniform(0.0, 3.0, shape).astype(np.float32)
        fb = 20
        vw = oracle.to_fixed(w, fb)
    dirs = S.circle_directions(d) if n == 2 else S.fibonacci_directions(d)
    lo, hi = (-SQ2, SQ2) if n == 2 else (-SQ3, SQ3)
    cx = P.CubicalComplex(cuda(w), frac_bits=fb)
    for T, (a, b) in ((40, (lo, hi)), (97, (math.nan, math.nan))):
        got = cx.wect(cuda(dirs), T, a, b).cpu().numpy()
        assert P.last_stencil_kernel() == "cubical_fwd_kernel"
        assert np.array_equal(got, oracle.wect_cubical(dims, vw, dirs, T, a, b)), (T, a, b)
    cx.device_status()


def test_tma_staged_256_wide_tile_batch(P, oracle):
    """A batch whose grids all have tensor maps (widths a multiple of 4, 16-byte aligned starts)."""
    rng = np.random.default_rng(41)
    dims_list = [[32, 20], [48, 33], [64, 64], [28, 40]]
    grids = [rng.integers(0, 256, tuple(reversed(dm))).astype(np.uint8) for dm in dims_list]
    dirs = S.circle_directions(160)
    T = 50
    b = P.CubicalBatch([cuda(g) for g in grids])
    out = b.wect(cuda(dirs), T, -SQ2, SQ2).cpu().numpy()
    for i, (dm, g) in enumerate(zip(dims_list, grids)):
        assert np.array_equal(out[i], oracle.wect_cubical(dm, g.ravel().astype(np.int64), dirs, T, -SQ2, SQ2)), i
