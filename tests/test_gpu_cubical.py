"""GPU parity of the cubical (stencil) path: the CUDA library through the C ABI against the
CPU oracle, element by element (all results are exact integers)."""
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import SQ2, SQ3, cuda, dev, grid_dims, lib, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


@pytest.fixture(scope="module")
def O(oracle):
    return oracle


CASES = [
    # dims (axis 0 first), d, T, lo, hi, weight kind
    ([37], 5, 7, -1.0, 1.0, "u8"),
    ([64, 64], 32, 64, -SQ2, SQ2, "u8"),
    ([129, 7], 70, 33, -SQ2, SQ2, "u8"),
    ([5, 131], 65, 2, -SQ2, SQ2, "u8"),
    ([31, 17, 9], 100, 128, -SQ3, SQ3, "u8"),
    ([16, 16, 16], 256, 128, -SQ3, SQ3, "u8"),
    ([23, 11, 13], 40, 50, -SQ3, SQ3, "f32"),
    ([12, 9, 10], 33, 17, -SQ3, SQ3, "i64"),
    ([19, 21], 17, 40, -SQ2, SQ2, "one"),
    ([9, 8, 7], 64, 9, -0.4, 0.3, "u8"),        # narrow range: many heights outside [lo, hi]
    ([2, 1, 3], 8, 5, -SQ3, SQ3, "u8"),          # axes of length 1 and 2
]


def _weights(dims, kind, seed):
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(dims))
    if kind == "u8":
        return rng.integers(0, 256, shape, dtype=np.uint8), 0
    if kind == "f32":
        return rng.random(shape, dtype=np.float32), 24
    if kind == "i64":
        return rng.integers(-(1 << 20), 1 << 20, shape).astype(np.int64), 0
    return None, 0


def _dirs(n, d, seed):
    if n == 1:
        return np.array([[1.0], [-1.0], [0.5], [-0.25], [0.0]] * (d // 5 + 1))[:d]
    if n == 2:
        return S.circle_directions(d) if seed % 2 == 0 else S.random_directions(d, 2, seed)
    return S.fibonacci_directions(d) if seed % 2 == 0 else S.random_directions(d, 3, seed)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_cubical_wect_matches_oracle(P, O, case):
    dims, d, T, lo, hi, kind = CASES[case]
    w, fb = _weights(dims, kind, seed=case)
    dirs = _dirs(len(dims), d, case)
    if w is None:
        cx = P.CubicalComplex(None, dims=dims)
        vw = np.zeros(int(np.prod(dims)), dtype=np.int64)
    else:
        cx = P.CubicalComplex(cuda(w), frac_bits=fb)
        vw = O.to_fixed(w, fb)
    got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
    ref = O.wect_cubical(dims, vw, dirs, T, lo, hi, weighted=w is not None)
    assert np.array_equal(got, ref)
    cx.device_status()


def test_default_range_and_degenerate_range(P, O):
    w = S.uniform_u8_grid([14, 9, 6], seed=5)
    dirs = S.fibonacci_directions(20)
    cx = P.CubicalComplex(cuda(w))
    got = cx.wect(cuda(dirs), 31).cpu().numpy()          # default [-M, M]
    ref = O.wect_cubical([14, 9, 6], w.ravel(), dirs, 31)
    assert np.array_equal(got, ref)
    got = cx.wect(cuda(dirs), 6, 0.1, 0.1).cpu().numpy()  # lo == hi
    ref = O.wect_cubical([14, 9, 6], w.ravel(), dirs, 6, 0.1, 0.1)
    assert np.array_equal(got, ref)


def test_directions_on_thresholds_and_axes(P, O):
    """Axis-aligned and diagonal directions put many heights exactly on thresholds."""
    dims = [33, 33]
    w = S.uniform_u8_grid(dims, seed=6)
    dirs = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [0.0, -1.0], [math.sqrt(0.5), math.sqrt(0.5)],
                     [-math.sqrt(0.5), math.sqrt(0.5)], [0.5, 0.5], [-0.0, 1.0], [1e-300, -1.0], [2.0, 3.0]])
    for T, lo, hi in [(33, -1.0, 1.0), (65, -2.0, 2.0), (64, -SQ2, SQ2), (17, -5.0, 5.0)]:
        cx = P.CubicalComplex(cuda(w))
        got = cx.wect(cuda(dirs), T, lo, hi).cpu().numpy()
        ref = O.wect_cubical(dims, w.ravel(), dirs, T, lo, hi)
        assert np.array_equal(got, ref), (T, lo, hi)


def test_grid2d_64_full(P, O):
    """64x64 u8 image (seed 1), d=32 on S^1, T=64 over [-sqrt2, sqrt2], and its unweighted
    ECF for the filter x (direction (1,0))."""
    wl = S.grid2d_64()
    cx = P.CubicalComplex(cuda(wl.grid))
    got = cx.wect(cuda(wl.dirs), wl.T, wl.lo, wl.hi).cpu().numpy()
    ref = O.wect_cubical(wl.dims, wl.grid.ravel(), wl.dirs, wl.T, wl.lo, wl.hi)
    assert np.array_equal(got, ref)
    X = O.grid_coords(wl.dims)
    e = cx.ecf(cuda(X[:, 0].copy()), wl.T, wl.lo, wl.hi, weighted=False).cpu().numpy()
    eref = O.wecf_cubical(wl.dims, wl.grid.ravel(), X[:, 0], wl.T, wl.lo, wl.hi, weighted=False)[0]
    assert np.array_equal(e, eref)
    # and it equals the direction (1,0) row of the unweighted transform
    cx1 = P.CubicalComplex(None, dims=wl.dims)
    row = cx1.wect(cuda(np.array([[1.0, 0.0]])), wl.T, wl.lo, wl.hi).cpu().numpy()[0]
    assert np.array_equal(e, row)


@pytest.mark.parametrize("weighted", [False, True])
def test_ecf_of_images(P, O, weighted):
    rng = np.random.default_rng(8)
    for dims in ([40, 23], [11, 12, 13]):
        w = rng.integers(0, 256, tuple(reversed(dims)), dtype=np.uint8)
        f = rng.random(int(np.prod(dims)))
        cx = P.CubicalComplex(cuda(w))
        for T, lo, hi in [(50, 0.0, 1.0), (7, math.nan, math.nan), (100, 0.2, 0.7)]:
            got = cx.ecf(cuda(f), T, lo, hi, weighted=weighted).cpu().numpy()
            ref = O.wecf_cubical(dims, w.ravel(), f, T, lo, hi, weighted=weighted)[0]
            assert np.array_equal(got, ref)


def test_set_weights_and_overflow_status(P, O):
    dims = [10, 9, 8]
    rng = np.random.default_rng(9)
    a = rng.random(tuple(reversed(dims)), dtype=np.float32)
    b = rng.random(tuple(reversed(dims)), dtype=np.float32)
    dirs = S.fibonacci_directions(16)
    cx = P.CubicalComplex(cuda(a), frac_bits=24)
    cx.set_weights(cuda(b))
    got = cx.wect(cuda(dirs), 20, -SQ3, SQ3).cpu().numpy()
    assert np.array_equal(got, O.wect_cubical(dims, O.to_fixed(b, 24), dirs, 20, -SQ3, SQ3))
    cx.device_status()
    cx.set_weights(cuda(b * 1e4))                      # 2^n * max|w| no longer fits the accumulator
    with pytest.raises(P.WectError) as ei:
        cx.device_status()
    assert ei.value.name == "OVERFLOW"


def test_argument_errors(P):
    w = cuda(S.uniform_u8_grid([8, 8], seed=1))
    cx = P.CubicalComplex(w)
    dirs = cuda(S.circle_directions(4))
    for T, lo, hi in [(1, -1.0, 1.0), (8, 1.0, -1.0), (8, math.inf, 1.0), (8, math.nan, 1.0)]:
        with pytest.raises(P.WectError) as ei:
            cx.wect(dirs, T, lo, hi)
        assert ei.value.name == "INVALID_ARG"
    bad = torch.tensor([[float("nan"), 1.0]], dtype=torch.float64, device=dev())
    cx.wect(bad, 8, -1.0, 1.0)
    with pytest.raises(P.WectError) as ei:
        cx.device_status()
    assert ei.value.name == "INVALID_ARG"
    with pytest.raises(P.WectError):
        P.CubicalComplex(cuda(np.array([[np.inf, 1.0]], dtype=np.float32)), frac_bits=8)


def test_output_table_with_8_byte_offset(P, O):
    """An int64 output table that is 8- but not 16-byte aligned (a slice) is cleared and filled
    exactly like an aligned one."""
    dims = [21, 17, 5]
    w = S.uniform_u8_grid(dims, seed=9)
    dirs = S.fibonacci_directions(33)
    cx = P.CubicalComplex(cuda(w))
    T = 19
    buf = torch.full((33 * T + 1,), 7, dtype=torch.int64, device="cuda")
    out = buf[1:].view(33, T)
    assert out.data_ptr() % 16 == 8
    got = cx.wect(cuda(dirs), T, -SQ3, SQ3, out=out).cpu().numpy()
    ref = O.wect_cubical(dims, w.ravel(), dirs, T, -SQ3, SQ3)
    assert np.array_equal(got, ref)
    assert int(buf[0]) == 7
