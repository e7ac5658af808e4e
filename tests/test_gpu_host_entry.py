"""wect_compute_host: weights and directions from host memory, the table into host memory.
Page-locked buffers are read and written by the kernels in place, pageable ones are staged; both
give the oracle's table bit for bit, and the same table as set_weights + wect_compute."""
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


def _host(a, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pinned else t.clone()


@pytest.mark.parametrize("pinned", [True, False])
def test_cubical_u8_host_buffers(P, oracle, pinned):
    rng = np.random.default_rng(5)
    dims = [37, 29, 11]
    w0 = rng.integers(0, 256, tuple(reversed(dims))).astype(np.uint8)
    w1 = rng.integers(0, 256, tuple(reversed(dims))).astype(np.uint8)
    dirs = S.fibonacci_directions(70)
    T = 45
    cx = P.CubicalComplex(cuda(w0))
    out = torch.empty((70, T), dtype=torch.int64)
    out = out.pin_memory() if pinned else out
    for w, (lo, hi) in ((w1, (-SQ3, SQ3)), (w0, (math.nan, math.nan)), (w1, (-0.4, 0.7))):
        got = cx.wect_host(_host(w, pinned), _host(dirs, pinned), T, lo, hi, out=out).numpy()
        ref = oracle.wect_cubical(dims, w.ravel().astype(np.int64), dirs, T, lo, hi)
        assert np.array_equal(got, ref), (lo, hi)
        # the device entry on the same weights gives the same table
        assert np.array_equal(cx.wect(cuda(dirs), T, lo, hi).cpu().numpy(), ref)
    cx.device_status()


def test_keep_weights_and_unweighted(P, oracle):
    rng = np.random.default_rng(6)
    w = rng.integers(0, 256, (23, 41)).astype(np.uint8)
    dims = [41, 23]
    dirs = S.circle_directions(40)
    cx = P.CubicalComplex(cuda(w))
    got = cx.wect_host(None, _host(dirs, True), 30, -SQ2, SQ2).numpy()
    assert np.array_equal(got, oracle.wect_cubical(dims, w.ravel().astype(np.int64), dirs, 30, -SQ2, SQ2))
    one = P.CubicalComplex(None, dims=dims)
    got = one.wect_host(None, _host(dirs, False), 30, -SQ2, SQ2).numpy()
    ref = oracle.wect_cubical(dims, np.ones(w.size, np.int64), dirs, 30, -SQ2, SQ2, weighted=False)
    assert np.array_equal(got, ref)


def test_float_weights_host(P, oracle):
    rng = np.random.default_rng(7)
    w = rng.uniform(-2.0, 2.0, (19, 33)).astype(np.float32)
    dims = [33, 19]
    dirs = S.circle_directions(25)
    cx = P.CubicalComplex(cuda(np.zeros_like(w)), frac_bits=18)
    got = cx.wect_host(_host(w, True), _host(dirs, True), 50, -SQ2, SQ2).numpy()
    ref = oracle.wect_cubical(dims, oracle.to_fixed(w, 18), dirs, 50, -SQ2, SQ2)
    assert np.array_equal(got, ref)
    with pytest.raises(ValueError):
        cx.wect_host(_host(w.astype(np.float64), True), _host(dirs, True), 50, -SQ2, SQ2)


@pytest.mark.parametrize("pinned", [True, False])
def test_simplicial_host_buffers(P, oracle, pinned):
    cx = S.random_simplicial(420, 3, 1200, 700, seed=11)
    dirs = S.random_directions(50, 3, 12)
    T = 64
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(np.zeros_like(cx.weights)))
    got = h.wect_host(_host(cx.weights, pinned), _host(dirs, pinned), T, -1.5, 1.5).numpy()
    vw = cx.weights.astype(np.int64)
    ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, T, -1.5, 1.5)
    assert np.array_equal(got, ref)


def test_voxel3d_128_host_equals_device(P):
    """The 128^3 benchmark volume, d = 256, T = 128: the host entry (page-locked buffers, the
    benchmark's end-to-end call) and the device entry give the same table; its last column is the
    Euler characteristic of the weighted complex, the same for every direction."""
    wl = S.voxel3d_128()
    d, T = len(wl.dirs), wl.T
    cx = P.CubicalComplex(cuda(np.zeros_like(wl.grid)))
    got = cx.wect_host(_host(wl.grid, True), _host(wl.dirs, True), T, wl.lo, wl.hi).numpy()
    ref = cx.wect(cuda(wl.dirs), T, wl.lo, wl.hi).cpu().numpy()
    assert got.shape == (d, T) and np.array_equal(got, ref)
    assert np.all(got[:, -1] == got[0, -1])


def test_back_to_back_calls_without_synchronisation(P, oracle):
    """Consecutive set_weights + wect calls (and host-buffer calls) queued on one stream with no
    host synchronisation in between: each call's programmatic launches must see its own weights
    and must not disturb the previous call's table."""
    rng = np.random.default_rng(21)
    dims = [45, 33, 7]
    ws = [rng.integers(0, 256, tuple(reversed(dims))).astype(np.uint8) for _ in range(6)]
    dirs = S.fibonacci_directions(96)
    T, lo, hi = 64, -SQ3, SQ3
    cx = P.CubicalComplex(cuda(ws[0]))
    dd = cuda(dirs)
    outs = [torch.empty((96, T), dtype=torch.int64, device=dd.device) for _ in ws]
    wd = [cuda(w) for w in ws]
    for w, o in zip(wd, outs):
        cx.set_weights(w)
        cx.wect(dd, T, lo, hi, out=o)
    hosts = [torch.empty((96, T), dtype=torch.int64).pin_memory() for _ in ws]
    wh = [_host(w, True) for w in ws]
    dh = _host(dirs, True)
    for w, o in zip(wh, hosts):
        cx.wect_host(w, dh, T, lo, hi, out=o, sync=False)
    torch.cuda.synchronize()
    for w, o, h in zip(ws, outs, hosts):
        ref = oracle.wect_cubical(dims, w.ravel().astype(np.int64), dirs, T, lo, hi)
        assert np.array_equal(o.cpu().numpy(), ref)
        assert np.array_equal(h.numpy(), ref)


def test_simplicial_back_to_back_calls(P, oracle):
    """The gathers' programmatic launches over consecutive calls with new weights."""
    cx = S.random_simplicial(350, 2, 900, 500, seed=23)
    dirs = S.random_directions(70, 2, 24)
    rng = np.random.default_rng(25)
    wlist = [rng.integers(0, 256, cx.nv).astype(np.uint8) for _ in range(4)]
    h = P.SimplicialComplex(cuda(cx.coords), [cuda(s) for s in cx.simplices], cuda(wlist[0]))
    dd = cuda(dirs)
    outs = []
    for w in wlist:
        h.set_weights(cuda(w))
        outs.append(h.wect(dd, 50, -1.5, 1.5))
    torch.cuda.synchronize()
    for w, o in zip(wlist, outs):
        vw = w.astype(np.int64)
        ref = oracle.wect_simplicial(cx.coords, cx.simplices, oracle.simplicial_weights(cx.simplices, vw), dirs, 50,
                                     -1.5, 1.5)
        assert np.array_equal(o.cpu().numpy(), ref)


def test_device_pointers_accepted(P, oracle):
    """The C entry takes device memory too (used in place): device weights, directions and table."""
    import ctypes as C

    rng = np.random.default_rng(31)
    dims = [40, 18]
    w = rng.integers(0, 256, tuple(reversed(dims))).astype(np.uint8)
    dirs = S.circle_directions(36)
    cx = P.CubicalComplex(cuda(np.zeros_like(w)))
    wd, dd = cuda(w), cuda(dirs)
    out = torch.empty((36, 40), dtype=torch.int64, device=dd.device)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert P.load().wect_compute_host(cx.handle, C.c_void_p(wd.data_ptr()), C.c_void_p(dd.data_ptr()), 36, 40,
                                      -SQ2, SQ2, C.c_void_p(out.data_ptr()), st) == 0
    ref = oracle.wect_cubical(dims, w.ravel().astype(np.int64), dirs, 40, -SQ2, SQ2)
    assert np.array_equal(out.cpu().numpy(), ref)
