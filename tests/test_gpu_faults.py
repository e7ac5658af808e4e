"""Failure handling through the C ABI, with failures injected on the host (no GPU fault):

- every device allocation of a sequence of calls (create, compute, adjoint, batch, builders) is
  made to fail in turn: each failure surfaces as OUT_OF_MEMORY, later calls still give the same
  results, and nothing leaks;
- a batch whose workspace grows between calls never replays a graph captured with the old
  buffers (the same dirs/out pointers come back after a call with larger d and T).
"""
import gc
import math

import numpy as np
import pytest

import synthetic as S
from gpu_common import SQ2, cuda, dev, lib, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    dev()
    return lib()


def _inputs():
    img = S.uniform_u8_grid([37, 29], seed=21)
    imgs = [S.uniform_u8_grid(dd, seed=22 + i) for i, dd in enumerate(([20, 17], [33, 9], [8, 40]))]
    vol = np.random.default_rng(25).random((6, 7, 5), dtype=np.float32)
    sc = S.random_simplicial(90, 2, 200, 100, seed=26)
    return img, imgs, vol, sc


def _sequence(P, inp):
    """One pass over the API's allocating calls; returns every result on the host."""
    img, imgs, vol, sc = inp
    d2 = cuda(S.circle_directions(12))
    d3 = cuda(S.fibonacci_directions(10))
    T = 17
    res = []
    cx = P.CubicalComplex(cuda(img))
    res.append(cx.wect(d2, T, -SQ2, SQ2))
    G = torch.arange(12 * T, dtype=torch.int64, device="cuda").reshape(12, T) - 90
    res.append(cx.backward(d2, T, -SQ2, SQ2, G, 0.25))
    filt = torch.linspace(-1.0, 1.0, cx.nv, dtype=torch.float64, device="cuda")
    res.append(cx.ecf(filt, T, -1.0, 1.0))
    res.append(cx.wecf(torch.stack([filt, -filt]), T, -1.0, 1.0))
    fr = P.FreudenthalComplex(cuda(vol), frac_bits=24)
    res.append(fr.wect(d3, T, -math.sqrt(3.0), math.sqrt(3.0)))
    sx = P.SimplicialComplex(cuda(sc.coords), [cuda(x) for x in sc.simplices], cuda(sc.weights))
    res.append(sx.wect(d2, T))
    bt = P.CubicalBatch([cuda(x) for x in imgs])
    res.append(bt.wect(d2, T, -SQ2, SQ2))
    Gb = torch.ones((3, 12, T), dtype=torch.int64, device="cuda")
    res.append(bt.backward(d2, T, -SQ2, SQ2, Gb, 1.0))
    res.append(bt.backward_f64(d2, T, -SQ2, SQ2, Gb.to(torch.float64) * 0.5))
    torch.cuda.synchronize()
    return [r.cpu() for r in res]


def test_every_allocation_failure_is_reported_and_recovered(P, oracle):
    inp = _inputs()
    P.debug_fail_alloc(-1)
    ref = _sequence(P, inp)
    img = inp[0]
    want = oracle.wect_cubical([37, 29], img.ravel(), S.circle_directions(12), 17, -SQ2, SQ2)
    assert np.array_equal(ref[0].numpy(), want)
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    finished = False
    try:
        for k in range(400):
            P.debug_fail_alloc(k)
            try:
                got = _sequence(P, inp)
            except P.WectError as e:
                assert e.name == "OUT_OF_MEMORY", f"allocation {k}: {e}"
                failures += 1
                continue
            finally:
                gc.collect()
            # the hook did not fire: the whole sequence has fewer than k + 1 allocations
            finished = True
            for a, b in zip(got, ref):
                assert torch.equal(a, b)
            break
    finally:
        P.debug_fail_alloc(-1)
    assert finished and failures > 20
    gc.collect()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (64 << 20), f"{(free0 - free1) >> 20} MiB not returned after {failures} failures"
    # and the library still works
    got = _sequence(P, inp)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)


def test_batch_graph_not_replayed_with_stale_workspace(P, oracle):
    imgs = [S.uniform_u8_grid(dd, seed=40 + i) for i, dd in enumerate(([30, 21], [17, 45]))]
    bt = P.CubicalBatch([cuda(x) for x in imgs])
    dA = cuda(S.circle_directions(64))
    dB = cuda(S.circle_directions(200))
    oA = torch.empty((2, 64, 40), dtype=torch.int64, device="cuda")
    oB = torch.empty((2, 200, 96), dtype=torch.int64, device="cuda")
    bt.wect(dA, 40, -SQ2, SQ2, out=oA)
    first = oA.clone()
    bt.wect(dB, 96, -SQ2, SQ2, out=oB)       # larger d and T: the workspace grows, other items
    oA.fill_(-7)
    bt.wect(dA, 40, -SQ2, SQ2, out=oA)       # same key as the first call
    torch.cuda.synchronize()
    assert torch.equal(oA, first)
    for i, x in enumerate(imgs):
        want = oracle.wect_cubical(list(reversed(x.shape)), x.ravel(), S.circle_directions(64), 40, -SQ2, SQ2)
        assert np.array_equal(oA[i].cpu().numpy(), want)
        wantB = oracle.wect_cubical(list(reversed(x.shape)), x.ravel(), S.circle_directions(200), 96, -SQ2, SQ2)
        assert np.array_equal(oB[i].cpu().numpy(), wantB)
