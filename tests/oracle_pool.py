"""The CPU oracle spread over the host cores, for the full-size parity tests.

TEST INFRASTRUCTURE ONLY.  Worker processes are started with ``spawn`` (safe after CUDA has
been initialised in the parent); each one regenerates the seeded synthetic workloads it needs
(cached per process) and runs the unchanged, single-threaded C oracle on one slice of the work:
a few directions of a transform, a few images of a batch, or one volume's adjoint.  The slices
are independent, so the union of the results is the oracle's result for the whole workload.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_CACHE: dict = {}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _O():
    from oracle import oracle as O

    O.build()
    return O


def _workload(name: str):
    if name not in _CACHE:
        import synthetic as S

        _CACHE[name] = getattr(S, name)()
    return _CACHE[name]


# ------------------------------------------------------------------ worker tasks


def voxel_dirs(i0: int, i1: int) -> np.ndarray:
    """Transform of the 128^3 voxel workload for directions i0 .. i1-1."""
    O = _O()
    wl = _workload("voxel3d_128")
    return O.wect_cubical(wl.dims, wl.grid.ravel().astype(np.int64), wl.dirs[i0:i1], wl.T, wl.lo, wl.hi)


def _mesh_inputs():
    key = "mesh2d_1024_inputs"
    if key not in _CACHE:
        O = _O()
        wl = _workload("mesh2d_1024")
        cx = wl.complex
        vw = O.fixed_from_f32(cx.weights, 24)
        _CACHE[key] = (wl, cx, O.simplicial_weights(cx.simplices, vw))
    return _CACHE[key]


def mesh_range() -> tuple:
    """The paper's default range [-M, M] of the 1024^2 mesh over all of its directions."""
    key = "mesh2d_1024_range"
    if key not in _CACHE:
        O = _O()
        wl, cx, _ = _mesh_inputs()
        _CACHE[key] = O.default_range_simplicial(cx.coords, wl.dirs)
    return _CACHE[key]


def mesh_dirs(idx: list) -> np.ndarray:
    """Transform of the 1024^2 mesh for the listed directions over its default range."""
    O = _O()
    wl, cx, sw = _mesh_inputs()
    lo, hi = mesh_range()
    return O.wect_simplicial(cx.coords, cx.simplices, sw, wl.dirs[idx], wl.T, lo, hi)


def images(i0: int, i1: int) -> list:
    """Transforms of images i0 .. i1-1 of the 4096-image batch."""
    O = _O()
    wl = _workload("image_batch")
    return [O.wect_cubical(list(reversed(x.shape)), x.ravel(), wl.dirs, wl.T, wl.lo, wl.hi)
            for x in wl.grids[i0:i1]]


def volume_adjoint(vw: np.ndarray, tw: np.ndarray, dims, dirs, T: int, lo: float, hi: float, N: int):
    """One volume of the differentiation workload: its transform W, the target's B, and the exact
    adjoint of the mean squared error (1/N) sum (W - B)^2 in real units (2^-24 fixed point)."""
    O = _O()
    W = O.wect_cubical(dims, vw, dirs, T, lo, hi)
    B = O.wect_cubical(dims, tw, dirs, T, lo, hi)
    g = O.wect_backward_cubical(dims, vw, dirs, T, lo, hi, W - B, 2.0 ** -23 / N)
    return W, B, g


def ecf_filter(dims, seed: int) -> np.ndarray:
    """Uniform [0, 1) float64 vertex filter of a grid (an intensity image or volume)."""
    return np.random.default_rng(seed).random(int(np.prod(dims)))


def ecf_grid(dims, seed: int, T: int) -> np.ndarray:
    """Unweighted ECF of the full cubical grid for the filter ecf_filter(dims, seed) over [0, 1]."""
    O = _O()
    nv = int(np.prod(dims))
    return O.wecf_cubical(dims, np.zeros(nv, dtype=np.int64), ecf_filter(dims, seed), T, 0.0, 1.0, weighted=False)[0]


def _noop(k):
    return k


# ------------------------------------------------------------------ pool


class OraclePool:
    """A spawn pool of one process per host core."""

    def __init__(self, nproc: int | None = None):
        _O()                                   # build the oracle once, before the workers load it
        self.nproc = nproc or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.nproc)

    def submit(self, fn, *args):
        return self.pool.apply_async(fn, args)

    def close(self):
        self.pool.terminate()
        self.pool.join()
