"""ctypes front end of the C oracle (wect_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  The product library never imports, links or executes anything here.

Every function takes and returns numpy arrays; weights are int64 fixed point.
The oracle follows the plain definition of the WECT (Section 3, proof of Algorithm 1):
W[p][q] = sum over simplices s with bin(max_{v in s} f_p(v)) <= q of (-1)^dim(s) w(s).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wect_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile wect_oracle.c with gcc (strict IEEE float64, no contraction) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_d = C.c_double
_i = C.c_int
_i64 = C.c_int64
_p = C.c_void_p


def _declare(L):
    L.wo_height.restype = _d
    L.wo_height.argtypes = [_i, _p, _p]
    L.wo_beta.restype = None
    L.wo_beta.argtypes = [_i, _d, _d, _p]
    L.wo_bin.restype = _i
    L.wo_bin.argtypes = [_d, _p, _i]
    L.wo_grid_coord.restype = _d
    L.wo_grid_coord.argtypes = [_i64, _i64]
    L.wo_fixed_from_f32_array.restype = None
    L.wo_fixed_from_f32_array.argtypes = [_p, _i64, _i, _p]
    L.wo_scatter_add.restype = None
    L.wo_scatter_add.argtypes = [_i64, _i64, _i64, _p, _p, _p]
    L.wo_cumsum_rows.restype = None
    L.wo_cumsum_rows.argtypes = [_i64, _i64, _p]
    L.wo_rmax_rows.restype = None
    L.wo_rmax_rows.argtypes = [_i64, _i64, _p, _p]
    L.wo_simplex_weights_max.restype = None
    L.wo_simplex_weights_max.argtypes = [_i, _i64, _p, _p, _p]
    L.wo_max_abs_height.restype = _d
    L.wo_max_abs_height.argtypes = [_i, _i64, _p, _i, _p]
    L.wo_grid_max_abs_height.restype = _d
    L.wo_grid_max_abs_height.argtypes = [_i, _p, _i, _p]
    L.wo_wecf_filters.restype = _i
    L.wo_wecf_filters.argtypes = [_i, _i64, _p, _i, _p, _p, _p, _i, _d, _d, _p]
    L.wo_wect_simplicial.restype = _i
    L.wo_wect_simplicial.argtypes = [_i, _i64, _p, _i, _p, _p, _p, _i, _p, _i, _d, _d, _p]
    L.wo_wecf_cubical_filters.restype = _i
    L.wo_wecf_cubical_filters.argtypes = [_i, _p, _p, _i, _i, _p, _i, _d, _d, _p]
    L.wo_wect_cubical.restype = _i
    L.wo_wect_cubical.argtypes = [_i, _p, _p, _i, _i, _p, _i, _d, _d, _p]
    L.wo_wect_backward_cubical.restype = _i
    L.wo_wect_backward_cubical.argtypes = [_i, _p, _p, _i, _p, _i, _d, _d, _p, _d, _p]
    L.wo_wect_backward_simplicial.restype = _i
    L.wo_wect_backward_simplicial.argtypes = [_i, _i64, _p, _p, _i, _p, _p, _i, _p, _i, _d, _d, _p, _d, _p]
    L.wo_i128_to_double.restype = _d
    L.wo_i128_to_double.argtypes = [_i64, C.c_uint64]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ primitives


def height(x, s) -> float:
    x = _c(x, np.float64)
    s = _c(s, np.float64)
    return lib().wo_height(len(x), _ptr(x), _ptr(s))


def beta(T: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(T, dtype=np.float64)
    lib().wo_beta(T, lo, hi, _ptr(out))
    return out


def bin_of(t: float, beta_table: np.ndarray) -> int:
    b = _c(beta_table, np.float64)
    return lib().wo_bin(float(t), _ptr(b), len(b))


def grid_coord(i: int, L: int) -> float:
    return lib().wo_grid_coord(i, L)


def fixed_from_f32(w, frac_bits: int) -> np.ndarray:
    w = _c(w, np.float32).ravel()
    out = np.empty(w.size, dtype=np.int64)
    lib().wo_fixed_from_f32_array(_ptr(w), w.size, frac_bits, _ptr(out))
    return out


def to_fixed(w, frac_bits: int = 0) -> np.ndarray:
    """Vertex weights of any supported dtype as int64 fixed point (u8 / ints as is, f32 rounded)."""
    w = np.asarray(w)
    if w.dtype == np.float32:
        return fixed_from_f32(w, frac_bits)
    if w.dtype.kind in "iu":
        return np.ascontiguousarray(w.ravel(), dtype=np.int64)
    raise TypeError(f"unsupported weight dtype {w.dtype}")


def scatter_add(S: np.ndarray, I: np.ndarray, V: np.ndarray) -> np.ndarray:
    S = _c(S, np.int64).copy()
    I = _c(I, np.int64)
    V = _c(V, np.int64)
    m0, m1 = S.shape
    lib().wo_scatter_add(m0, m1, I.shape[1], _ptr(I), _ptr(V), _ptr(S))
    return S


def cumsum_rows(S: np.ndarray) -> np.ndarray:
    S = _c(S, np.int64).copy()
    lib().wo_cumsum_rows(S.shape[0], S.shape[1], _ptr(S))
    return S


def rmax_rows(Tm: np.ndarray) -> np.ndarray:
    Tm = _c(Tm, np.int64)
    out = np.empty(Tm.shape[0], dtype=np.int64)
    lib().wo_rmax_rows(Tm.shape[0], Tm.shape[1], _ptr(Tm), _ptr(out))
    return out


def i128_to_double(v: int) -> float:
    lo = v & ((1 << 64) - 1)
    hi = v >> 64
    return lib().wo_i128_to_double(hi, lo)


# ------------------------------------------------------------------ ranges


def default_range_simplicial(coords, dirs):
    coords = _c(coords, np.float64)
    dirs = _c(dirs, np.float64)
    M = lib().wo_max_abs_height(coords.shape[1], coords.shape[0], _ptr(coords), dirs.shape[0], _ptr(dirs))
    return -M, M


def default_range_grid(dims, dirs):
    dims_a = _c(dims, np.int64)
    dirs = _c(dirs, np.float64)
    M = lib().wo_grid_max_abs_height(len(dims_a), _ptr(dims_a), dirs.shape[0], _ptr(dirs))
    return -M, M


def _resolve(lo, hi, fn):
    if math.isnan(lo) and math.isnan(hi):
        return fn()
    return float(lo), float(hi)


# ------------------------------------------------------------------ transforms


def simplex_weights_max(simplices: np.ndarray, vw: np.ndarray) -> np.ndarray:
    s = _c(simplices, np.int32)
    vw = _c(vw, np.int64)
    out = np.empty(s.shape[0], dtype=np.int64)
    lib().wo_simplex_weights_max(s.shape[1] - 1, s.shape[0], _ptr(s), _ptr(vw), _ptr(out))
    return out


def _simplicial_args(nv, simplices, weights):
    max_dim = len(simplices)
    counts = np.array([nv] + [s.shape[0] for s in simplices], dtype=np.int64)
    sl = [_c(s, np.int32) for s in simplices]
    wl = [_c(w, np.int64) for w in weights]
    sp = (C.c_void_p * (max_dim + 1))(None, *[_ptr(s) for s in sl])
    wp = (C.c_void_p * (max_dim + 1))(*[_ptr(w) for w in wl])
    return max_dim, counts, sl, wl, sp, wp


def simplicial_weights(simplices, vw, mode="max"):
    """Per-dimension weight lists: [vertex weights, w(edges), w(triangles), ...]."""
    vw = _c(vw, np.int64)
    if mode == "max":
        return [vw] + [simplex_weights_max(s, vw) for s in simplices]
    if mode == "one":
        return [np.ones_like(vw)] + [np.ones(s.shape[0], dtype=np.int64) for s in simplices]
    raise ValueError(mode)


def wect_simplicial(coords, simplices, weights, dirs, T, lo=math.nan, hi=math.nan) -> np.ndarray:
    """weights: list per dimension (index 0 = vertices) of int64 simplex weights."""
    coords = _c(coords, np.float64)
    dirs = _c(dirs, np.float64)
    lo, hi = _resolve(lo, hi, lambda: default_range_simplicial(coords, dirs))
    nv, n = coords.shape
    max_dim, counts, sl, wl, sp, wp = _simplicial_args(nv, simplices, weights)
    out = np.empty((dirs.shape[0], T), dtype=np.int64)
    rc = lib().wo_wect_simplicial(n, nv, _ptr(coords), max_dim, _ptr(counts), sp, wp,
                                  dirs.shape[0], _ptr(dirs), T, lo, hi, _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def wecf_simplicial(f, simplices, weights, T, lo=math.nan, hi=math.nan) -> np.ndarray:
    """Algorithm 1 for m filters given as f[m][nv]."""
    f = np.atleast_2d(_c(f, np.float64))
    m, nv = f.shape
    if math.isnan(lo) and math.isnan(hi):
        M = float(np.max(np.abs(f))) if f.size else 0.0
        lo, hi = -M, M
    max_dim, counts, sl, wl, sp, wp = _simplicial_args(nv, simplices, weights)
    out = np.empty((m, T), dtype=np.int64)
    rc = lib().wo_wecf_filters(m, nv, _ptr(f), max_dim, _ptr(counts), sp, wp, T, lo, hi, _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def wect_cubical(dims, vw, dirs, T, lo=math.nan, hi=math.nan, weighted=True) -> np.ndarray:
    dims_a = _c(dims, np.int64)
    vw = _c(np.asarray(vw).ravel(), np.int64)
    dirs = _c(dirs, np.float64)
    lo, hi = _resolve(lo, hi, lambda: default_range_grid(dims, dirs))
    out = np.empty((dirs.shape[0], T), dtype=np.int64)
    rc = lib().wo_wect_cubical(len(dims_a), _ptr(dims_a), _ptr(vw), int(weighted), dirs.shape[0], _ptr(dirs),
                               T, lo, hi, _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def wecf_cubical(dims, vw, f, T, lo=math.nan, hi=math.nan, weighted=True) -> np.ndarray:
    """WECF of a full cubical grid for m vertex filters f[m][nv] (the ECF when m = 1)."""
    dims_a = _c(dims, np.int64)
    vw = _c(np.asarray(vw).ravel(), np.int64)
    f = np.atleast_2d(_c(f, np.float64))
    if math.isnan(lo) and math.isnan(hi):
        M = float(np.max(np.abs(f))) if f.size else 0.0
        lo, hi = -M, M
    out = np.empty((f.shape[0], T), dtype=np.int64)
    rc = lib().wo_wecf_cubical_filters(len(dims_a), _ptr(dims_a), _ptr(vw), int(weighted), f.shape[0], _ptr(f),
                                       T, lo, hi, _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def grid_coords(dims) -> np.ndarray:
    """[nv][n] coordinates of the grid vertices (axis 0 fastest), via the oracle's coordinate rule."""
    n = len(dims)
    axes = [np.array([grid_coord(i, L) for i in range(L)], dtype=np.float64) for L in dims]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")            # slowest axis first
    cols = [m.ravel() for m in reversed(mesh)]                      # back to axis 0 first
    return np.ascontiguousarray(np.stack(cols, axis=1)) if n else np.zeros((1, 0))


def wect_backward_cubical(dims, vw, dirs, T, lo, hi, G, scale) -> np.ndarray:
    dims_a = _c(dims, np.int64)
    vw = _c(np.asarray(vw).ravel(), np.int64)
    dirs = _c(dirs, np.float64)
    G = _c(G, np.int64)
    out = np.empty(vw.size, dtype=np.float32)
    rc = lib().wo_wect_backward_cubical(len(dims_a), _ptr(dims_a), _ptr(vw), dirs.shape[0], _ptr(dirs), T, lo, hi,
                                        _ptr(G), scale, _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def wect_backward_simplicial(coords, vw, simplices, dirs, T, lo, hi, G, scale) -> np.ndarray:
    coords = _c(coords, np.float64)
    vw = _c(vw, np.int64)
    dirs = _c(dirs, np.float64)
    G = _c(G, np.int64)
    nv, n = coords.shape
    max_dim, counts, sl, wl, sp, wp = _simplicial_args(nv, simplices, [vw] * (len(simplices) + 1))
    out = np.empty(nv, dtype=np.float32)
    rc = lib().wo_wect_backward_simplicial(n, nv, _ptr(coords), _ptr(vw), max_dim, _ptr(counts), sp,
                                           dirs.shape[0], _ptr(dirs), T, lo, hi, _ptr(G), scale, _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out
