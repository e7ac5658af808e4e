"""GB300 (sm_103a) weighted Euler characteristic transform: Python binding of libwect.so.

This module only marshals arguments: every step of the transform runs in the CUDA library
(include/wect.h).  PyTorch provides device memory and the current stream.  There is no CPU
path: importing the binding without the built library, or calling it without a CUDA device,
raises.

Low-level functions carry the C names (``wect_complex_create_cubical``, ``wect_compute``,
``ecf_compute``, ``wect_backward``, ``wect_batch_*``).  The classes ``CubicalComplex``,
``SimplicialComplex`` and ``CubicalBatch`` wrap the handles; ``WECTFunction`` (batches of
grids) and ``ComplexWECTFunction`` (one grid or simplicial complex) are the
``torch.autograd.Function`` classes whose backward is the library's exact adjoint.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

from ._build import LIB as _LIB_PATH

__all__ = [
    "WectError", "load", "CubicalComplex", "FreudenthalComplex", "SimplicialComplex", "CubicalBatch", "WECTFunction",
    "ComplexWECTFunction",     "wect", "ecf", "launch_count", "library_path",
]

W_U8, W_I64_FIXED, W_F32, W_ONE = 0, 1, 2, 3
SW_MAX_OF_VERTICES, SW_EXPLICIT = 0, 1
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "OVERFLOW", 5: "TIMEOUT", 6: "UNSUPPORTED"}


class WectError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = _STATUS.get(status, str(status))


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libwect.so (built in-tree by ``__graft_entry__.build()`` / ``_build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libwect.so is not built ({_LIB_PATH}); run paper_2511_03909_gb300._build.build()")
    L = C.CDLL(_LIB_PATH)
    _declare(L)
    _lib = L
    return L


_st = C.c_int
_p = C.c_void_p
_i = C.c_int
_i64 = C.c_int64
_d = C.c_double


def _declare(L):
    sig = {
        "wect_complex_create_cubical": (_st, [_i, _p, _p, _i, _i, _p, _p]),
        "wect_complex_create_freudenthal": (_st, [_i, _p, _p, _i, _i, _p, _p]),
        "wect_complex_create_simplicial": (_st, [_i, _i64, _p, _i, _p, _p, _p, _i, _i, _i, _p, _p, _p]),
        "wect_complex_set_weights": (_st, [_p, _p, _p]),
        "wect_complex_num_vertices": (_i64, [_p]),
        "wect_complex_cell_counts": (_st, [_p, _p]),
        "wect_complex_device_status": (_st, [_p, _p]),
        "wect_complex_destroy": (None, [_p]),
        "wect_compute": (_st, [_p, _p, _i, _i, _d, _d, _p, _p]),
        "wect_compute_host": (_st, [_p, _p, _p, _i, _i, _d, _d, _p, _p]),
        "ecf_compute": (_st, [_p, _p, _i, _d, _d, _i, _p, _p]),
        "wecf_compute": (_st, [_p, _p, _i, _i, _d, _d, _i, _p, _p]),
        "wect_backward": (_st, [_p, _p, _i, _i, _d, _d, _p, _d, _p, _p]),
        "wect_backward_f64": (_st, [_p, _p, _i, _i, _d, _d, _p, _p, _p]),
        "wect_batch_create": (_st, [_i, _p, _p]),
        "wect_batch_create_cubical": (_st, [_i, _i, _p, _p, _i, _i, _p, _p]),
        "wect_batch_set_weights": (_st, [_p, _p, _p]),
        "wect_batch_count": (_i, [_p]),
        "wect_batch_total_vertices": (_i64, [_p]),
        "wect_batch_compute": (_st, [_p, _p, _i, _i, _d, _d, _p, _p]),
        "wect_batch_compute_loop": (_st, [_p, _p, _i, _i, _d, _d, _p, _p]),
        "wect_batch_backward": (_st, [_p, _p, _i, _i, _d, _d, _p, _d, _p, _p]),
        "wect_batch_backward_f64": (_st, [_p, _p, _i, _i, _d, _d, _p, _p, _p]),
        "wect_batch_autotune": (_st, [_p, _p, _i, _i, _d, _d, _p, _p]),
        "wect_batch_tuned_shape": (_st, [_p, _i, _i, _p]),
        "wect_batch_destroy": (None, [_p]),
        "wect_last_error": (C.c_char_p, []),
        "wect_version": (C.c_char_p, []),
        "wect_last_stencil_kernel": (C.c_char_p, []),
        "wect_kernel_launch_count": (_i64, []),
        "wect_profile_enable": (_st, [_i]),
        "wect_profile_read": (_st, [_p, _p]),
        "wect_cubical_compute_static": (_st, [_i, _p, _p, _i, _p, _i, _i, _d, _d, _p, _p]),
        "wect_cubical_static_status": (_st, [_p]),
        "wect_debug_fail_alloc": (_st, [_i64]),
        "wect_debug_stencil_variant": (_st, [_i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return [
        "wect_complex_create_cubical", "wect_complex_create_freudenthal", "wect_complex_create_simplicial",
        "wect_complex_set_weights",
        "wect_complex_num_vertices", "wect_complex_cell_counts", "wect_complex_device_status",
        "wect_complex_destroy", "wect_compute", "wect_compute_host", "ecf_compute", "wecf_compute", "wect_backward", "wect_backward_f64",
        "wect_batch_create",
        "wect_batch_create_cubical", "wect_batch_set_weights", "wect_batch_count", "wect_batch_total_vertices",
        "wect_batch_compute", "wect_batch_compute_loop", "wect_batch_backward", "wect_batch_backward_f64",
        "wect_batch_autotune", "wect_batch_tuned_shape",
        "wect_batch_destroy", "wect_last_error", "wect_version", "wect_last_stencil_kernel", "wect_kernel_launch_count",
        "wect_profile_enable", "wect_profile_read", "wect_cubical_compute_static", "wect_cubical_static_status",
        "wect_debug_fail_alloc", "wect_debug_stencil_variant",
    ]


def _check(status: int):
    if status != 0:
        raise WectError(status, load().wect_last_error().decode(errors="replace"))


def _stream(device=None) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor | None) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


def _require_cuda(t: torch.Tensor, name: str, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype} (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _wtype_of(w: torch.Tensor | None):
    if w is None:
        return W_ONE
    return {torch.uint8: W_U8, torch.int64: W_I64_FIXED, torch.float32: W_F32}[w.dtype]


def launch_count() -> int:
    """Kernels this process launched through the library (graph replays included)."""
    return int(load().wect_kernel_launch_count())


def profile_enable(on: bool = True):
    """Record CUDA events around each call's dominant kernel (see wect_profile_read)."""
    _check(load().wect_profile_enable(int(on)))


def profile_read():
    """(summed kernel milliseconds, number of timed launches) since the last read."""
    ms = C.c_double()
    n = C.c_int64()
    _check(load().wect_profile_read(C.byref(ms), C.byref(n)))
    return float(ms.value), int(n.value)


def last_stencil_kernel() -> str:
    """Name of the stencil kernel the last cubical forward used."""
    return load().wect_last_stencil_kernel().decode()


def debug_fail_alloc(k: int):
    """Test hook: the next k device allocations of the library succeed and the one after fails
    as out of memory (k < 0 disarms)."""
    _check(load().wect_debug_fail_alloc(int(k)))


def stencil_variant(variant: int):
    """wect_debug_stencil_variant: 0 = choose the cubical stencil kernel by cost, 1 = the
    per-vertex kernel only, 2 = the run-based kernel wherever it applies, 3 = the per-vertex
    kernel without the TMA staging of the neighbouring rows."""
    _check(load().wect_debug_stencil_variant(int(variant)))


def version() -> str:
    return load().wect_version().decode()


# ------------------------------------------------------------------ complexes


class _Complex:
    _h = None
    n = 0
    nv = 0
    frac_bits = 0
    wdtype = None       # torch dtype of the vertex weights (None: unweighted)

    def __del__(self):
        if self._h is not None and _lib is not None:
            try:
                _lib.wect_complex_destroy(self._h)
            except Exception:
                pass
            self._h = None

    @property
    def handle(self):
        return self._h

    def cell_counts(self):
        buf = (C.c_int64 * 5)()
        _check(load().wect_complex_cell_counts(self._h, buf))
        return [int(x) for x in buf]

    def set_weights(self, w: torch.Tensor):
        _require_cuda(w, "weights")
        _check(load().wect_complex_set_weights(self._h, _ptr(w), _stream()))

    def device_status(self):
        _check(load().wect_complex_device_status(self._h, _stream()))

    def wect(self, dirs: torch.Tensor, T: int, lo: float = math.nan, hi: float = math.nan,
             out: torch.Tensor | None = None) -> torch.Tensor:
        """[d][T] int64 WECT (wect_compute)."""
        _require_cuda(dirs, "dirs", torch.float64)
        d = dirs.shape[0]
        if dirs.dim() != 2 or dirs.shape[1] != self.n:
            raise ValueError(f"dirs must be [d][{self.n}]")
        if out is None:
            out = torch.empty((d, T), dtype=torch.int64, device=dirs.device)
        _require_cuda(out, "out", torch.int64)
        _check(load().wect_compute(self._h, _ptr(dirs), d, T, lo, hi, _ptr(out), _stream()))
        return out

    def wect_host(self, weights: torch.Tensor | None, dirs: torch.Tensor, T: int, lo: float = math.nan,
                  hi: float = math.nan, out: torch.Tensor | None = None, sync: bool = True) -> torch.Tensor:
        """wect_compute_host: new weights (or None to keep the current ones) and directions from
        host memory, the [d][T] int64 table into host memory (a page-locked tensor is allocated when
        out is None).  Page-locked tensors are read and written by the kernels directly.  With
        sync=False the caller synchronises the current stream before reading out."""
        for t, name in ((weights, "weights"), (dirs, "dirs"), (out, "out")):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous host tensor")
        if dirs.dtype != torch.float64 or dirs.dim() != 2 or dirs.shape[1] != self.n:
            raise ValueError(f"dirs must be float64 [d][{self.n}]")
        if weights is not None and (weights.numel() != self.nv or
                                    (self.wdtype is not None and weights.dtype != self.wdtype)):
            raise ValueError(f"weights must be {self.wdtype} with one value per vertex")
        d = dirs.shape[0]
        if out is None:
            out = torch.empty((d, T), dtype=torch.int64).pin_memory()
        if out.dtype != torch.int64 or out.numel() != d * T:
            raise ValueError("out must be int64 [d][T]")
        _check(load().wect_compute_host(self._h, None if weights is None else C.c_void_p(weights.data_ptr()),
                                        C.c_void_p(dirs.data_ptr()), d, T, lo, hi, C.c_void_p(out.data_ptr()),
                                        _stream()))
        if sync:
            torch.cuda.current_stream().synchronize()
        return out

    def ecf(self, filt: torch.Tensor, T: int, lo: float = math.nan, hi: float = math.nan, weighted: bool = False,
            out: torch.Tensor | None = None) -> torch.Tensor:
        """[T] int64 ECF / WECF of one vertex filter (ecf_compute)."""
        _require_cuda(filt, "filter", torch.float64)
        if filt.numel() != self.nv:
            raise ValueError("filter must have one value per vertex")
        if out is None:
            out = torch.empty(T, dtype=torch.int64, device=filt.device)
        _check(load().ecf_compute(self._h, _ptr(filt), T, lo, hi, int(weighted), _ptr(out), _stream()))
        return out

    def wecf(self, filters: torch.Tensor, T: int, lo: float = math.nan, hi: float = math.nan,
             weighted: bool = True, out: torch.Tensor | None = None) -> torch.Tensor:
        """[m][T] int64 WECF table of m vertex filters given as [m][nv] float64 (wecf_compute)."""
        _require_cuda(filters, "filters", torch.float64)
        if filters.dim() != 2 or filters.shape[1] != self.nv:
            raise ValueError("filters must be [m][nv]")
        m = filters.shape[0]
        if out is None:
            out = torch.empty((m, T), dtype=torch.int64, device=filters.device)
        _require_cuda(out, "out", torch.int64)
        _check(load().wecf_compute(self._h, _ptr(filters), m, T, lo, hi, int(weighted), _ptr(out), _stream()))
        return out

    def backward(self, dirs: torch.Tensor, T: int, lo: float, hi: float, dW: torch.Tensor, scale: float,
                 grad: torch.Tensor | None = None) -> torch.Tensor:
        """[nv] float32 adjoint (wect_backward)."""
        _require_cuda(dirs, "dirs", torch.float64)
        _require_cuda(dW, "dW", torch.int64)
        if grad is None:
            grad = torch.empty(self.nv, dtype=torch.float32, device=dirs.device)
        _check(load().wect_backward(self._h, _ptr(dirs), dirs.shape[0], T, lo, hi, _ptr(dW), float(scale), _ptr(grad),
                                    _stream()))
        return grad

    def backward_f64(self, dirs: torch.Tensor, T: int, lo: float, hi: float, G: torch.Tensor,
                     grad: torch.Tensor | None = None) -> torch.Tensor:
        """Adjoint for a float64 upstream gradient in real units (wect_backward_f64)."""
        _require_cuda(dirs, "dirs", torch.float64)
        _require_cuda(G, "G", torch.float64)
        if G.shape != (dirs.shape[0], T):
            raise ValueError("G must be [d][T]")
        if grad is None:
            grad = torch.empty(self.nv, dtype=torch.float32, device=dirs.device)
        _check(load().wect_backward_f64(self._h, _ptr(dirs), dirs.shape[0], T, lo, hi, _ptr(G), _ptr(grad), _stream()))
        return grad


class CubicalComplex(_Complex):
    """Full cubical complex of an n-dimensional grid (wect_complex_create_cubical).

    ``weights``: CUDA tensor of shape (L_{n-1}, ..., L_0) (axis 0 fastest), dtype uint8, int64
    (fixed point) or float32 (converted with ``frac_bits``); ``None`` for the unweighted complex
    (then ``dims`` gives the axis lengths, axis 0 first).
    """

    def __init__(self, weights: torch.Tensor | None, frac_bits: int = 0, dims=None):
        L = load()
        self.frac_bits = int(frac_bits)
        if weights is not None:
            _require_cuda(weights, "weights")
            dims = list(reversed(weights.shape))
            self.wdtype = weights.dtype
        elif dims is None:
            raise ValueError("dims is required for an unweighted grid")
        self.n = len(dims)
        self.dims = [int(x) for x in dims]
        self.nv = int(math.prod(self.dims))
        dims_a = (C.c_int64 * self.n)(*self.dims)
        h = C.c_void_p()
        _check(L.wect_complex_create_cubical(self.n, dims_a, _ptr(weights), _wtype_of(weights), frac_bits, _stream(),
                                             C.byref(h)))
        self._h = h


class FreudenthalComplex(_Complex):
    """Freudenthal (Kuhn) triangulation of a full grid, built on the device
    (wect_complex_create_freudenthal): a simplicial complex.  ``weights`` and ``dims`` as for
    CubicalComplex."""

    def __init__(self, weights: torch.Tensor | None, frac_bits: int = 0, dims=None):
        L = load()
        self.frac_bits = int(frac_bits)
        if weights is not None:
            _require_cuda(weights, "weights")
            dims = list(reversed(weights.shape))
            self.wdtype = weights.dtype
        elif dims is None:
            raise ValueError("dims is required for an unweighted grid")
        self.n = len(dims)
        self.dims = [int(x) for x in dims]
        self.nv = int(math.prod(self.dims))
        dims_a = (C.c_int64 * self.n)(*self.dims)
        h = C.c_void_p()
        _check(L.wect_complex_create_freudenthal(self.n, dims_a, _ptr(weights), _wtype_of(weights), frac_bits,
                                                 _stream(), C.byref(h)))
        self._h = h


class SimplicialComplex(_Complex):
    """Geometric simplicial complex (wect_complex_create_simplicial).

    ``coords``: [nv][n] float64 CUDA; ``simplices``: list of int32 CUDA tensors [k_i][i+1] for
    i = 1..max_dim; ``weights``: [nv] CUDA (uint8 / int64 fixed / float32) or None (unweighted);
    ``simplex_weights``: optional list (index 0 = vertices) of int64 CUDA tensors (explicit mode).
    """

    def __init__(self, coords: torch.Tensor, simplices, weights: torch.Tensor | None = None, frac_bits: int = 0,
                 simplex_weights=None):
        L = load()
        self.frac_bits = int(frac_bits)
        _require_cuda(coords, "coords", torch.float64)
        self.nv, self.n = int(coords.shape[0]), int(coords.shape[1])
        self.wdtype = None if weights is None else weights.dtype
        self.max_dim = len(simplices)
        counts = (C.c_int64 * (self.max_dim + 1))(self.nv, *[int(s.shape[0]) for s in simplices])
        for i, s in enumerate(simplices):
            _require_cuda(s, f"simplices[{i + 1}]", torch.int32)
        sp = (C.c_void_p * (self.max_dim + 1))(None, *[s.data_ptr() for s in simplices])
        self._keep = (coords, list(simplices))
        mode = SW_MAX_OF_VERTICES
        swp = None
        if simplex_weights is not None:
            mode = SW_EXPLICIT
            swp = (C.c_void_p * (self.max_dim + 1))(*[(w.data_ptr() if w is not None else None) for w in simplex_weights])
        h = C.c_void_p()
        _check(L.wect_complex_create_simplicial(self.n, self.nv, _ptr(coords), self.max_dim, counts, sp, _ptr(weights),
                                                _wtype_of(weights), frac_bits, mode, swp, _stream(), C.byref(h)))
        self._h = h
        self._keep = None


# ------------------------------------------------------------------ batches


class CubicalBatch:
    """Many cubical grids computed by one persistent, graph-captured launch.

    ``CubicalBatch(weights_list)`` copies each grid (uint8 / int64 / float32 CUDA tensors of
    the same dtype and rank) into one batch-owned buffer (wect_batch_create_cubical).
    """

    def __init__(self, weights_list=None, frac_bits: int = 0, flat: torch.Tensor | None = None, dims=None):
        L = load()
        if weights_list is not None:
            self.n = weights_list[0].dim()
            dims = [list(reversed(w.shape)) for w in weights_list]
            flat = torch.cat([w.reshape(-1) for w in weights_list])
        elif flat is None or dims is None:
            raise ValueError("give weights_list, or flat weights and dims")
        self.n = len(dims[0])
        self.count = len(dims)
        self.dims = [[int(x) for x in dd] for dd in dims]
        self.sizes = [int(math.prod(dd)) for dd in self.dims]
        self.total = sum(self.sizes)
        self.dtype = flat.dtype
        _require_cuda(flat, "weights")
        dims_a = (C.c_int64 * (self.count * self.n))(*[x for dd in self.dims for x in dd])
        h = C.c_void_p()
        _check(L.wect_batch_create_cubical(self.count, self.n, dims_a, _ptr(flat), _wtype_of(flat), frac_bits, _stream(),
                                           C.byref(h)))
        self._h = h
        self.frac_bits = frac_bits

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            try:
                _lib.wect_batch_destroy(self._h)
            except Exception:
                pass
            self._h = None

    def set_weights(self, flat: torch.Tensor):
        _require_cuda(flat, "weights")
        if flat.numel() != self.total or flat.dtype != self.dtype:
            raise ValueError("weights must match the batch's size and dtype")
        _check(load().wect_batch_set_weights(self._h, _ptr(flat), _stream()))

    def wect(self, dirs: torch.Tensor, T: int, lo: float, hi: float, out: torch.Tensor | None = None,
             loop: bool = False) -> torch.Tensor:
        _require_cuda(dirs, "dirs", torch.float64)
        d = dirs.shape[0]
        if out is None:
            out = torch.empty((self.count, d, T), dtype=torch.int64, device=dirs.device)
        fn = load().wect_batch_compute_loop if loop else load().wect_batch_compute
        _check(fn(self._h, _ptr(dirs), d, T, lo, hi, _ptr(out), _stream()))
        return out

    def backward_f64(self, dirs: torch.Tensor, T: int, lo: float, hi: float, G: torch.Tensor,
                     grad: torch.Tensor | None = None) -> torch.Tensor:
        """Adjoint for a float64 upstream gradient in real units (wect_batch_backward_f64)."""
        _require_cuda(G, "G", torch.float64)
        if grad is None:
            grad = torch.empty(self.total, dtype=torch.float32, device=dirs.device)
        _check(load().wect_batch_backward_f64(self._h, _ptr(dirs), dirs.shape[0], T, lo, hi, _ptr(G), _ptr(grad),
                                              _stream()))
        return grad

    def autotune(self, dirs: torch.Tensor, T: int, lo: float, hi: float):
        scratch = torch.empty((self.count, dirs.shape[0], T), dtype=torch.int64, device=dirs.device)
        _check(load().wect_batch_autotune(self._h, _ptr(dirs), dirs.shape[0], T, lo, hi, _ptr(scratch), _stream()))

    def tuned_shape(self, d: int, T: int):
        """(directions per lane, tile width, run kernel, CTA size) chosen by autotune for (d, T),
        or None when (d, T) is not tuned."""
        buf = (C.c_int * 4)()
        _check(load().wect_batch_tuned_shape(self._h, int(d), int(T), buf))
        return None if buf[1] == 0 else (int(buf[0]), int(buf[1]), bool(buf[2]), int(buf[3]))

    def backward(self, dirs: torch.Tensor, T: int, lo: float, hi: float, dW: torch.Tensor, scale: float,
                 grad: torch.Tensor | None = None) -> torch.Tensor:
        _require_cuda(dW, "dW", torch.int64)
        if grad is None:
            grad = torch.empty(self.total, dtype=torch.float32, device=dirs.device)
        _check(load().wect_batch_backward(self._h, _ptr(dirs), dirs.shape[0], T, lo, hi, _ptr(dW), float(scale),
                                          _ptr(grad), _stream()))
        return grad


# ------------------------------------------------------------------ autograd


class WECTFunction(torch.autograd.Function):
    """W = WECT(weights) for a CubicalBatch, with the library's exact adjoint as backward.

    forward(batch, weights_flat_f32, dirs, T, lo, hi) -> float64 [count][d][T] in real units
    (int64 fixed-point result * 2^-frac_bits).  backward passes the float64 upstream gradient to
    wect_batch_backward_f64 (quantised to int64 fixed point on the device, no host sync).
    """

    @staticmethod
    def forward(ctx, batch: CubicalBatch, w: torch.Tensor, dirs: torch.Tensor, T: int, lo: float, hi: float):
        batch.set_weights(w.detach().contiguous())
        W = batch.wect(dirs, T, lo, hi)
        ctx.batch, ctx.dirs, ctx.T, ctx.lo, ctx.hi = batch, dirs, T, lo, hi
        return W.to(torch.float64) * (2.0 ** -batch.frac_bits)     # exact: a power of two

    @staticmethod
    def backward(ctx, gW: torch.Tensor):
        b = ctx.batch
        grad = b.backward_f64(ctx.dirs, ctx.T, ctx.lo, ctx.hi, gW.to(torch.float64).contiguous())
        return None, grad, None, None, None, None


class ComplexWECTFunction(torch.autograd.Function):
    """W = WECT(vertex weights) of one complex (grid, Freudenthal or simplicial in max-of-vertices
    mode), with the library's exact adjoint as backward.

    forward(complex, weights, dirs, T, lo, hi) -> float64 [d][T] in real units (the int64
    fixed-point result * 2^-frac_bits).  ``weights`` are the vertex weights in the form the
    complex was created with (set on the complex by the forward).  backward passes the float64
    upstream gradient to wect_backward_f64 (quantised on the device, no host sync) and returns
    a float32 gradient per vertex, in the shape of ``weights``.
    """

    @staticmethod
    def forward(ctx, cx: _Complex, w: torch.Tensor, dirs: torch.Tensor, T: int, lo: float, hi: float):
        cx.set_weights(w.detach().contiguous())
        W = cx.wect(dirs, T, lo, hi)
        ctx.cx, ctx.dirs, ctx.T, ctx.lo, ctx.hi, ctx.wshape = cx, dirs, T, lo, hi, w.shape
        return W.to(torch.float64) * (2.0 ** -cx.frac_bits)     # exact: a power of two

    @staticmethod
    def backward(ctx, gW: torch.Tensor):
        grad = ctx.cx.backward_f64(ctx.dirs, ctx.T, ctx.lo, ctx.hi, gW.to(torch.float64).contiguous())
        return None, grad.view(ctx.wshape), None, None, None, None


# ------------------------------------------------------------------ allocation-free variant


def cubical_wect_static(weights: torch.Tensor | None, dirs: torch.Tensor, T: int, lo: float = math.nan,
                        hi: float = math.nan, out: torch.Tensor | None = None, dims=None) -> torch.Tensor:
    """wect_cubical_compute_static: the WECT of a uint8 (or unweighted) grid without any device
    allocation by the library (scratch in a static device array; see include/wect.h).  ``out``
    may be preallocated by the caller, so that the call itself allocates nothing either."""
    if weights is not None:
        _require_cuda(weights, "weights", torch.uint8)
        dims = list(reversed(weights.shape))
    _require_cuda(dirs, "dirs", torch.float64)
    n = len(dims)
    d = dirs.shape[0]
    if out is None:
        out = torch.empty((d, T), dtype=torch.int64, device=dirs.device)
    _require_cuda(out, "out", torch.int64)
    dims_a = (C.c_int64 * n)(*[int(x) for x in dims])
    _check(load().wect_cubical_compute_static(n, dims_a, _ptr(weights), W_U8 if weights is not None else W_ONE,
                                              _ptr(dirs), d, T, lo, hi, _ptr(out), _stream()))
    return out


def cubical_static_status():
    """wect_cubical_static_status: raise WectError when the device-side checks of the last
    allocation-free call on this device failed (a non-finite direction); clears the status."""
    _check(load().wect_cubical_static_status(_stream()))


# ------------------------------------------------------------------ one-shot helpers


def wect(weights: torch.Tensor, dirs: torch.Tensor, T: int, lo: float = math.nan, hi: float = math.nan,
         frac_bits: int = 0) -> torch.Tensor:
    """WECT of the cubical complex of a grid of vertex weights."""
    return CubicalComplex(weights, frac_bits).wect(dirs, T, lo, hi)


def ecf(values: torch.Tensor, T: int, lo: float = math.nan, hi: float = math.nan) -> torch.Tensor:
    """ECF of an image or volume (the intensity is the vertex filter, every cell has weight 1)."""
    cx = CubicalComplex(None, dims=list(reversed(values.shape)))
    return cx.ecf(values.reshape(-1).to(torch.float64).contiguous(), T, lo, hi, weighted=False)
