"""FP64 CPU oracle for dealiased real linear convolutions.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.  The
product path (the CUDA library and its binding) never imports, links or calls
it, and the oracle imports nothing from the product package.

Two layers:

* ``hdoracle.c`` (loaded through ctypes): the plain definition of the result.
  O1 ``direct_conv`` is direct FP64 summation, O1' ``direct_corr`` the adjoint
  correlation, O2 ``fft_conv`` an explicitly zero-padded radix-2 FFT
  convolution written from scratch; ``direct_conv_multi``/``fft_conv_multi``
  the same two for n >= 2 1D arrays of possibly different lengths.
* ``steps.py``: an FP64 NumPy transcription of the paper's equations step by
  step (residue transforms, conjugate-symmetry cases, implicit packing, the RCM
  operator and its multidimensional form), used to pin intermediate quantities
  and the algebraic identities the paper states.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle, LIB_PATH

_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH) or _stale():
            build_oracle()
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        for name in ("hd_direct_conv", "hd_direct_corr", "hd_fft_conv"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int, P, P, P, P, P]
            fn.restype = ctypes.c_int
        lib.hd_direct_conv_points.argtypes = [ctypes.c_int, P, ctypes.c_int64, P, P, P, P]
        lib.hd_direct_conv_points.restype = ctypes.c_int
        lib.hd_batch_conv1d.argtypes = [ctypes.c_int64, P, P, P, P, P, ctypes.c_int]
        lib.hd_batch_conv1d.restype = ctypes.c_int
        for name in ("hd_direct_conv_multi", "hd_fft_conv_multi"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, P]
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def _stale():
    src = os.path.join(os.path.dirname(__file__), "hdoracle.c")
    return os.path.getmtime(src) > os.path.getmtime(LIB_PATH)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(f, g, K):
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    if f.shape != g.shape or f.ndim < 1 or f.ndim > 3:
        raise ValueError("f and g must share a 1D/2D/3D shape")
    L = np.asarray(f.shape, dtype=np.int64)
    K = L.copy() if K is None else np.asarray(K, dtype=np.int64).reshape(L.shape)
    return f, g, L, K


def direct_conv(f, g, K=None):
    """O1: h[k] = sum_j f[j] g[k-j] for 0 <= k_i < K_i (default K = L)."""
    f, g, L, K = _prep(f, g, K)
    h = np.empty(tuple(K), dtype=np.float64)
    rc = _load().hd_direct_conv(f.ndim, _ptr(L), _ptr(K), _ptr(f), _ptr(g), _ptr(h))
    if rc:
        raise ValueError(f"hd_direct_conv failed ({rc})")
    return h


def direct_conv_points(f, g, points):
    """O1 at chosen output multi-indices (rows of ``points``), by direct summation."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    L = np.asarray(f.shape, dtype=np.int64)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int64).reshape(-1, f.ndim))
    out = np.empty(len(pts), dtype=np.float64)
    rc = _load().hd_direct_conv_points(f.ndim, _ptr(L), len(pts), _ptr(pts), _ptr(f), _ptr(g), _ptr(out))
    if rc:
        raise ValueError(f"hd_direct_conv_points failed ({rc})")
    return out


def direct_corr(u, g, L=None):
    """O1': grad[j] = sum_k u[k] g[k-j]; the adjoint of f -> conv_K(f, g).

    ``u`` has the output extents K, ``g`` the input extents L."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    Ls = np.asarray(g.shape, dtype=np.int64)
    K = np.asarray(u.shape, dtype=np.int64)
    grad = np.empty(g.shape, dtype=np.float64)
    rc = _load().hd_direct_corr(g.ndim, _ptr(Ls), _ptr(K), _ptr(u), _ptr(g), _ptr(grad))
    if rc:
        raise ValueError(f"hd_direct_corr failed ({rc})")
    return grad


def fft_conv(f, g, K=None):
    """O2: explicitly zero-padded FP64 FFT convolution, first K per dim."""
    f, g, L, K = _prep(f, g, K)
    h = np.empty(tuple(K), dtype=np.float64)
    rc = _load().hd_fft_conv(f.ndim, _ptr(L), _ptr(K), _ptr(f), _ptr(g), _ptr(h))
    if rc:
        raise ValueError(f"hd_fft_conv failed ({rc})")
    return h


def batch_conv1d(f, g, offsets, lengths, use_fft=True):
    """Independent 1D convolutions on flat arrays (item i at offsets[i])."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    Ls = np.ascontiguousarray(lengths, dtype=np.int64)
    h = np.zeros_like(f)
    rc = _load().hd_batch_conv1d(len(Ls), _ptr(off), _ptr(Ls), _ptr(f), _ptr(g), _ptr(h),
                                 1 if use_fft else 0)
    if rc:
        raise ValueError(f"hd_batch_conv1d failed ({rc})")
    return h


def _multi(name, xs, K):
    xs = [np.ascontiguousarray(x, dtype=np.float64) for x in xs]
    if len(xs) < 2 or any(x.ndim != 1 for x in xs):
        raise ValueError("need n >= 2 one-dimensional arrays")
    L = np.array([len(x) for x in xs], dtype=np.int64)
    S = int(L.sum() - len(xs) + 1)
    K = int(L.max()) if K is None else int(K)
    ptrs = (ctypes.c_void_p * len(xs))(*[x.ctypes.data for x in xs])
    h = np.empty(K, dtype=np.float64)
    rc = getattr(_load(), name)(len(xs), _ptr(L), ptrs, K, _ptr(h))
    if rc:
        raise ValueError(f"{name} failed ({rc}); K must satisfy 1 <= K <= {S}")
    return h


def direct_conv_multi(xs, K=None):
    """O1m: x^1 * ... * x^n (1D, lengths may differ), first K outputs
    (default max L_i; K = sum L_i - n + 1 is the whole convolution), by
    direct FP64 summation one array after the other."""
    return _multi("hd_direct_conv_multi", xs, K)


def fft_conv_multi(xs, K=None):
    """O2m: the same through one zero-padded FP64 FFT of every array."""
    return _multi("hd_fft_conv_multi", xs, K)
