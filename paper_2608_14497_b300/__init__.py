"""Python binding of libhdconv.so: hybrid-dealiased real convolutions on a B300.

The binding only marshals arguments: every step of a convolution runs in the
CUDA kernels of ``libhdconv.so`` (built in-tree by ``build.py``).  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the library
cannot be loaded, or no CUDA device is present, calls raise.

Low-level names mirror the C ABI of ``include/hdconv.h`` (``hd_conv1d`` ...),
taking raw device pointers; the ``conv1d`` / ``conv2d`` / ``conv3d`` /
``conv1d_batched`` helpers take torch CUDA tensors.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhdconv.so")

HD_OK, HD_EINVAL, HD_ENOMEM, HD_ECUDA, HD_ETIMEOUT, HD_EUNSUPPORTED = range(6)
HD_EXPLICIT, HD_EXPLICIT_RCM, HD_HYBRID_CS, HD_HYBRID_RCM, HD_HYBRID_CSRCM = range(5)
HD_FP32, HD_SPLIT_BF16, HD_SPLIT_FP16 = range(3)

ALGOS = {"explicit": HD_EXPLICIT, "explicitRCM": HD_EXPLICIT_RCM, "hybridCS": HD_HYBRID_CS,
         "hybridRCM": HD_HYBRID_RCM, "hybridCSRCM": HD_HYBRID_CSRCM}
PRECS = {"fp32": HD_FP32, "split_bf16": HD_SPLIT_BF16, "split_fp16": HD_SPLIT_FP16}

# Every symbol include/hdconv.h declares.
EXPORTS = ("hd_create", "hd_destroy", "hd_conv1d", "hd_conv2d", "hd_conv3d", "hd_batch_plan_create",
           "hd_batch_plan_destroy", "hd_conv1d_batched", "hd_conv_adjoint", "hd_plan", "hd_last_device_error",
           "hd_strerror", "hd_last_error_string", "hd_conv1d_rcm_noalloc",
           "hd_tuning_table", "hd_batch_plan_launches", "hd_conv_batch", "hd_conv_ext", "hd_conv1d_staged",
           "hd_conv1d_multi")


class HDError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.hd_last_error_string().decode() if _lib is not None else ""
        strerr = _lib.hd_strerror(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {strerr} ({status}) {msg}")


class DimParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("q", ctypes.c_int32)]


_lib = None


def load(build_if_missing=False):
    """Load libhdconv.so (optionally building it first); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhdconv.so not built ({LIB_PATH}); run paper_2608_14497_b300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    DP = ctypes.POINTER(DimParams)
    sig = {
        "hd_create": ([ctypes.POINTER(P), I], I),
        "hd_destroy": ([P], I),
        "hd_conv1d": ([P, I, I, P, P, P, I64, DP, P], I),
        "hd_conv2d": ([P, I, I, P, P, P, I64, I64, DP, P], I),
        "hd_conv3d": ([P, I, I, P, P, P, I64, I64, I64, DP, P], I),
        "hd_batch_plan_create": ([P, I, I32, P, P, ctypes.POINTER(P)], I),
        "hd_batch_plan_destroy": ([P], I),
        "hd_conv1d_batched": ([P, P, P, P, P, P], I),
        "hd_conv_adjoint": ([P, I, I, P, I32, P, P, P, P, P, P], I),
        "hd_plan": ([P, I, I64, DP], I),
        "hd_last_device_error": ([P], I),
        "hd_strerror": ([I], ctypes.c_char_p),
        "hd_last_error_string": ([], ctypes.c_char_p),
        "hd_conv1d_rcm_noalloc": ([P, P, P, I64, DP, P], I),
        "hd_tuning_table": ([P, I32, P, P, P, P], I),
        "hd_batch_plan_launches": ([P, P], I),
        "hd_conv_batch": ([P, I, I, I, P, I32, P, P, P, P], I),
        "hd_conv_ext": ([P, I, I, I, P, P, P, P, P, DP, P], I),
        "hd_conv1d_staged": ([P, I, I64, I64, I32, I32, I32, P, P, P, P], I),
        "hd_conv1d_multi": ([P, I32, P, P, I64, I32, I32, P, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status, where):
    if status != HD_OK:
        raise HDError(status, where)


# --- thin wrappers with the C names (raw pointers) -------------------------------
def hd_create(device=0):
    lib = load()
    ctx = ctypes.c_void_p()
    _check(lib.hd_create(ctypes.byref(ctx), device), "hd_create")
    return ctx


def hd_destroy(ctx):
    return load().hd_destroy(ctx)


def _params(prm, n):
    if prm is None:
        return None
    arr = (DimParams * n)()
    for i, (m, q) in enumerate(prm):
        arr[i].m, arr[i].q = int(m), int(q)
    return arr


def hd_conv1d(ctx, algo, prec, f_ptr, g_ptr, h_ptr, L, prm=None, stream=0):
    return load().hd_conv1d(ctx, algo, prec, f_ptr, g_ptr, h_ptr, L, _params(prm, 1), stream)


def hd_conv2d(ctx, algo, prec, f_ptr, g_ptr, h_ptr, L1, L2, prm=None, stream=0):
    return load().hd_conv2d(ctx, algo, prec, f_ptr, g_ptr, h_ptr, L1, L2, _params(prm, 2), stream)


def hd_conv3d(ctx, algo, prec, f_ptr, g_ptr, h_ptr, L1, L2, L3, prm=None, stream=0):
    return load().hd_conv3d(ctx, algo, prec, f_ptr, g_ptr, h_ptr, L1, L2, L3, _params(prm, 3), stream)


def hd_plan(ctx, algo, L):
    out = DimParams()
    _check(load().hd_plan(ctx, algo, L, ctypes.byref(out)), "hd_plan")
    return out.m, out.q


def hd_batch_plan_create(ctx, algo, offsets, lengths):
    import numpy as np
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    Ls = np.ascontiguousarray(lengths, dtype=np.int32)
    plan = ctypes.c_void_p()
    _check(load().hd_batch_plan_create(ctx, algo, len(Ls), off.ctypes.data, Ls.ctypes.data, ctypes.byref(plan)),
           "hd_batch_plan_create")
    return plan


def hd_batch_plan_destroy(plan):
    return load().hd_batch_plan_destroy(plan)


def hd_conv1d_batched(ctx, plan, f_ptr, g_ptr, h_ptr, stream=0):
    return load().hd_conv1d_batched(ctx, plan, f_ptr, g_ptr, h_ptr, stream)


def hd_conv_ext(ctx, algo, prec, Ls, Ks, f_ptr, g_ptr, h_ptr, prm=None, stream=0):
    n = len(Ls)
    la = (ctypes.c_int64 * n)(*[int(x) for x in Ls])
    ka = (ctypes.c_int64 * n)(*[int(x) for x in Ks]) if Ks is not None else None
    return load().hd_conv_ext(ctx, algo, prec, n, la, ka, f_ptr, g_ptr, h_ptr, _params(prm, n), stream)


def hd_conv_batch(ctx, algo, prec, Ls, batch, f_ptr, g_ptr, h_ptr, stream=0):
    arr = (ctypes.c_int64 * len(Ls))(*[int(x) for x in Ls])
    return load().hd_conv_batch(ctx, algo, prec, len(Ls), arr, batch, f_ptr, g_ptr, h_ptr, stream)


def hd_conv1d_staged(ctx, algo, L, K, M, q, batch, f_ptr, g_ptr, h_ptr, stream=0):
    return load().hd_conv1d_staged(ctx, algo, L, K, M, q, batch, f_ptr, g_ptr, h_ptr, stream)


def hd_conv1d_multi(ctx, x_ptrs, Ls, K, M, q, h_ptr, stream=0):
    n = len(x_ptrs)
    xa = (ctypes.c_void_p * n)(*x_ptrs)
    la = (ctypes.c_int64 * n)(*[int(v) for v in Ls])
    return load().hd_conv1d_multi(ctx, n, xa, la, K, M, q, h_ptr, stream)


def hd_conv_adjoint(ctx, algo, Ls, batch, gh_ptr, f_ptr, g_ptr, gf_ptr, gg_ptr, stream=0):
    arr = (ctypes.c_int64 * len(Ls))(*[int(x) for x in Ls])
    return load().hd_conv_adjoint(ctx, algo, len(Ls), arr, batch, gh_ptr, f_ptr, g_ptr, gf_ptr, gg_ptr, stream)


def hd_conv1d_rcm_noalloc(f_ptr, g_ptr, h_ptr, L, prm=None, stream=0):
    """hybridRCM 1D with no device allocation (scratch in a static device array)."""
    return load().hd_conv1d_rcm_noalloc(f_ptr, g_ptr, h_ptr, L, _params(prm, 1), stream)


def hd_tuning_table(ctx):
    """[(C, m, microseconds per convolution of length 2 C m)] of the autotuner."""
    import numpy as np
    n = ctypes.c_int32(0)
    _check(load().hd_tuning_table(ctx, 0, None, None, None, ctypes.byref(n)), "hd_tuning_table")
    C = np.zeros(max(1, n.value), np.int32)
    m = np.zeros(max(1, n.value), np.int32)
    us = np.zeros(max(1, n.value), np.float64)
    _check(load().hd_tuning_table(ctx, n.value, C.ctypes.data, m.ctypes.data, us.ctypes.data, ctypes.byref(n)),
           "hd_tuning_table")
    return [(int(C[i]), int(m[i]), float(us[i])) for i in range(n.value)]


def hd_last_device_error(ctx):
    return load().hd_last_device_error(ctx)


# --- torch helpers ---------------------------------------------------------------
_ctx = {}


def context(device=None):
    import torch
    dev = torch.cuda.current_device() if device is None else device
    if dev not in _ctx:
        _ctx[dev] = hd_create(dev)
    return _ctx[dev]


def _stream_ptr():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check_tensor(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")


def conv(f, g, algo="hybridRCM", params=None, out=None, prec="fp32", out_extent=None):
    """h = the linear convolution of f and g (1D/2D/3D), the first L outputs per
    dimension, or the first K with out_extent=K (L <= K <= 2L-1; "full" for 2L-1)."""
    import torch
    _check_tensor(f, "f")
    _check_tensor(g, "g")
    if f.shape != g.shape or f.dim() not in (1, 2, 3):
        raise ValueError("f and g must share a 1D/2D/3D shape")
    if out_extent is not None:
        K = tuple(2 * n - 1 for n in f.shape) if out_extent == "full" else tuple(int(k) for k in (
            out_extent if hasattr(out_extent, "__len__") else (out_extent,)))
        h = torch.empty(K, dtype=f.dtype, device=f.device) if out is None else out
        _check_tensor(h, "out")
        if tuple(h.shape) != K:
            raise ValueError("out must have the output extents")
        st = hd_conv_ext(context(f.device.index), ALGOS[algo], PRECS[prec], tuple(f.shape), K, f.data_ptr(),
                         g.data_ptr(), h.data_ptr(), params, _stream_ptr())
        _check(st, f"conv_ext[{algo}]")
        return h
    h = torch.empty_like(f) if out is None else out
    _check_tensor(h, "out")
    ctx = context(f.device.index)
    a, p = ALGOS[algo], PRECS[prec]
    if f.dim() == 1:
        st = hd_conv1d(ctx, a, p, f.data_ptr(), g.data_ptr(), h.data_ptr(), f.shape[0], params, _stream_ptr())
    elif f.dim() == 2:
        st = hd_conv2d(ctx, a, p, f.data_ptr(), g.data_ptr(), h.data_ptr(), *f.shape, params, _stream_ptr())
    else:
        st = hd_conv3d(ctx, a, p, f.data_ptr(), g.data_ptr(), h.data_ptr(), *f.shape, params, _stream_ptr())
    _check(st, f"conv{f.dim()}d[{algo}]")
    return h


def conv_batch(f, g, ndim, algo="hybridRCM", out=None):
    """Independent convolutions of f[b] with g[b] over a leading batch dimension
    (one hd_conv_batch call)."""
    import torch
    _check_tensor(f, "f")
    _check_tensor(g, "g")
    if f.shape != g.shape or f.dim() != ndim + 1:
        raise ValueError("f and g must be (batch, *extents) with matching shapes")
    h = torch.empty_like(f) if out is None else out
    _check_tensor(h, "out")
    ctx = context(f.device.index)
    st = hd_conv_batch(ctx, ALGOS[algo], HD_FP32, tuple(f.shape[1:]), f.shape[0], f.data_ptr(), g.data_ptr(),
                       h.data_ptr(), _stream_ptr())
    _check(st, "conv_batch")
    return h


def conv_staged(f, g, M=0, q=0, out_extent=None, out=None, algo="hybridRCM"):
    """hybridRCM or hybridCS in 1D through the three-kernel path
    (hd_conv1d_staged): f and g of shape (L,) or (batch, L); (M, q) = (0, 0)
    lets the planner choose."""
    import torch
    _check_tensor(f, "f")
    _check_tensor(g, "g")
    if f.shape != g.shape or f.dim() not in (1, 2):
        raise ValueError("f and g must share a (L,) or (batch, L) shape")
    L = f.shape[-1]
    batch = f.shape[0] if f.dim() == 2 else 1
    K = L if out_extent is None else (2 * L - 1 if out_extent == "full" else int(out_extent))
    shape = (K,) if f.dim() == 1 else (batch, K)
    h = torch.empty(shape, dtype=f.dtype, device=f.device) if out is None else out
    _check_tensor(h, "out")
    if tuple(h.shape) != shape:
        raise ValueError("out must have the output extents")
    st = hd_conv1d_staged(context(f.device.index), ALGOS[algo], L, K, M, q, batch, f.data_ptr(), g.data_ptr(),
                          h.data_ptr(), _stream_ptr())
    _check(st, "conv_staged")
    return h


def conv_multi(xs, out_extent=None, M=0, q=0, out=None):
    """x^1 * ... * x^n for 1D float32 CUDA tensors of possibly different
    lengths (hd_conv1d_multi); out_extent: K (default max L_i) or "full"."""
    import torch
    for i, x in enumerate(xs):
        _check_tensor(x, f"xs[{i}]")
        if x.dim() != 1:
            raise ValueError("conv_multi takes 1D tensors")
    Ls = [x.shape[0] for x in xs]
    S = sum(Ls) - len(Ls) + 1
    K = max(Ls) if out_extent is None else (S if out_extent == "full" else int(out_extent))
    h = torch.empty(K, dtype=torch.float32, device=xs[0].device) if out is None else out
    _check_tensor(h, "out")
    if tuple(h.shape) != (K,):
        raise ValueError("out must hold K floats")
    st = hd_conv1d_multi(context(xs[0].device.index), [x.data_ptr() for x in xs], Ls, K, M, q, h.data_ptr(),
                         _stream_ptr())
    _check(st, "conv_multi")
    return h


def adjoint(grad_h, f, g, algo="hybridRCM", need_f=True, need_g=True):
    """(grad_f, grad_g) of h = conv(f, g) for a batch (leading dimension)."""
    import torch
    for t, nme in ((grad_h, "grad_h"), (f, "f"), (g, "g")):
        _check_tensor(t, nme)
    gf = torch.empty_like(f) if need_f else None
    gg = torch.empty_like(g) if need_g else None
    ctx = context(f.device.index)
    Ls = tuple(f.shape[1:])
    st = hd_conv_adjoint(ctx, ALGOS[algo], Ls, f.shape[0], grad_h.data_ptr(), f.data_ptr(), g.data_ptr(),
                         gf.data_ptr() if gf is not None else None, gg.data_ptr() if gg is not None else None,
                         _stream_ptr())
    _check(st, "adjoint")
    return gf, gg


def _autograd_fn():
    import torch

    class HDConvFn(torch.autograd.Function):
        """h = conv(f, g) over a leading batch dimension; the backward pass runs
        the adjoint kernels (spectra are recomputed, nothing is stored)."""

        @staticmethod
        def forward(ctx, f, g, algo="hybridRCM"):
            f, g = f.contiguous(), g.contiguous()
            ctx.save_for_backward(f, g)
            ctx.algo = algo
            return conv_batch(f, g, f.dim() - 1, algo)

        @staticmethod
        def backward(ctx, grad_h):
            f, g = ctx.saved_tensors
            gf, gg = adjoint(grad_h.contiguous(), f, g, ctx.algo, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
            return gf, gg, None

    return HDConvFn


_HDConvFn = None


def hd_conv_fn(f, g, algo="hybridRCM"):
    """Differentiable batched convolution (torch.autograd.Function HDConvFn)."""
    global _HDConvFn
    if _HDConvFn is None:
        _HDConvFn = _autograd_fn()
    return _HDConvFn.apply(f, g, algo)


class BatchPlan:
    """Host-built plan of many 1D convolutions of uneven lengths on flat arrays
    (algo: hybridRCM, hybridCS, hybridCSRCM, or explicitRCM, the explicit-padding
    baseline)."""

    def __init__(self, offsets, lengths, algo="hybridRCM", device=None):
        self.ctx = context(device)
        self.algo = algo
        self.handle = hd_batch_plan_create(self.ctx, ALGOS[algo], offsets, lengths)

    def __call__(self, f, g, out=None):
        import torch
        _check_tensor(f, "f")
        _check_tensor(g, "g")
        h = torch.empty_like(f) if out is None else out
        _check(hd_conv1d_batched(self.ctx, self.handle, f.data_ptr(), g.data_ptr(), h.data_ptr(), _stream_ptr()),
               "conv1d_batched")
        return h

    @property
    def launches(self):
        """Kernel launches one call of the plan enqueues."""
        n = ctypes.c_int32(0)
        _check(load().hd_batch_plan_launches(self.handle, ctypes.byref(n)), "hd_batch_plan_launches")
        return n.value

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            hd_batch_plan_destroy(self.handle)
            self.handle = None
