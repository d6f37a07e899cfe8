"""Seeded synthetic inputs shaped like the paper's benchmark workloads.

Shared by the tests and the benchmark; holds none of the method's arithmetic.
Values are drawn in FP64 with numpy.random.default_rng(seed) (f first, then g)
and cast to FP32.
"""
import numpy as np


def uniform_pair(shape, seed):
    """f, g i.i.d. uniform in [-1, 1)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1.0, 1.0, shape).astype(np.float32)
    g = rng.uniform(-1.0, 1.0, shape).astype(np.float32)
    return f, g


def normal_pair(shape, seed):
    """f, g i.i.d. standard normal."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(shape).astype(np.float32)
    g = rng.standard_normal(shape).astype(np.float32)
    return f, g


def integer_pair(shape, seed, lo=-8, hi=8):
    """f, g i.i.d. integers in [lo, hi] (exactly representable)."""
    rng = np.random.default_rng(seed)
    f = rng.integers(lo, hi + 1, shape).astype(np.float32)
    g = rng.integers(lo, hi + 1, shape).astype(np.float32)
    return f, g


def geometric_pair(L, a=0.9995, b=-0.999):
    """f_j = a^j, g_j = b^j (FP64 values; cast by the caller)."""
    j = np.arange(L, dtype=np.float64)
    return a ** j, b ** j


def batch_lengths(n=4096, lo=500, hi=70000, seed=2):
    """n lengths uniform on {lo..hi} and the flat offsets of the items."""
    rng = np.random.default_rng(seed)
    Ls = rng.integers(lo, hi + 1, n).astype(np.int64)
    off = np.zeros(n, dtype=np.int64)
    off[1:] = np.cumsum(Ls)[:-1]
    return off, Ls


def batch_values(total, seed=3):
    """Flat f and g of `total` standard-normal values each."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(total).astype(np.float32)
    g = rng.standard_normal(total).astype(np.float32)
    return f, g
