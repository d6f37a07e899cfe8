"""Convolutions of n >= 2 arrays of possibly different lengths (hd_conv1d_multi:
Sec. 4.1's implicitly packed convolution of more than two arrays, Eqs. Akn,
Rnk and RnMk; Sec. 7's arrays of different sizes with a shared (m, q)) against
the FP64 oracle O2m, element by element."""
import numpy as np
import pytest

import oracle
from tests.conftest import record_rel, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


def arrays(lengths, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1, 1, L).astype(np.float32) for L in lengths]


# a long signal with a short kernel (the CNN case of Sec. 7), the reverse
# order, equal lengths, length-1 arrays, and long/long pairs
PAIRS = [(4096, 64), (64, 4096), (37, 5), (1, 1), (1, 300), (100000, 1000), (1000000, 4096), (250000, 250000),
         (70000, 3)]


@pytest.mark.parametrize("Lf,Lg", PAIRS)
@pytest.mark.parametrize("kind", ["max", "full"])
def test_two_arrays_unequal(hd, Lf, Lg, kind):
    xs = arrays((Lf, Lg), seed=4000 + Lf + 7 * Lg)
    S = Lf + Lg - 1
    K = S if kind == "full" else max(Lf, Lg)
    ref = oracle.fft_conv_multi([x.astype(np.float64) for x in xs], K)
    h = host(hd.conv_multi([dev(x) for x in xs], out_extent=K))
    err = rel_l2(h, ref)
    if Lf * Lg >= 10 ** 8:
        record_rel(f"1D unequal lengths {Lf} * {Lg}, K={K}", err, TOL, K)
    assert h.shape == (K,)
    assert err <= TOL, (Lf, Lg, K)


@pytest.mark.parametrize("lengths", [(300, 200, 250), (4096, 4096, 4096), (5000, 17, 900, 3), (1000,) * 8,
                                     (64,) * 16, (200000, 1000, 50)])
def test_n_arrays(hd, lengths):
    """The whole convolution within 1e-5 relL2.  A truncated output is held to
    1e-5 of the whole result's norm: the rounding of the transforms spreads
    over every output, and with many arrays the first K outputs can be orders
    of magnitude smaller than the peak of the convolution (for eight uniform
    arrays of 1000 the first 1000 outputs hold ~1e-3 of its norm)."""
    xs = arrays(lengths, seed=4100 + sum(lengths))
    S = sum(lengths) - len(lengths) + 1
    full = oracle.fft_conv_multi([x.astype(np.float64) for x in xs], S)
    nrm = np.linalg.norm(full)
    for K in (max(lengths), S):
        h = host(hd.conv_multi([dev(x) for x in xs], out_extent=K))
        assert np.linalg.norm(h - full[:K]) <= TOL * nrm, (lengths, K)
    assert rel_l2(h, full) <= TOL


def _geometric3(hd, a, b, c):
    L = (3000, 2000, 2500)
    xs = [(r ** np.arange(n, dtype=np.float64)).astype(np.float32) for r, n in zip((a, b, c), L)]
    k = np.arange(2000, dtype=np.float64)
    ref = (a ** (k + 2) / ((a - b) * (a - c)) + b ** (k + 2) / ((b - a) * (b - c)) +
           c ** (k + 2) / ((c - a) * (c - b)))
    h = host(hd.conv_multi([dev(x) for x in xs], out_extent=2000))
    kap = np.prod([np.linalg.norm(x.astype(np.float64)) for x in xs]) / np.linalg.norm(ref)
    return rel_l2(h, ref), kap


def test_three_geometric_closed_form(hd):
    """Positive ratios (no cancellation): the partial-fraction closed form of
    the three-array convolution within 1e-5."""
    err, _ = _geometric3(hd, 0.9995, 0.999, 0.5)
    assert err <= TOL


def test_three_geometric_alternating(hd):
    """b = -0.999: the spectra of the first two arrays peak at opposite ends,
    so the product cancels (kappa = prod ||x_i|| / ||h|| ~ 26); the bound is
    the FP32 FFT-convolution bound scaled by kappa, as for two arrays."""
    err, kap = _geometric3(hd, 0.9995, -0.999, 0.5)
    assert err <= 18 * np.log2(8192) * np.finfo(np.float32).eps * kap


@pytest.mark.parametrize("M,q", [(512, 2), (512, 10), (1024, 16), (2048, 64), (4608, 18), (512, 256), (1024, 512),
                                 (512, 1024), (4096, 256)])
def test_explicit_parameters(hd, M, q):
    lengths = (6000, 300, 77)
    S = sum(lengths) - 2
    if 2 * M * q < S:
        pytest.skip("does not dealias")
    xs = arrays(lengths, seed=4200 + M + q)
    ref = oracle.fft_conv_multi([x.astype(np.float64) for x in xs], S)
    h = host(hd.conv_multi([dev(x) for x in xs], out_extent="full", M=M, q=q))
    assert rel_l2(h, ref) <= TOL


@pytest.mark.parametrize("M,q", [(2048, 256), (1024, 512), (512, 1024)])
def test_long_arrays_compile_time_engine(hd, M, q):
    """Three long arrays (many blocks of each) through stages A and C on the
    compile-time engine, with the n-ary product in stage B."""
    lengths = (300000, 100000, 5)
    S = sum(lengths) - 2
    xs = arrays(lengths, seed=4300 + q)
    ref = oracle.fft_conv_multi([x.astype(np.float64) for x in xs], S)
    h = host(hd.conv_multi([dev(x) for x in xs], out_extent="full", M=M, q=q))
    assert rel_l2(h, ref) <= TOL


def test_equal_pair_matches_binary_path(hd):
    """n = 2 with equal lengths is the ordinary convolution."""
    xs = arrays((90000, 90000), seed=4300)
    a = host(hd.conv_multi([dev(x) for x in xs]))
    b = host(hd.conv(dev(xs[0]), dev(xs[1])))
    ref = oracle.fft_conv_multi([x.astype(np.float64) for x in xs], 90000)
    assert rel_l2(a, ref) <= TOL and rel_l2(b, ref) <= TOL


def test_output_may_alias_an_input(hd):
    xs = arrays((5000, 100), seed=4400)
    ref = oracle.fft_conv_multi([x.astype(np.float64) for x in xs], 5000)
    t0, t1 = dev(xs[0]), dev(xs[1])
    hd.conv_multi([t0, t1], out=t0)
    assert rel_l2(host(t0), ref) <= TOL


def test_argument_errors(hd):
    a, b = dev(np.ones(100)), dev(np.ones(10))
    for kw in (dict(out_extent=110), dict(M=300, q=2), dict(M=512, q=0), dict(M=512, q=3)):
        with pytest.raises(hd.HDError) as e:
            hd.conv_multi([a, b], **kw)
        assert e.value.status == hd.HD_EINVAL, kw
    with pytest.raises(hd.HDError) as e:
        hd.conv_multi([a])
    assert e.value.status == hd.HD_EINVAL
    with pytest.raises(hd.HDError) as e:
        hd.conv_multi([b] * 17)
    assert e.value.status == hd.HD_EINVAL
