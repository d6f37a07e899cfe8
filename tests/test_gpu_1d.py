"""GPU parity of the 1D paths against the FP64 oracle (relL2 <= 1e-5, FP32)."""
import numpy as np
import pytest

import oracle
from oracle import steps
from paper_2608_14497_b300 import inputs
from tests.conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
HYBRID = ("hybridRCM", "hybridCS")
ALL = ("hybridRCM", "hybridCS", "explicit", "explicitRCM")


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    assert torch.cuda.is_available()
    return m


def run(hd, f, g, algo, params=None):
    tf = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    h = hd.conv(tf, tg, algo=algo, params=params)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("algo", ALL)
def test_L4096_uniform(hd, algo):
    f, g = inputs.uniform_pair(4096, seed=1)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL


@pytest.mark.parametrize("algo", ALL)
def test_L4096_integer_exact(hd, algo):
    f, g = inputs.integer_pair(4096, seed=7)
    ref = oracle.direct_conv(f, g)
    h = run(hd, f, g, algo)
    assert np.abs(h - ref).max() < 0.5
    assert np.array_equal(np.rint(h), ref)


def kappa(f, g, h):
    """Normwise condition number of the convolution, ||f|| ||g|| / ||h||."""
    return np.linalg.norm(f) * np.linalg.norm(g) / np.linalg.norm(h)


def fp32_fft_conv_bound(N, kap):
    """Normwise bound for an FP32 FFT convolution: three transforms of log2 N
    radix-2-equivalent stages, each adding at most about 6 units of roundoff
    (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 24.1), scaled
    by the conditioning ||f|| ||g|| / ||h||."""
    return 18 * np.log2(N) * np.finfo(np.float32).eps * kap


@pytest.mark.parametrize("algo", ALL)
def test_L4096_geometric_closed_form(hd, algo):
    """Positive ratios: no cancellation, the FP32 result meets 1e-5."""
    a, b = 0.9995, 0.999
    f, g = inputs.geometric_pair(4096, a, b)
    k = np.arange(4096, dtype=np.float64)
    ref = (a ** (k + 1) - b ** (k + 1)) / (a - b)
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL


@pytest.mark.parametrize("algo", ALL)
def test_L4096_geometric_alternating(hd, algo):
    """a = 0.9995, b = -0.999: heavy cancellation (kappa ~ 43), so the bound
    is the FP32 FFT-convolution bound scaled by kappa, not 1e-5."""
    a, b = 0.9995, -0.999
    f, g = inputs.geometric_pair(4096, a, b)
    k = np.arange(4096, dtype=np.float64)
    ref = (a ** (k + 1) - b ** (k + 1)) / (a - b)
    err = rel_l2(run(hd, f, g, algo), ref)
    assert err <= fp32_fft_conv_bound(2 * 4096, kappa(f, g, ref))


def ladder_ceil(n):
    """Smallest {1, 3, 5, 9} * 2^a >= n: the explicit baselines' DFT length."""
    best = None
    for base in (1, 3, 5, 9):
        x = base
        while x < n:
            x *= 2
        best = x if best is None else min(best, x)
    return best


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("L", [1, 2, 3, 5, 17, 100, 127, 1000, 3001, 5000, 8192, 12345, 20000, 70000])
def test_ragged_lengths_default_plan(hd, algo, L):
    f, g = inputs.uniform_pair(L, seed=L)
    if algo == "explicit" and ladder_ceil(L) > 16384:
        # the r2c explicit baseline transforms the padded row in one CTA
        with pytest.raises(hd.HDError) as e:
            run(hd, f, g, algo)
        assert e.value.status == hd.HD_EUNSUPPORTED
        return
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL


@pytest.mark.parametrize("L", list(range(1, 17)))
def test_brute_force_every_valid_m_q(hd, L):
    f, g = inputs.uniform_pair(L, seed=200 + L)
    ref = oracle.direct_conv(f, g)
    for m in range(1, 2 * L + 1):
        for q in (-(-(2 * L - 1) // m), -(-(2 * L - 1) // m) + 1):
            if steps.cs_valid(L, m, q):
                assert rel_l2(run(hd, f, g, "hybridCS", [(m, q)]), ref) <= TOL, (L, m, q)
        for q in (-(-L // m), -(-L // m) + 1):
            if steps.rcm_valid(L, m, q):
                assert rel_l2(run(hd, f, g, "hybridRCM", [(m, q)]), ref) <= TOL, (L, m, q)


@pytest.mark.parametrize("L,m,q,algo", [
    (5000, 512, 10, "hybridRCM"), (5000, 700, 8, "hybridRCM"), (5000, 625, 9, "hybridRCM"),
    (4999, 1000, 10, "hybridCS"), (4999, 1001, 11, "hybridCS"), (5000, 768, 14, "hybridCS"),
    (70000, 4096, 18, "hybridRCM"), (70000, 8000, 18, "hybridCS"), (4096, 7 * 11 * 13, 5, "hybridRCM"),
])
def test_explicit_parameters_p_gt_1(hd, L, m, q, algo):
    f, g = inputs.normal_pair(L, seed=300)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo, [(m, q)]), ref) <= TOL


@pytest.mark.parametrize("L", [4096, 9000, 17777, 20000, 40001, 65536, 70000, 73728])
def test_cluster_path_sizes(hd, L):
    """Lengths that exercise clusters of 1, 2, 4 and 8 CTAs (planner choice)."""
    f, g = inputs.normal_pair(L, seed=500 + L)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, "hybridRCM"), ref) <= TOL


@pytest.mark.parametrize("algo", ALL)
def test_in_place(hd, algo):
    f, g = inputs.uniform_pair(3000, seed=9)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    tf = torch.from_numpy(f).cuda()
    tg = torch.from_numpy(g).cuda()
    hd.conv(tf, tg, algo=algo, out=tf)
    torch.cuda.synchronize()
    assert rel_l2(tf.cpu().numpy(), ref) <= TOL


def test_invalid_parameters_rejected(hd):
    f = torch.zeros(100, device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.conv(f, f, algo="hybridRCM", params=[(10, 5)])  # qm = 50 < L
    assert e.value.status == hd.HD_EINVAL
    with pytest.raises(hd.HDError) as e:
        hd.conv(f, f, algo="hybridCS", params=[(101, 2)])  # q even, m odd
    assert e.value.status == hd.HD_EINVAL
    with pytest.raises(hd.HDError) as e:
        hd.conv(f, f, algo="hybridCS", params=[(50, 3)])  # qm = 150 < 2L-1
    assert e.value.status == hd.HD_EINVAL


# DFT lengths whose last pass is a composite butterfly (leftover power of two
# times the odd factor: radix 6, 10, 12, 18, 20, 24): m in {96, 160, 192, 288,
# 320, 384, 1536, 2560, 3072, 4608}.  The single-call plan takes the smallest
# cluster whose largest length suffices (C = 1 up to L = 9216) and the smallest
# ladder length m with 2 m >= L, so L = 2m and L = 2m - 5 land on these m.
@pytest.mark.parametrize("m", [96, 160, 192, 288, 320, 384, 1536, 2560, 3072, 4608])
@pytest.mark.parametrize("delta", [0, 5])
def test_composite_last_pass_lengths(hd, m, delta):
    L = 2 * m - delta
    f, g = inputs.uniform_pair(L, seed=500 + m + delta)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, "hybridRCM"), ref) <= TOL


@pytest.mark.parametrize("L", [9000, 20001, 40000, 65536, 70000, 73728])
def test_explicit_rcm_long_lengths(hd, L):
    """explicitRCM beyond one CTA: zero-padded copies on the cluster kernel."""
    f, g = inputs.normal_pair(L, seed=700 + L)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, "explicitRCM"), ref) <= TOL


# single calls pick the cluster size by a latency model: every size it can
# choose (one CTA up to clusters of 16), first L and full outputs
@pytest.mark.parametrize("L", [4096, 4097, 8192, 9000, 16384, 20000, 32768, 40000, 65536, 73728])
@pytest.mark.parametrize("full", [False, True])
def test_single_call_cluster_choice(hd, L, full):
    ctx = hd.context()
    m, q = hd.hd_plan(ctx, hd.HD_HYBRID_RCM, L)
    assert q in (2, 4, 8, 16, 32) and m % 256 == 0 and m * q >= L
    f, g = inputs.normal_pair(L, seed=7200 + L)
    K = 2 * L - 1 if full else L
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), (K,))
    tf = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    h = hd.conv(tf, tg, algo="hybridRCM", out_extent="full" if full else None)
    torch.cuda.synchronize()
    assert rel_l2(h.cpu().numpy().astype(np.float64), ref) <= TOL, (L, m, q)
