"""Output extents K (L <= K <= 2L-1 per dimension; K = 2L-1 the full linear
convolution) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import steps
from paper_2608_14497_b300 import inputs
from tests.conftest import record_rel, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5
ALL = ("hybridRCM", "hybridCS", "explicit", "explicitRCM")


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    return m


def run(hd, f, g, algo, K, params=None):
    tf = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    h = hd.conv(tf, tg, algo=algo, params=params, out_extent=K)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("L", [1, 2, 3, 17, 1000, 4096, 9000, 20001, 70000])
@pytest.mark.parametrize("full", [True, False])
def test_1d_output_extent(hd, algo, L, full):
    K = 2 * L - 1 if full else min(2 * L - 1, L + 7)
    if algo == "explicit" and L > 8192:
        pytest.skip("the r2c explicit baseline transforms the padded row in one CTA (L <= 8192)")
    f, g = inputs.normal_pair(L, seed=1100 + L)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), (K,))
    err = rel_l2(run(hd, f, g, algo, K), ref)
    if full and L >= 4096:
        record_rel(f"1D L={L} full output {algo}", err, TOL, K)
    assert err <= TOL


@pytest.mark.parametrize("L", list(range(1, 17)))
def test_brute_force_full_output(hd, L):
    """Every valid (m, q) for L <= 16 with the full 2L-1 outputs."""
    f, g = inputs.uniform_pair(L, seed=1200 + L)
    K = 2 * L - 1
    ref = oracle.direct_conv(f, g, (K,))
    for m in range(1, 2 * L + 1):
        for q in (-(-(2 * L - 1) // m), -(-(2 * L - 1) // m) + 1):
            if steps.cs_valid(L, m, q):
                assert rel_l2(run(hd, f, g, "hybridCS", K, [(m, q)]), ref) <= TOL, (L, m, q)
        for q in (-(-L // m), -(-L // m) + 1):
            if steps.rcm_valid(L, m, q):
                assert rel_l2(run(hd, f, g, "hybridRCM", K, [(m, q)]), ref) <= TOL, (L, m, q)


@pytest.mark.parametrize("algo", ["hybridRCM", "explicit", "explicitRCM"])
@pytest.mark.parametrize("shape", [(1, 1), (5, 7), (33, 17), (64, 64), (100, 37), (3, 200), (300, 260)])
def test_2d_full_output(hd, algo, shape):
    f, g = inputs.uniform_pair(shape, seed=sum(shape) + 13)
    K = tuple(2 * n - 1 for n in shape)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), K)
    assert rel_l2(run(hd, f, g, algo, K), ref) <= TOL


@pytest.mark.parametrize("algo", ["hybridRCM", "explicit", "explicitRCM"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (12, 10, 9), (16, 16, 16), (40, 33, 130)])
def test_3d_full_output(hd, algo, shape):
    f, g = inputs.normal_pair(shape, seed=sum(shape) + 17)
    K = tuple(2 * n - 1 for n in shape)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), K)
    assert rel_l2(run(hd, f, g, algo, K), ref) <= TOL


@pytest.mark.parametrize("algo", ["hybridRCM", "explicitRCM"])
def test_2d_full_output_L1024(hd, algo):
    """The 2D config's smallest size with the full (2L-1)^2 output, every output against O2."""
    L = 1024
    f, g = inputs.uniform_pair((L, L), seed=4)
    K = (2 * L - 1, 2 * L - 1)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), K)
    err = record_rel(f"2D L={L} full output {algo}", rel_l2(run(hd, f, g, algo, K), ref), TOL, K[0] * K[1])
    assert err <= TOL


def test_mixed_extents(hd):
    f, g = inputs.uniform_pair((21, 30, 45), seed=5)
    K = (21, 50, 89)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), K)
    assert rel_l2(run(hd, f, g, "hybridRCM", K), ref) <= TOL


def test_output_extent_errors(hd):
    x = torch.zeros(64, device="cuda")
    y = torch.zeros(127, device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.conv(x, x, out_extent=128, out=torch.zeros(128, device="cuda"))  # K > 2L-1
    assert e.value.status == hd.HD_EINVAL
    with pytest.raises(hd.HDError) as e:
        hd.conv(x, x, out_extent=63, out=torch.zeros(63, device="cuda"))  # K < L
    assert e.value.status == hd.HD_EINVAL
    # a longer output may not alias an input
    st = hd.hd_conv_ext(hd.context(), hd.HD_HYBRID_RCM, hd.HD_FP32, (64,), (127,), y.data_ptr(), x.data_ptr(),
                        y.data_ptr(), None, 0)
    assert st == hd.HD_EINVAL
    f2 = torch.zeros((8, 8), device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.conv(f2, f2, algo="hybridCS", out_extent="full")
    assert e.value.status == hd.HD_EUNSUPPORTED
