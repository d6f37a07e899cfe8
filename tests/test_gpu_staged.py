"""The three-kernel hybridRCM path (hd_conv1d_staged; the block sums of
Eq. forwardr and the accumulation of Eq. accumulation as q-point DFTs over the
blocks, App. A) against the FP64 oracle, element by element."""
import numpy as np
import pytest

import oracle
from paper_2608_14497_b300 import inputs
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


# (L, M, q): q = 2 (one CTA pair), q with radices 2/4/5 and 3, a prime radix
# (q = 14, 2 x 7), p < q/2 (many empty blocks), q = 1024, every stage-B
# length, ragged tails in both s and t; the q-point DFTs run on the
# plan-driven engine for q = 2, 4, 10, 12, 14, 30, 100, 150, on the compile-time
# one for q = 256, 512, 1024 and on the structured one for the rest.
CASES = [
    (1, 512, 2), (2, 512, 2), (777, 512, 2), (1000, 512, 4), (4097, 512, 10), (5000, 512, 14),
    (9000, 1024, 12), (9000, 1024, 30), (20001, 2048, 10), (40000, 4096, 10), (40000, 4608, 10),
    (70001, 512, 150), (3000, 512, 1024), (100000, 1024, 100), (123457, 2048, 64),
    # lengths of the structured engine ({1, 3, 5, 9} x 2^a >= 16)
    (9000, 512, 48), (60000, 512, 144), (100000, 1024, 160), (200000, 512, 768), (7000, 4608, 16),
    # the compile-time engine of stages A and C (q = 256, 512, 1024) with every
    # stage-B length behind it and few or many blocks (p from 30 to q/2): the
    # stage-B runtimes differ, so a load of w' that ran ahead of the wait for
    # stage B would show here
    (60000, 1024, 256), (200000, 1024, 256), (262144, 2048, 256), (300000, 4096, 256), (200000, 512, 512),
    (500000, 1024, 512), (500000, 512, 1024), (150000, 4608, 256),
]


@pytest.mark.parametrize("L,M,q", CASES)
@pytest.mark.parametrize("kind", ["L", "L+7", "full"])
def test_staged_parity(hd, L, M, q, kind):
    K = {"L": L, "L+7": min(2 * L - 1, L + 7), "full": 2 * L - 1}[kind]
    f, g = inputs.normal_pair(L, seed=3100 + L + q)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), (K,))
    h = host(hd.conv_staged(dev(f), dev(g), M=M, q=q, out_extent=K))
    assert h.shape == (K,)
    assert rel_l2(h, ref) <= TOL, (L, M, q, K)


@pytest.mark.parametrize("L", [1 << 18, 500000, 1000000])
def test_staged_full_size(hd, L):
    """The sizes beyond the cluster kernel through the public call (the planner
    picks the three-kernel path), every output compared."""
    ctx = hd.context()
    M, q = hd.hd_plan(ctx, hd.HD_HYBRID_RCM, L)
    assert M * q >= L and q % 2 == 0 and M in (512, 1024, 2048, 4096, 4608)
    f, g = inputs.uniform_pair(L, seed=3200 + L % 1000)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    h = host(hd.conv(dev(f), dev(g), algo="hybridRCM"))
    err = rel_l2(h, ref)
    record_rel(f"1D L={L} hybridRCM three-kernel path (M={M}, q={q})", err, TOL, L)
    assert err <= TOL


def test_staged_full_output_1e6(hd):
    L = 1000000
    f, g = inputs.normal_pair(L, seed=3300)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), (2 * L - 1,))
    h = host(hd.conv(dev(f), dev(g), algo="hybridRCM", out_extent="full"))
    err = rel_l2(h, ref)
    record_rel("1D L=1000000 full output, three-kernel path", err, TOL, 2 * L - 1)
    assert err <= TOL


def test_staged_integer_exact(hd):
    """Small integers: every output of the truncated convolution is an integer
    well inside FP32's exact range, so rounding the result recovers it."""
    L = 100000
    rng = np.random.default_rng(3400)
    f = rng.integers(-3, 4, L).astype(np.float64)
    g = rng.integers(-3, 4, L).astype(np.float64)
    pts = np.unique(np.concatenate([np.arange(64), rng.integers(0, L, 256), np.arange(L - 64, L)]))
    ref = oracle.direct_conv_points(f, g, pts[:, None])
    h = host(hd.conv(dev(f), dev(g), algo="hybridRCM"))
    assert np.array_equal(np.rint(h[pts]), ref)
    assert np.abs(h[pts] - ref).max() < 0.25


def test_staged_batch(hd):
    L, B = 90000, 3
    fs, gs = zip(*(inputs.uniform_pair(L, seed=3500 + b) for b in range(B)))
    f, g = np.stack(fs), np.stack(gs)
    h = host(hd.conv_batch(dev(f), dev(g), 1, algo="hybridRCM"))
    hs = host(hd.conv_staged(dev(f), dev(g), M=1024, q=90, out_extent="full"))
    for b in range(B):
        ref = oracle.fft_conv(f[b].astype(np.float64), g[b].astype(np.float64), (2 * L - 1,))
        assert rel_l2(h[b], ref[:L]) <= TOL
        assert rel_l2(hs[b], ref) <= TOL


def test_staged_in_place(hd):
    L = 80000
    f, g = inputs.uniform_pair(L, seed=3600)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    tf, tg = dev(f), dev(g)
    hd.conv(tf, tg, algo="hybridRCM", out=tf)
    assert rel_l2(host(tf), ref) <= TOL


def test_staged_argument_errors(hd):
    f, g = dev(np.ones(5000)), dev(np.ones(5000))
    for M, q in ((300, 10), (512, 9), (512, 2), (512, 0), (0, 10), (512, 1026)):
        with pytest.raises(hd.HDError) as e:
            hd.conv_staged(f, g, M=M, q=q)
        assert e.value.status == hd.HD_EINVAL, (M, q)
    # a longer output may not overlap the inputs
    L = 5000
    buf = dev(np.ones(4 * L))
    with pytest.raises(hd.HDError) as e:
        hd.conv_staged(buf[:L], g, M=512, q=10, out=buf[L // 2:L // 2 + 2 * L - 1], out_extent="full")
    assert e.value.status == hd.HD_EINVAL


# --- hybridCS on the three kernels (App. A's inner loop for real data) -------------
CS_CASES = [(1, 512, 2), (777, 512, 4), (4097, 512, 18), (5000, 512, 20), (9000, 1024, 18), (20001, 2048, 20),
            (40000, 4608, 18), (100000, 1024, 256), (3000, 512, 1024),
            (60000, 1024, 256), (262144, 2048, 256), (300000, 4096, 256), (100000, 512, 512), (200000, 512, 1024)]


@pytest.mark.parametrize("L,M,q", CS_CASES)
@pytest.mark.parametrize("kind", ["L", "full"])
def test_staged_cs_parity(hd, L, M, q, kind):
    K = L if kind == "L" else 2 * L - 1
    f, g = inputs.normal_pair(L, seed=3700 + L + q)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), (K,))
    h = host(hd.conv_staged(dev(f), dev(g), M=M, q=q, out_extent=K, algo="hybridCS"))
    assert rel_l2(h, ref) <= TOL, (L, M, q, K)


@pytest.mark.parametrize("L", [9000, 1 << 18, 1000000])
def test_staged_cs_full_size(hd, L):
    """hybridCS beyond one CTA (L > 8192) through the public call."""
    M, q = hd.hd_plan(hd.context(), hd.HD_HYBRID_CS, L)
    assert M * q >= 2 * L - 1 and M in (512, 1024, 2048, 4096, 4608)
    f, g = inputs.uniform_pair(L, seed=3800 + L % 1000)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    h = host(hd.conv(dev(f), dev(g), algo="hybridCS"))
    err = rel_l2(h, ref)
    if L >= 1 << 18:
        record_rel(f"1D L={L} hybridCS three-kernel path (M={M}, q={q})", err, TOL, L)
    assert err <= TOL


def test_staged_cs_batch_and_errors(hd):
    L, B = 30000, 3
    fs, gs = zip(*(inputs.uniform_pair(L, seed=3900 + b) for b in range(B)))
    f, g = np.stack(fs), np.stack(gs)
    h = host(hd.conv_batch(dev(f), dev(g), 1, algo="hybridCS"))
    for b in range(B):
        ref = oracle.fft_conv(f[b].astype(np.float64), g[b].astype(np.float64))
        assert rel_l2(h[b], ref) <= TOL
    x = dev(np.ones(5000))
    with pytest.raises(hd.HDError) as e:
        hd.conv_staged(x, x, M=512, q=18, algo="hybridCS")  # 9216 < 2L - 1
    assert e.value.status == hd.HD_EINVAL
    with pytest.raises(hd.HDError) as e:
        hd.conv_staged(x, x, M=512, q=20, algo="explicit")
    assert e.value.status == hd.HD_EINVAL


@pytest.mark.parametrize("L", [512, 513, 1000, 2048, 2049, 4096, 6000, 8192, 8193])
@pytest.mark.parametrize("kind", ["L", "full"])
def test_single_cs_call_short_lengths(hd, L, kind):
    """Single hybridCS calls from L = 513 on take the three kernels (q = 4 and
    the smallest M >= (2L - 1) / 4 up to L = 8192); L = 512 stays on one CTA."""
    M, q = hd.hd_plan(hd.context(), hd.HD_HYBRID_CS, L)
    if L > 512:
        assert M * q >= 2 * L - 1 and M in (512, 1024, 2048, 4096, 4608)
        if L <= 8192:
            assert q == 4
    K = L if kind == "L" else 2 * L - 1
    f, g = inputs.normal_pair(L, seed=7300 + L)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), (K,))
    h = host(hd.conv(dev(f), dev(g), algo="hybridCS", out_extent=K))
    assert rel_l2(h, ref) <= TOL, (L, K)


def test_single_cs_call_in_place(hd):
    L = 4096
    f, g = inputs.uniform_pair(L, seed=7400)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    tf, tg = dev(f), dev(g)
    hd.conv(tf, tg, algo="hybridCS", out=tf)
    assert rel_l2(host(tf), ref) <= TOL
