"""hd_conv_batch: a batch of equal-size 1D/2D/3D convolutions in one call
(hybridRCM: one pass sequence over every item) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_14497_b300 import inputs
from tests.conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    return m


@pytest.mark.parametrize("algo", ["hybridRCM", "hybridCS", "explicitRCM", "explicit"])
@pytest.mark.parametrize("shape", [(1000,), (4096,), (30001,), (70000,), (17, 33), (64, 64), (100, 37),
                                   (5, 6, 7), (12, 10, 9)])
def test_batch_every_item(hd, algo, shape):
    B = 5
    f, g = inputs.normal_pair((B,) + shape, seed=sum(shape) + 7)
    if algo.startswith("explicit") and len(shape) == 1 and shape[0] > 8192:
        pytest.skip("explicit 1D baselines transform the padded row in one CTA (L <= 8192)")
    h = hd.conv_batch(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), len(shape), algo=algo)
    torch.cuda.synchronize()
    hh = h.cpu().numpy()
    for b in range(B):
        ref = oracle.fft_conv(f[b].astype(np.float64), g[b].astype(np.float64))
        assert rel_l2(hh[b], ref) <= TOL, (algo, shape, b)


def test_batch_matches_single_calls_bitwise_1d(hd):
    """A batch whose clusters fit in one wave takes the single-call (C, m), so
    one cluster launch over the batch gives the single-call result per item."""
    B, L = 7, 20000
    f, g = inputs.uniform_pair((B, L), seed=91)
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    hb = hd.conv_batch(tf, tg, 1)
    for b in range(B):
        hs = hd.conv(tf[b].contiguous(), tg[b].contiguous())
        assert torch.equal(hb[b], hs)


@pytest.mark.parametrize("L,B", [(1, 3), (100, 40), (1000, 64), (4096, 33), (8192, 9)])
def test_cs_batch_three_kernels(hd, L, B):
    """A hybridCS batch of short lengths on the three kernels: every item."""
    f, g = inputs.normal_pair((B, L), seed=7500 + L)
    h = hd.conv_batch(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), 1, algo="hybridCS")
    torch.cuda.synchronize()
    hh = h.cpu().numpy()
    for b in range(B):
        ref = oracle.fft_conv(f[b].astype(np.float64), g[b].astype(np.float64))
        assert rel_l2(hh[b], ref) <= TOL, (L, b)
