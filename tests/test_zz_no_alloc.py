"""The allocation-free hybridRCM entry point against the regular one.

hd_conv1d_rcm_noalloc serves callers that may not allocate device memory; it
keeps its scratch in a static device array.  Its output must match hd_conv1d
(hybridRCM) within the FP32 tolerance of the other tests, on two calls in a
row (the second call reuses the array the first one left behind).  This file
is collected last so that a first failure here comes after every other test.
"""
import numpy as np
import pytest

from paper_2608_14497_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    return m


def rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


@pytest.mark.parametrize("L,prm", [(1, None), (1000, None), (4096, None), (4096, [(512, 8)]), (70000, None),
                                   (200000, None), (33333, [(1000, 34)])])
def test_noalloc_matches_regular_entry_point(hd, L, prm):
    f, g = inputs.normal_pair(L, seed=900 + L)
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    ref = hd.conv(tf, tg, algo="hybridRCM", params=prm)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full_like(tf, float("nan"))
        st = hd.hd_conv1d_rcm_noalloc(tf.data_ptr(), tg.data_ptr(), out.data_ptr(), L, prm, stream)
        assert st == hd.HD_OK, hd.load().hd_strerror(st)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel(out, ref) <= TOL


def test_noalloc_rejects_beyond_limit(hd):
    x = torch.zeros(8, device="cuda")
    assert hd.hd_conv1d_rcm_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 524289, None, 0) == hd.HD_EUNSUPPORTED
    assert hd.hd_conv1d_rcm_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 0, None, 0) == hd.HD_EINVAL
