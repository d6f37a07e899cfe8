"""The allocation-free hybridRCM entry point against the regular one.

hd_conv1d_rcm_noalloc serves callers that may not allocate device memory; it
keeps its scratch in a static device array.  Its output must match hd_conv1d
(hybridRCM) within the FP32 tolerance of the other tests, on two calls in a
row (the second call reuses the array the first one left behind).  This file
is collected last so that a first failure here comes after every other test.
"""
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
    if L >= 33333:
        # and directly against the FP64 oracle (O2)
        exact = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
        err = record_rel(f"noalloc 1D L={L} prm={prm}", rel_l2(out.cpu().numpy(), exact), TOL, L)
        assert err <= TOL


def test_noalloc_rejects_beyond_limit(hd):
    x = torch.zeros(8, device="cuda")
    assert hd.hd_conv1d_rcm_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 524289, None, 0) == hd.HD_EUNSUPPORTED
    assert b"524288" in hd.load().hd_last_error_string()
    assert hd.hd_conv1d_rcm_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 0, None, 0) == hd.HD_EINVAL
    # q m just above the table's 532480 entries
    assert hd.hd_conv1d_rcm_noalloc(x.data_ptr(), x.data_ptr(), x.data_ptr(), 4096, [(4096, 131)], 0) == \
        hd.HD_EUNSUPPORTED
    assert b"q m" in hd.load().hd_last_error_string()
