"""Split-precision path: radix-16 DFT passes of the 2D/3D hybridRCM kernels on
tensor cores with hi/lo bfloat16 operands and FP32 accumulation.  Bar:
relL2 <= 5e-5 against the FP64 oracle (the FP32 path's bar is 1e-5)."""
import numpy as np
import pytest

import oracle
from paper_2608_14497_b300 import inputs
from tests.conftest import record_rel, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL_SPLIT = 5e-5


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    return m


def run(hd, f, g, prec):
    tf = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    h = hd.conv(tf, tg, algo="hybridRCM", prec=prec)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.float64)


# (shape, whether some DFT length of the default plan (ladder lengths) is a multiple of 16, so a
# tensor-core pass runs)
@pytest.mark.parametrize("shape,tc", [((16, 16), True), ((64, 64), True), ((100, 37), True), ((256, 256), True),
                                      ((32, 32, 32), True), ((48, 40, 64), True), ((5, 6, 7), False)])
def test_split_precision_small(hd, shape, tc):
    f, g = inputs.normal_pair(shape, seed=80 + len(shape))
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    err = rel_l2(run(hd, f, g, "split_bf16"), ref)
    assert err <= TOL_SPLIT
    e32 = rel_l2(run(hd, f, g, "fp32"), ref)
    if tc:
        assert e32 < err  # the tensor-core passes ran (lower precision than FP32)
    else:
        assert e32 == err


def test_split_precision_3d_L256_every_output(hd):
    """Every output of 3D L = 256 (split precision) against O2."""
    f, g = inputs.normal_pair((256, 256, 256), seed=5)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    h = run(hd, f, g, "split_bf16")
    assert np.isfinite(h).all()
    err = record_rel("3D L=256 hybridRCM split_bf16", rel_l2(h, ref), TOL_SPLIT, h.size)
    assert err <= TOL_SPLIT


def test_split_precision_3d_L384_faces_and_points(hd):
    """3D L = 384 (split precision): every output on three face diagonals and
    2000 random points against direct FP64 sums."""
    L = 384
    f, g = inputs.normal_pair((L, L, L), seed=5)
    h = run(hd, f, g, "split_bf16")
    i = np.arange(L)
    z = np.zeros(L, dtype=np.int64)
    rng = np.random.default_rng(L)
    pts = np.concatenate([np.stack([z, i, i], 1), np.stack([i, z, i], 1),
                          np.stack([i, i, np.full(L, L - 1)], 1), rng.integers(0, L, (2000, 3))])
    ref = oracle.direct_conv_points(f.astype(np.float64), g.astype(np.float64), pts)
    got = h[tuple(pts.T)]
    err = record_rel("3D L=384 hybridRCM split_bf16 (faces + 2000 points)",
                     np.linalg.norm(got - ref) / np.linalg.norm(ref), TOL_SPLIT, len(pts))
    assert err <= TOL_SPLIT


def test_split_precision_other_algorithms_rejected(hd):
    f = torch.zeros((8, 8), device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.conv(f, f, algo="explicit", prec="split_bf16")
    assert e.value.status == hd.HD_EUNSUPPORTED


def test_split_fp16_declared_unsupported(hd):
    f = torch.zeros((8, 8), device="cuda")
    with pytest.raises(hd.HDError) as e:
        hd.conv(f, f, algo="hybridRCM", prec="split_fp16")
    assert e.value.status == hd.HD_EUNSUPPORTED
