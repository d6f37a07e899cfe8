"""GPU parity of the 2D/3D paths (recursive decomposition) and the explicit
baselines against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_14497_b300 import inputs
from tests.conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5
ALL = ("hybridRCM", "hybridCS", "explicit", "explicitRCM")


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    return m


def run(hd, f, g, algo, params=None):
    tf = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    h = hd.conv(tf, tg, algo=algo, params=params)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 7), (16, 16), (33, 17), (64, 64), (100, 37), (128, 128), (3, 200)])
def test_2d_small(hd, algo, shape):
    f, g = inputs.uniform_pair(shape, seed=sum(shape))
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (5, 6, 7), (8, 8, 8), (12, 10, 9), (16, 16, 16), (3, 20, 33)])
def test_3d_small(hd, algo, shape):
    f, g = inputs.normal_pair(shape, seed=sum(shape))
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL


@pytest.mark.parametrize("algo", ALL)
def test_2d_integer_exact(hd, algo):
    f, g = inputs.integer_pair((48, 40), seed=60)
    ref = oracle.direct_conv(f, g)
    h = run(hd, f, g, algo)
    assert np.array_equal(np.rint(h), ref)


@pytest.mark.parametrize("prm,algo", [
    ([(9, 2), (5, 2)], "hybridRCM"), ([(17, 1), (3, 4)], "hybridRCM"), ([(6, 3), (2, 5)], "hybridRCM"),
    ([(10, 2), (10, 2)], "hybridCS"), ([(6, 3), (7, 3)], "hybridCS"), ([(18, 1), (4, 5)], "hybridCS"),
])
def test_2d_explicit_parameters(hd, prm, algo):
    f, g = inputs.uniform_pair((9, 10), seed=61)
    ref = oracle.direct_conv(f, g)
    assert rel_l2(run(hd, f, g, algo, prm), ref) <= TOL


def sampled_check(hd, f, g, algo, npts, seed):
    h = run(hd, f, g, algo)
    rng = np.random.default_rng(seed)
    pts = np.stack([rng.integers(0, n, npts) for n in f.shape], axis=1)
    ref = oracle.direct_conv_points(f.astype(np.float64), g.astype(np.float64), pts)
    got = h[tuple(pts.T)]
    assert np.isfinite(h).all()
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("L", [1024, 2048, 3000])
def test_2d_full_size_sampled(hd, algo, L):
    f, g = inputs.uniform_pair((L, L), seed=4)
    assert sampled_check(hd, f, g, algo, 200, seed=L) <= TOL


@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("L", [256, 384])
def test_3d_full_size_sampled(hd, algo, L):
    f, g = inputs.normal_pair((L, L, L), seed=5)
    assert sampled_check(hd, f, g, algo, 60, seed=L) <= TOL


@pytest.mark.parametrize("algo", ALL)
def test_2d_in_place(hd, algo):
    f, g = inputs.uniform_pair((70, 90), seed=62)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    hd.conv(tf, tg, algo=algo, out=tf)
    torch.cuda.synchronize()
    assert rel_l2(tf.cpu().numpy(), ref) <= TOL


# Shapes whose default DFT lengths (ladder lengths) end in a composite pass:
# outer m = 160, 288, 1536 (radix 10, 18, 6), rows m = 96, 192, 320 (packed
# lengths 96, 191 and 320 for hybridRCM; radix 6, 12, 20), explicit 2 * ladder.
@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("shape", [(160, 192), (288, 381), (1500, 40), (100, 640)])
def test_2d_composite_last_pass(hd, algo, shape):
    f, g = inputs.uniform_pair(shape, seed=sum(shape))
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL
