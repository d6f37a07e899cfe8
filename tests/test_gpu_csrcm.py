"""The combined CS+RCM algorithm (hybridCSRCM, the combination Sec. 6.3
proposes: hybridCS's residues with residue 0 multiplied in packed form by the
RCM operator of Eq. RCM) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import steps
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def run(hd, f, g, K=None, params=None, algo="hybridCSRCM"):
    h = hd.conv(dev(f), dev(g), algo=algo, params=params, out_extent=K)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("L", [1, 2, 3, 17, 127, 1000, 4096, 4097, 9000, 20001])
@pytest.mark.parametrize("full", [False, True])
def test_parity(hd, L, full):
    f, g = inputs.normal_pair(L, seed=5000 + L)
    K = 2 * L - 1 if full else L
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), (K,))
    assert rel_l2(run(hd, f, g, K=K if full else None), ref) <= TOL


@pytest.mark.parametrize("L", list(range(1, 17)))
def test_brute_force_every_valid_m_q(hd, L):
    """Every valid (m, q) for L <= 16 (the constraints of hybridCS), first L
    and full 2L-1 outputs: p > 1, q odd and even, m odd and even."""
    f, g = inputs.uniform_pair(L, seed=5100 + L)
    for K in (L, 2 * L - 1):
        ref = oracle.direct_conv(f, g, (K,))
        for m in range(1, 2 * L + 1):
            for q in (-(-(2 * L - 1) // m), -(-(2 * L - 1) // m) + 1):
                if steps.cs_valid(L, m, q):
                    assert rel_l2(run(hd, f, g, K=K, params=[(m, q)]), ref) <= TOL, (L, m, q, K)


@pytest.mark.parametrize("L,m,q", [(1000, 200, 10), (1000, 250, 9), (3000, 1000, 6), (4096, 2048, 4), (5000, 5000, 2)])
def test_explicit_parameters(hd, L, m, q):
    f, g = inputs.uniform_pair(L, seed=5200 + m + q)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, params=[(m, q)]), ref) <= TOL


def test_integer_exact(hd):
    f, g = inputs.integer_pair(4096, seed=5300)
    ref = oracle.direct_conv(f, g)
    h = run(hd, f, g)
    assert np.abs(h - ref).max() < 0.5
    assert np.array_equal(np.rint(h), ref)


def test_same_results_as_hybridCS(hd):
    """Same residues, same DFT lengths: only residue 0's multiply differs, so
    the two agree to rounding."""
    f, g = inputs.normal_pair(6000, seed=5400)
    a = run(hd, f, g)
    b = run(hd, f, g, algo="hybridCS")
    assert rel_l2(a, b) <= 2 * TOL


def test_batched_plan(hd):
    rng = np.random.default_rng(5500)
    Ls = rng.integers(1, 6000, 40).astype(np.int32)
    Ls[:3] = [1, 2, 4096]
    off = np.concatenate([[0], np.cumsum(Ls)[:-1]]).astype(np.int64)
    f = rng.standard_normal(int(Ls.sum())).astype(np.float32)
    g = rng.standard_normal(int(Ls.sum())).astype(np.float32)
    plan = hd.BatchPlan(off, Ls, algo="hybridCSRCM")
    h = plan(dev(f), dev(g))
    torch.cuda.synchronize()
    h = h.cpu().numpy().astype(np.float64)
    ref = oracle.batch_conv1d(f.astype(np.float64), g.astype(np.float64), off, Ls.astype(np.int64))
    for o, L in zip(off, Ls):
        assert rel_l2(h[o:o + L], ref[o:o + L]) <= TOL, L


def test_nd_full_output_unsupported(hd):
    f = dev(np.ones((8, 8)))
    with pytest.raises(hd.HDError) as e:
        hd.conv(f, f, algo="hybridCSRCM", out_extent="full")
    assert e.value.status == hd.HD_EUNSUPPORTED


# --- 2D / 3D: the combined form along the first dimension ------------------------
def nd_case(shape, seed):
    return inputs.normal_pair(shape, seed=seed)


@pytest.mark.parametrize("shape", [(37, 50), (64, 33), (12, 9, 14)])
@pytest.mark.parametrize("q0", [2, 3, 4, 5, 6])
def test_nd_first_dimension_residues(hd, shape, q0):
    """(m0, q0) along the first dimension: q0 = 2 is the packed recursion alone;
    q0 >= 3 adds hybridCS's complex residues 1..ceil(q0/2)-1 to the
    period-2m0 convolution of residues 0 and q0/2."""
    L0 = shape[0]
    m0 = -(-(2 * L0 - 1) // q0)
    f, g = nd_case(shape, 5600 + q0 + sum(shape))
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    prm = [(m0, q0)] + [(0, 0)] * (len(shape) - 1)
    h = run(hd, f, g, params=prm)
    assert rel_l2(h, ref) <= TOL, (shape, m0, q0)
    if q0 > 2:  # an odd m0 is allowed: residue q0/2 is not hybridCS's half-length transform here
        prm = [(m0 + (1 - m0 % 2), q0)] + [(0, 0)] * (len(shape) - 1)
        assert rel_l2(run(hd, f, g, params=prm), ref) <= TOL


@pytest.mark.parametrize("shape", [(1024, 1024), (64, 64, 64), (1000, 700)])
def test_nd_planner_and_large(hd, shape):
    f, g = inputs.uniform_pair(shape, seed=5700 + shape[0])
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g), ref) <= TOL
    if len(shape) == 2:  # p0 = 4 blocks, q0 = 8 residues along the first dimension
        m0 = -(-shape[0] // 4)
        prm = [(m0, -(-(2 * shape[0] - 1) // m0)), (0, 0)]
        assert rel_l2(run(hd, f, g, params=prm), ref) <= TOL
