"""GPU parity of the 2D/3D paths (recursive decomposition) and the explicit
baselines against the FP64 oracle."""
import numpy as np
import pytest

import oracle
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


_O2 = {}


def full_size_case(shape):
    """Seeded full-size inputs (2D: U[-1,1) seed 4; 3D: N(0,1) seed 5) and the
    FP64 oracle O2 on them, computed once per shape."""
    if shape not in _O2:
        if len(shape) == 2:
            f, g = inputs.uniform_pair(shape, seed=4)
        else:
            f, g = inputs.normal_pair(shape, seed=5)
        _O2.clear()  # one full-size reference held at a time (3D L=256: 134 MB)
        _O2[shape] = (f, g, oracle.fft_conv(f.astype(np.float64), g.astype(np.float64)))
    return _O2[shape]


@pytest.mark.parametrize("L", [1024, 2048, 3000])
@pytest.mark.parametrize("algo", ALL)
def test_2d_full_size_every_output(hd, algo, L):
    """Every output of the 2D configs against O2 (element by element)."""
    f, g, ref = full_size_case((L, L))
    h = run(hd, f, g, algo)
    assert np.isfinite(h).all()
    err = record_rel(f"2D L={L} {algo}", rel_l2(h, ref), TOL, h.size)
    assert err <= TOL
    # no row, column or boundary block may be off on its own
    rows = np.linalg.norm(h - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    assert rows.max() <= 20 * TOL


@pytest.mark.parametrize("algo", ALL)
def test_3d_L256_every_output(hd, algo):
    """Every output of 3D L = 256 against O2 (element by element)."""
    f, g, ref = full_size_case((256, 256, 256))
    h = run(hd, f, g, algo)
    assert np.isfinite(h).all()
    err = record_rel(f"3D L=256 {algo}", rel_l2(h, ref), TOL, h.size)
    assert err <= TOL
    planes = np.linalg.norm((h - ref).reshape(256, -1), axis=1) / np.linalg.norm(ref.reshape(256, -1), axis=1)
    assert planes.max() <= 20 * TOL


def face_diagonal_points(L, nrand, seed):
    """Every output on the diagonals of the faces k0 = 0, k1 = 0 and k2 = L-1,
    plus nrand random points."""
    i = np.arange(L)
    z = np.zeros(L, dtype=np.int64)
    last = np.full(L, L - 1, dtype=np.int64)
    rng = np.random.default_rng(seed)
    rnd = rng.integers(0, L, (nrand, 3))
    return np.concatenate([np.stack([z, i, i], 1), np.stack([i, z, i], 1), np.stack([i, i, last], 1), rnd])


@pytest.mark.parametrize("algo", ALL)
def test_3d_L384_faces_and_points(hd, algo):
    """3D L = 384 (O2 would need a 1024^3 grid): direct FP64 sums at every
    output on three face diagonals and at 2000 random points."""
    L = 384
    f, g = inputs.normal_pair((L, L, L), seed=5)
    h = run(hd, f, g, algo)
    assert np.isfinite(h).all()
    pts = face_diagonal_points(L, 2000, seed=L)
    ref = oracle.direct_conv_points(f.astype(np.float64), g.astype(np.float64), pts)
    got = h[tuple(pts.T)]
    err = record_rel(f"3D L=384 {algo} (faces + 2000 points)", np.linalg.norm(got - ref) / np.linalg.norm(ref),
                     TOL, len(pts))
    assert err <= TOL


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


# Rows whose real length fits 256 R3 take the one-residue row pass (q = 1):
# packed row lengths 65..128 with L <= 256, 129..256 with L <= 512, ragged and
# odd, first L outputs and the full 2L-1 (output rows up to M).
@pytest.mark.parametrize("shape", [(40, 200), (17, 256), (9, 129), (6, 7, 250), (5, 3, 511), (33, 500)])
@pytest.mark.parametrize("full", [False, True])
def test_one_residue_rows(hd, shape, full):
    f, g = inputs.normal_pair(shape, seed=900 + sum(shape))
    K = tuple(2 * n - 1 for n in shape) if full else tuple(shape)
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64), K)
    tf = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    tg = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    h = hd.conv(tf, tg, algo="hybridRCM", out_extent=K if full else None)
    torch.cuda.synchronize()
    assert rel_l2(h.cpu().numpy().astype(np.float64), ref) <= TOL


# the column passes' compile-time residue lengths (m = 256, 384, 1024, 2048,
# 3072 for L = 256, 384, 1024, 2048, 3000 along an outer dimension) with column
# counts that leave a partial last strip (B not a multiple of the strip width),
# along the first and, in 3D, the middle dimension; every output against O2
@pytest.mark.parametrize("algo", ("hybridRCM", "hybridCS", "hybridCSRCM"))
@pytest.mark.parametrize("shape", [(384, 379), (256, 61), (1024, 33), (2048, 9), (3000, 17), (384, 7, 13),
                                   (5, 384, 11), (256, 3, 29)])
def test_compile_time_column_lengths(hd, algo, shape):
    f, g = inputs.uniform_pair(shape, seed=7000 + sum(shape))
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL


# a middle-dimension column pass with fewer than 8 columns per block (Lp = 3,
# 5, 6, 7) and hundreds of blocks: the strip width must stay a power of two
@pytest.mark.parametrize("algo", ALL)
@pytest.mark.parametrize("shape", [(300, 5, 11), (160, 9, 5), (200, 3, 9), (150, 4, 14)])
def test_3d_narrow_middle_blocks(hd, algo, shape):
    f, g = inputs.normal_pair(shape, seed=7100 + sum(shape))
    ref = oracle.fft_conv(f.astype(np.float64), g.astype(np.float64))
    assert rel_l2(run(hd, f, g, algo), ref) <= TOL
