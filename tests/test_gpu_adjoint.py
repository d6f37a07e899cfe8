"""GPU adjoint (gradients of the truncated convolution) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_14497_b300 import inputs
from tests.conftest import record_rel, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-5
ALGOS = ("hybridRCM", "hybridCS", "explicit", "explicitRCM")


@pytest.fixture(scope="module")
def hd():
    import paper_2608_14497_b300 as m
    m.load()
    return m


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("shape", [(1,), (7,), (64,), (1000,), (5, 7), (33, 40), (4, 5, 6), (9, 8, 7)])
def test_adjoint_matches_direct_correlation(hd, algo, shape):
    rng = np.random.default_rng(70)
    f, g, u = (rng.uniform(-1, 1, (2,) + shape).astype(np.float32) for _ in range(3))
    gf, gg = hd.adjoint(cuda(u), cuda(f), cuda(g), algo)
    gf, gg = gf.cpu().numpy(), gg.cpu().numpy()
    for b in range(2):
        assert rel_l2(gf[b], oracle.direct_corr(u[b], g[b])) <= TOL
        assert rel_l2(gg[b], oracle.direct_corr(u[b], f[b])) <= TOL


def test_adjoint_finite_differences_L64(hd):
    """Central differences of the FP64 oracle's <conv(f, g), u> at L = 64."""
    rng = np.random.default_rng(71)
    L = 64
    f, g, u = (rng.uniform(-1, 1, L) for _ in range(3))
    eps = 1e-3
    fd_f, fd_g = np.empty(L), np.empty(L)
    for j in range(L):
        e = np.zeros(L)
        e[j] = eps
        fd_f[j] = (np.sum(oracle.direct_conv(f + e, g) * u) - np.sum(oracle.direct_conv(f - e, g) * u)) / (2 * eps)
        fd_g[j] = (np.sum(oracle.direct_conv(f, g + e) * u) - np.sum(oracle.direct_conv(f, g - e) * u)) / (2 * eps)
    gf, gg = hd.adjoint(cuda(u[None]), cuda(f[None]), cuda(g[None]), "hybridRCM")
    assert rel_l2(gf.cpu().numpy()[0], fd_f) <= TOL
    assert rel_l2(gg.cpu().numpy()[0], fd_g) <= TOL


def test_autograd_function_dot_product(hd):
    """torch.autograd through HDConvFn: <conv(f,g), u> = <f, grad_f> = <g, grad_g> (FP64 oracle values)."""
    rng = np.random.default_rng(72)
    shape = (3, 40, 48)
    f, g, u = (rng.uniform(-1, 1, shape).astype(np.float32) for _ in range(3))
    tf = cuda(f).requires_grad_(True)
    tg = cuda(g).requires_grad_(True)
    h = hd.hd_conv_fn(tf, tg, "hybridRCM")
    (h * cuda(u)).sum().backward()
    for b in range(3):
        assert rel_l2(h.detach().cpu().numpy()[b], oracle.direct_conv(f[b], g[b])) <= TOL
        assert rel_l2(tf.grad.cpu().numpy()[b], oracle.direct_corr(u[b], g[b])) <= TOL
        assert rel_l2(tg.grad.cpu().numpy()[b], oracle.direct_corr(u[b], f[b])) <= TOL


def test_adjoint_batch16_1024_sampled(hd):
    """The differentiable 2D workload: batch 16 of 1024 x 1024, sampled gradients."""
    B, L = 16, 1024
    f, g = inputs.uniform_pair((B, L, L), seed=6)
    rng = np.random.default_rng(73)
    u = rng.uniform(-1, 1, (B, L, L)).astype(np.float32)
    tf = cuda(f).requires_grad_(True)
    tg = cuda(g).requires_grad_(True)
    h = hd.hd_conv_fn(tf, tg, "hybridRCM")
    h.backward(cuda(u))
    gfa, gga = tf.grad.cpu().numpy(), tg.grad.cpu().numpy()
    for b in (0, 7, 15):
        pts = np.stack([rng.integers(0, L, 40), rng.integers(0, L, 40)], axis=1)
        rpts = (L - 1) - pts
        ur = u[b][::-1, ::-1]
        ref_f = oracle.direct_conv_points(ur.astype(np.float64), g[b].astype(np.float64), rpts)
        ref_g = oracle.direct_conv_points(ur.astype(np.float64), f[b].astype(np.float64), rpts)
        got_f = gfa[b][tuple(pts.T)]
        got_g = gga[b][tuple(pts.T)]
        assert np.linalg.norm(got_f - ref_f) / np.linalg.norm(ref_f) <= TOL
        assert np.linalg.norm(got_g - ref_g) / np.linalg.norm(ref_g) <= TOL


def test_adjoint_batch16_1024_full_items(hd):
    """Two whole items of the 16 x 1024^2 workload against O2 in FP64:
    grad_f = rev(conv(rev(u), g)) and grad_g = rev(conv(rev(u), f)) on both axes."""
    B, L = 16, 1024
    f, g = inputs.uniform_pair((B, L, L), seed=6)
    rng = np.random.default_rng(74)
    u = rng.uniform(-1, 1, (B, L, L)).astype(np.float32)
    gf, gg = hd.adjoint(cuda(u), cuda(f), cuda(g), "hybridRCM")
    gf, gg = gf.cpu().numpy(), gg.cpu().numpy()
    for b in (0, 11):
        ur = u[b][::-1, ::-1].astype(np.float64)
        ref_f = oracle.fft_conv(ur, g[b].astype(np.float64))[::-1, ::-1]
        ref_g = oracle.fft_conv(ur, f[b].astype(np.float64))[::-1, ::-1]
        ef = record_rel(f"adjoint 16x1024^2 item {b} grad_f", rel_l2(gf[b], ref_f), TOL, ref_f.size)
        eg = record_rel(f"adjoint 16x1024^2 item {b} grad_g", rel_l2(gg[b], ref_g), TOL, ref_g.size)
        assert ef <= TOL and eg <= TOL


@pytest.mark.parametrize("shape", [(5, 7), (33, 40), (4, 5, 6), (9, 8, 7), (64, 3)])
@pytest.mark.parametrize("which", ["f", "g"])
def test_adjoint_single_gradient(hd, shape, which):
    """Only one gradient requested (the other pointer NULL, its input absent)."""
    rng = np.random.default_rng(75)
    f, g, u = (rng.uniform(-1, 1, (3,) + shape).astype(np.float32) for _ in range(3))
    gf, gg = hd.adjoint(cuda(u), cuda(f), cuda(g), "hybridRCM", need_f=(which == "f"), need_g=(which == "g"))
    for b in range(3):
        if which == "f":
            assert gg is None
            assert rel_l2(gf.cpu().numpy()[b], oracle.direct_corr(u[b], g[b])) <= TOL
        else:
            assert gf is None
            assert rel_l2(gg.cpu().numpy()[b], oracle.direct_corr(u[b], f[b])) <= TOL


def test_adjoint_rejects_overlap(hd):
    """A gradient that overlaps an input would be read after it is written."""
    x = torch.zeros((2, 8, 8), device="cuda")
    y = torch.zeros_like(x)
    out = torch.zeros_like(x)
    ctx = hd.context()
    st = hd.hd_conv_adjoint(ctx, hd.HD_HYBRID_RCM, (8, 8), 2, out.data_ptr(), x.data_ptr(), y.data_ptr(),
                            x.data_ptr(), None, 0)
    assert st == hd.HD_EINVAL
    assert b"overlap" in hd.load().hd_last_error_string()
    st = hd.hd_conv_adjoint(ctx, hd.HD_HYBRID_RCM, (8, 8), 2, out.data_ptr(), x.data_ptr(), y.data_ptr(),
                            out.data_ptr(), None, 0)
    assert st == hd.HD_EINVAL


def test_autograd_non_contiguous_inputs(hd):
    """Transposed (non-contiguous) leaves: forward and backward both run."""
    rng = np.random.default_rng(76)
    f, g, u = (rng.uniform(-1, 1, (2, 24, 20)).astype(np.float32) for _ in range(3))
    tf = cuda(f.transpose(0, 2, 1)).transpose(1, 2).requires_grad_(True)  # values of f, strides transposed
    tg = cuda(g)
    tg = tg.requires_grad_(True)
    assert not tf.is_contiguous()
    h = hd.hd_conv_fn(tf, tg, "hybridRCM")
    (h * cuda(u)).sum().backward()
    for b in range(2):
        assert rel_l2(h.detach().cpu().numpy()[b], oracle.direct_conv(f[b], g[b])) <= TOL
        assert rel_l2(tf.grad.cpu().numpy()[b], oracle.direct_corr(u[b], g[b])) <= TOL
        assert rel_l2(tg.grad.cpu().numpy()[b], oracle.direct_corr(u[b], f[b])) <= TOL
