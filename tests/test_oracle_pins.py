"""Pins for the FP64 oracle, checked against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every check is against a closed
form, exact integer arithmetic (NumPy / SciPy direct convolution on int64), an
identity the paper states, or brute force over every valid parameter choice.
"""
import math
import os

import numpy as np
import pytest
import scipy.signal

import oracle
from oracle import steps
from tests.conftest import rel_l2

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _geom_1d(a, b, L):
    k = np.arange(L, dtype=np.float64)
    return (a ** (k + 1) - b ** (k + 1)) / (a - b)


# --- P6: O1 and O2 agree ------------------------------------------------------
@pytest.mark.parametrize("shape", [(1,), (2,), (7,), (64,), (1000,), (4096,), (5, 7), (33, 17), (5, 6, 7)])
def test_direct_vs_fft(shape):
    rng = np.random.default_rng(11)
    f = rng.uniform(-1, 1, shape)
    g = rng.uniform(-1, 1, shape)
    assert rel_l2(oracle.fft_conv(f, g), oracle.direct_conv(f, g)) < 1e-13
    K = tuple(2 * n - 1 for n in shape)
    assert rel_l2(oracle.fft_conv(f, g, K), oracle.direct_conv(f, g, K)) < 1e-13


# --- P2: exact integers against library int64 convolution ---------------------
@pytest.mark.parametrize("shape", [(1,), (9,), (300,), (4096,), (13, 11), (6, 5, 7)])
def test_integer_exact(shape):
    rng = np.random.default_rng(12)
    fi = rng.integers(-8, 9, shape)
    gi = rng.integers(-8, 9, shape)
    full = scipy.signal.convolve(fi, gi, method="direct")
    assert full.dtype == np.int64
    trunc = full[tuple(slice(0, n) for n in shape)]
    h1 = oracle.direct_conv(fi.astype(float), gi.astype(float))
    assert np.array_equal(h1, trunc.astype(float))
    h2 = oracle.fft_conv(fi.astype(float), gi.astype(float))
    assert np.array_equal(np.rint(h2), trunc.astype(float))
    assert np.abs(h2 - trunc).max() < 1e-6
    K = tuple(2 * n - 1 for n in shape)
    assert np.array_equal(oracle.direct_conv(fi.astype(float), gi.astype(float), K), full.astype(float))


# --- P1: geometric closed form -------------------------------------------------
def test_geometric_golden_fixture():
    rows = [l.split() for l in open(os.path.join(GOLD, "geometric_L16.txt")) if not l.startswith("#")]
    ref = np.array([float(r[1]) for r in rows])
    L = len(ref)
    a, b = 0.9995, -0.999
    f = a ** np.arange(L)
    g = b ** np.arange(L)
    for h in (oracle.direct_conv(f, g), oracle.fft_conv(f, g), steps.conv_hybrid_cs(f, g, 32, 1),
              steps.conv_hybrid_rcm(f, g, 8, 2), steps.conv_explicit(f, g), steps.conv_explicit_rcm(f, g)):
        assert np.abs(h - ref).max() < 1e-13


@pytest.mark.parametrize("L", [4096, 70000])
def test_geometric_closed_form_1d(L):
    a, b = 0.9995, -0.999
    f = a ** np.arange(L)
    g = b ** np.arange(L)
    ref = _geom_1d(a, b, L)
    assert rel_l2(oracle.fft_conv(f, g), ref) < 1e-12
    if L <= 4096:
        assert rel_l2(oracle.direct_conv(f, g), ref) < 1e-13


def test_geometric_closed_form_nd():
    ab = [(0.999, -0.998), (0.9995, -0.999), (0.997, -0.995)]
    for shape in [(48, 40), (12, 10, 9)]:
        d = len(shape)
        f = np.ones(shape)
        g = np.ones(shape)
        ref = np.ones(shape)
        for ax in range(d):
            a, b = ab[ax]
            sh = [1] * d
            sh[ax] = shape[ax]
            f = f * (a ** np.arange(shape[ax])).reshape(sh)
            g = g * (b ** np.arange(shape[ax])).reshape(sh)
            ref = ref * _geom_1d(a, b, shape[ax]).reshape(sh)
        assert rel_l2(oracle.direct_conv(f, g), ref) < 1e-13
        assert rel_l2(oracle.fft_conv(f, g), ref) < 1e-12


# --- P5: special cases ----------------------------------------------------------
def test_delta_shift_commutative_bilinear():
    rng = np.random.default_rng(13)
    L = 37
    g = rng.normal(size=L)
    for j in (0, 1, 5, 36):
        d = np.zeros(L)
        d[j] = 1.0
        h = oracle.direct_conv(d, g)
        ref = np.zeros(L)
        ref[j:] = g[: L - j]
        assert np.array_equal(h, ref)
        assert np.abs(oracle.fft_conv(d, g) - ref).max() < 1e-14
    f, f2 = rng.normal(size=L), rng.normal(size=L)
    assert np.allclose(oracle.direct_conv(f, g), oracle.direct_conv(g, f), rtol=0, atol=1e-13)
    lhs = oracle.direct_conv(2.5 * f - 0.75 * f2, g)
    rhs = 2.5 * oracle.direct_conv(f, g) - 0.75 * oracle.direct_conv(f2, g)
    assert np.abs(lhs - rhs).max() < 1e-12


# --- adjoint: dot-product test and central finite differences ------------------
@pytest.mark.parametrize("shape", [(64,), (9, 11), (5, 4, 6)])
def test_adjoint_dot_product(shape):
    rng = np.random.default_rng(14)
    f, g, u = (rng.normal(size=shape) for _ in range(3))
    lhs = np.sum(oracle.direct_conv(f, g) * u)
    assert abs(lhs - np.sum(f * oracle.direct_corr(u, g))) < 1e-11 * max(1, abs(lhs))
    assert abs(lhs - np.sum(g * oracle.direct_corr(u, f))) < 1e-11 * max(1, abs(lhs))


def test_adjoint_finite_differences_L64():
    rng = np.random.default_rng(15)
    L = 64
    f, g, u = (rng.uniform(-1, 1, L) for _ in range(3))
    grad = oracle.direct_corr(u, g)
    eps = 1e-3
    fd = np.empty(L)
    for j in range(L):
        e = np.zeros(L)
        e[j] = eps
        fd[j] = (np.sum(oracle.direct_conv(f + e, g) * u) - np.sum(oracle.direct_conv(f - e, g) * u)) / (2 * eps)
    assert np.abs(fd - grad).max() < 1e-10


def test_adjoint_is_reversed_convolution():
    """grad_f = rev(conv_L(rev(u), g)): the reading of the adjoint the library uses."""
    rng = np.random.default_rng(16)
    for shape in [(50,), (7, 9), (4, 5, 3)]:
        g, u = rng.normal(size=shape), rng.normal(size=shape)
        rev = tuple(slice(None, None, -1) for _ in shape)
        assert np.abs(oracle.direct_corr(u, g) - oracle.direct_conv(u[rev], g)[rev]).max() < 1e-12


# --- P3: brute force over every valid (m, q) for L <= 16 -----------------------
def _qs(qmin):
    return (qmin, qmin + 1)


@pytest.mark.parametrize("L", list(range(1, 17)))
def test_brute_force_cs_rcm_complex(L):
    rng = np.random.default_rng(100 + L)
    f = rng.uniform(-1, 1, L)
    g = rng.uniform(-1, 1, L)
    ref = oracle.direct_conv(f, g)
    for m in range(1, 2 * L + 1):
        for q in _qs(-(-(2 * L - 1) // m)):
            if steps.cs_valid(L, m, q):
                assert rel_l2(steps.conv_hybrid_cs(f, g, m, q), ref) < 1e-12, (L, m, q)
        for q in _qs(-(-L // m)):
            if steps.rcm_valid(L, m, q):
                assert rel_l2(steps.conv_hybrid_rcm(f, g, m, q), ref) < 1e-12, (L, m, q)
    fc = f + 1j * rng.uniform(-1, 1, L)
    gc = g + 1j * rng.uniform(-1, 1, L)
    refc = np.convolve(fc, gc)[:L]
    for m in range(1, 2 * L + 1):
        q = -(-(2 * L - 1) // m)
        assert np.abs(steps.conv_complex_hybrid(fc, gc, m, q) - refc).max() < 1e-12


def test_explicit_baselines_1d():
    rng = np.random.default_rng(17)
    for L in (1, 2, 3, 10, 31, 256):
        f, g = rng.uniform(-1, 1, L), rng.uniform(-1, 1, L)
        ref = oracle.direct_conv(f, g)
        assert rel_l2(steps.conv_explicit(f, g), ref) < 1e-12
        assert rel_l2(steps.conv_explicit_rcm(f, g), ref) < 1e-12


# --- P4: identities the paper states ---------------------------------------------
def test_residue_conjugate_symmetry():
    """Eq. hrHerm: conj(h_r) = h_{q-r} for the spectrum of real data."""
    rng = np.random.default_rng(18)
    for (L, m, q) in [(20, 8, 5), (20, 6, 7), (33, 16, 4)]:
        f = rng.normal(size=L)
        p = -(-L // m)
        F = steps.hybrid_forward(f, m, q)
        h = [steps.residue_contribution(F[r::q], m, q, p, r) for r in range(q)]
        for r in range(1, q):
            assert np.abs(np.conj(h[r]) - h[q - r]).max() < 1e-11


def test_residue_q2_closure_and_even_indices():
    """Eq. realq2symmetry and Eq. forwardq2 (even indices of Eq. resq2)."""
    rng = np.random.default_rng(19)
    for (L, m, q) in [(12, 8, 4), (21, 10, 6), (7, 4, 4), (16, 16, 2)]:
        f = rng.normal(size=L)
        Fr = steps.forward_residue(f, m, q, q // 2)
        assert np.abs(np.conj(Fr) - Fr[::-1]).max() < 1e-11
        assert np.abs(steps.cs_forward(f, m, q, q // 2) - Fr[0::2]).max() < 1e-11
        F0 = steps.forward_residue(f, m, q, 0)
        assert np.abs(steps.cs_forward(f, m, q, 0) - F0[: m // 2 + 1]).max() < 1e-11


def test_fourier_unpack_pack():
    """Eqs. fourierUnpack / fourierPack against the library DFT of the real data."""
    rng = np.random.default_rng(20)
    for N in (1, 2, 5, 16, 37):
        f = rng.normal(size=2 * N)
        Ft = steps.dft(steps.pack(f), +1)
        F = steps.dft(f, +1)[: N + 1]
        assert np.abs(steps.fourier_unpack(Ft) - F).max() < 1e-11
        assert np.abs(steps.fourier_pack(F) - Ft).max() < 1e-11


def test_rcm_operator_forms():
    """Eq. RCM equals Eq. RCM-U; Alg. 4 equals Eq. RCM; associativity (Sec. 4.1);
    and the RCM product is the DFT of the packing of the cyclic convolution."""
    rng = np.random.default_rng(21)
    for N in (2, 4, 10, 64):
        F1, F2, F3 = (rng.normal(size=N) + 1j * rng.normal(size=N) for _ in range(3))
        assert np.abs(steps.rcm(F1, F2) - steps.rcm_via_U(F1, F2)).max() < 1e-11
        A, B = F1.copy(), F2.copy()
        steps.mult_rcm(A, B, A, B, True)
        assert np.abs(A - steps.rcm(F1, F2)).max() < 1e-11
        lhs = steps.rcm(steps.rcm(F1, F2), F3)
        rhs = steps.rcm(F1, steps.rcm(F2, F3))
        assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(lhs).max()
        f, g = rng.normal(size=2 * N), rng.normal(size=2 * N)
        cyc = np.real(np.fft.ifft(np.fft.fft(f) * np.fft.fft(g)))
        Ft, Gt = steps.dft(steps.pack(f), +1), steps.dft(steps.pack(g), +1)
        assert np.abs(steps.rcm(Ft, Gt) - steps.dft(steps.pack(cyc), +1)).max() < 1e-10


def test_rcm_W_symmetry():
    """conj(W_{l,r}) = W_{m-l-1, q-r} for r not in {0, q/2} (Sec. 4)."""
    rng = np.random.default_rng(22)
    m, q = 7, 6
    Ft = rng.normal(size=q * m) + 1j * rng.normal(size=q * m)
    Gt = rng.normal(size=q * m) + 1j * rng.normal(size=q * m)
    for r in (1, 2, 4, 5):
        for l in range(m):
            w1 = np.conj(steps.rcm_W(Ft, Gt, m, q, l, r))
            w2 = steps.rcm_W(Ft, Gt, m, q, m - l - 1, q - r)
            assert abs(w1 - w2) < 1e-12
    H = steps.rcm_residue_pairs(Ft, Gt, m, q)
    assert np.abs(H - steps.rcm(Ft, Gt)).max() < 1e-11


def test_C_n_slice_identity():
    """Sec. 5: C_n(A,B,C,D)_{(k1,...)} = C_{n-1}(A^{k1}, B^{k1}, C^{k1*}, D^{k1*})."""
    rng = np.random.default_rng(23)
    for shape in [(6, 5), (4, 3, 8)]:
        A, B, C, D = (rng.normal(size=shape) + 1j * rng.normal(size=shape) for _ in range(4))
        full = steps.C_op(A, B, C, D)
        M1 = shape[0]
        for k1 in range(M1):
            k1s = (M1 - k1) % M1
            assert np.abs(full[k1] - steps.C_op(A[k1], B[k1], C[k1s], D[k1s])).max() < 1e-12
        assert np.abs(steps.C_op(A, B, A, B) - steps.rcm_ndim(A, B)).max() < 1e-14


def test_nd_step_algorithms_vs_direct():
    rng = np.random.default_rng(24)
    f, g = rng.uniform(-1, 1, (9, 10)), rng.uniform(-1, 1, (9, 10))
    ref = oracle.direct_conv(f, g)
    assert rel_l2(steps.conv_explicit_rcm_2d(f, g), ref) < 1e-12
    for prm in [((9, 2), (5, 2)), ((17, 1), (3, 4)), ((6, 3), (2, 5))]:
        assert rel_l2(steps.conv_hybrid_rcm_nd(f, g, prm), ref) < 1e-12
    with pytest.raises(ValueError):
        steps.conv_hybrid_rcm_nd(f, g, ((6, 3), (2, 3)))
    for prm in [((9, 2), (5, 2))]:
        assert rel_l2(steps.conv_hybrid_rcm_nd(f, g, prm), ref) < 1e-12
    for prm in [((10, 2), (10, 2)), ((6, 3), (7, 3)), ((17, 1), (4, 5)), ((4, 5), (19, 1))]:
        assert rel_l2(steps.conv_hybrid_cs_nd(f, g, prm), ref) < 1e-12
    f3, g3 = rng.uniform(-1, 1, (5, 4, 7)), rng.uniform(-1, 1, (5, 4, 7))
    ref3 = oracle.direct_conv(f3, g3)
    assert rel_l2(steps.conv_hybrid_rcm_nd(f3, g3, ((5, 2), (4, 2), (4, 2))), ref3) < 1e-12
    assert rel_l2(steps.conv_hybrid_cs_nd(f3, g3, ((6, 2), (4, 2), (7, 2))), ref3) < 1e-12
    f2, g2 = rng.uniform(-1, 1, (6, 7)), rng.uniform(-1, 1, (6, 7))
    assert rel_l2(steps.conv_explicit_rcm_2d(f2, g2), oracle.direct_conv(f2, g2)) < 1e-12


# --- planted mistakes: each pin above must catch a plausible error -------------
def test_planted_sign_convention_is_caught(monkeypatch):
    """Flip the root-of-unity sign (zeta_N = e^{-2 pi i/N}): the RCM factor
    (1 + zeta_N^k) then belongs to the other convention and P3 fails."""
    rng = np.random.default_rng(25)
    f, g = rng.uniform(-1, 1, 12), rng.uniform(-1, 1, 12)
    ref = oracle.direct_conv(f, g)
    good = steps.zeta
    monkeypatch.setattr(steps, "rcm_W", lambda Ft, Gt, m, q, l, r: (
        0.25 * (Ft[q * l + r] - np.conj(Ft[(q * m - q * l - r) % (q * m)]))
        * (Gt[q * l + r] - np.conj(Gt[(q * m - q * l - r) % (q * m)])) * (1 + good(q * m, -(q * l + r)))))
    assert rel_l2(steps.conv_hybrid_rcm(f, g, 4, 3), ref) > 1e-3


def test_planted_pairing_index_is_caught(monkeypatch):
    """Pair l with m-l (instead of m-l-1) for r != 0: the conjugate partner is wrong."""
    rng = np.random.default_rng(26)
    f, g = rng.uniform(-1, 1, 14), rng.uniform(-1, 1, 14)
    ref = oracle.direct_conv(f, g)

    def bad_W(Ft, Gt, m, q, l, r):
        k = q * l + r
        kc = (q * (m - l) + q - r) % (q * m) if r else (q * m - k) % (q * m)
        return 0.25 * (Ft[k] - np.conj(Ft[kc])) * (Gt[k] - np.conj(Gt[kc])) * (1 + steps.zeta(q * m, k))

    monkeypatch.setattr(steps, "rcm_W", bad_W)
    assert rel_l2(steps.conv_hybrid_rcm(f, g, 4, 4), ref) > 1e-3


def test_planted_dropped_q2_term_is_caught(monkeypatch):
    """Drop the (-1)^t sign of Eq. accumulateq2: P3 fails whenever p > 1."""
    rng = np.random.default_rng(27)
    f, g = rng.uniform(-1, 1, 11), rng.uniform(-1, 1, 11)
    ref = oracle.direct_conv(f, g)
    orig = steps.cs_backward

    def bad(H, m, q, p, r):
        out = orig(H, m, q, p, r)
        if 2 * r == q and p > 1:
            out = out.reshape(p, m)
            out[1::2] *= -1
            out = out.reshape(-1)
        return out

    monkeypatch.setattr(steps, "cs_backward", bad)
    assert rel_l2(steps.conv_hybrid_cs(f, g, 6, 4), ref) > 1e-3


def test_direct_points_match_full_and_closed_form():
    rng = np.random.default_rng(28)
    for shape in [(40,), (9, 11), (5, 6, 7)]:
        f, g = rng.normal(size=shape), rng.normal(size=shape)
        full = oracle.direct_conv(f, g)
        pts = np.stack([rng.integers(0, n, 25) for n in shape], axis=1)
        assert np.allclose(oracle.direct_conv_points(f, g, pts), full[tuple(pts.T)], rtol=0, atol=1e-12)
    # separable geometric inputs at a large 3D size: closed form at sampled points
    L = 64
    a, b = (0.99, 0.995, 0.98), (-0.97, 0.96, -0.99)
    f = np.einsum("i,j,k->ijk", *[a[i] ** np.arange(L) for i in range(3)])
    g = np.einsum("i,j,k->ijk", *[b[i] ** np.arange(L) for i in range(3)])
    pts = np.stack([rng.integers(0, L, 20) for _ in range(3)], axis=1)
    ref = np.prod([_geom_1d(a[i], b[i], L)[pts[:, i]] for i in range(3)], axis=0)
    assert np.allclose(oracle.direct_conv_points(f, g, pts), ref, rtol=1e-11, atol=0)


# --- the batched oracle (flat arrays, item i at offsets[i], length Ls[i]) -------
def _uneven_batch(seed=21):
    """About 30 uneven items with gaps between them (L = 1 included)."""
    rng = np.random.default_rng(seed)
    Ls = np.concatenate([[1, 2, 3], rng.integers(1, 700, 27)]).astype(np.int64)
    gaps = rng.integers(0, 9, len(Ls)).astype(np.int64)
    off = np.zeros(len(Ls), dtype=np.int64)
    off[0] = gaps[0]
    for i in range(1, len(Ls)):
        off[i] = off[i - 1] + Ls[i - 1] + gaps[i]
    total = int(off[-1] + Ls[-1] + 5)
    f = rng.uniform(-1, 1, total)
    g = rng.uniform(-1, 1, total)
    return off, Ls, f, g


def _check_batch(h, f, g, off, Ls):
    """Every item equals the single-array direct convolution of its slices, and
    every position outside the items is left at zero."""
    covered = np.zeros(len(f), dtype=bool)
    for o, L in zip(off, Ls):
        ref = oracle.direct_conv(f[o:o + L], g[o:o + L])
        if not (rel_l2(h[o:o + L], ref) < 1e-13):
            return False
        covered[o:o + L] = True
    return bool(np.all(h[~covered] == 0.0))


@pytest.mark.parametrize("use_fft", [True, False])
def test_batch_conv1d_matches_per_item(use_fft):
    off, Ls, f, g = _uneven_batch()
    h = oracle.batch_conv1d(f, g, off, Ls, use_fft=use_fft)
    assert _check_batch(h, f, g, off, Ls)
    # and item by item against O2 on the same slices
    for o, L in zip(off, Ls):
        assert rel_l2(h[o:o + L], oracle.fft_conv(f[o:o + L], g[o:o + L])) < 1e-13


def test_batch_conv1d_integer_exact():
    rng = np.random.default_rng(22)
    Ls = np.array([1, 5, 64, 300, 17], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(Ls)[:-1]]).astype(np.int64)
    fi = rng.integers(-8, 9, int(Ls.sum()))
    gi = rng.integers(-8, 9, int(Ls.sum()))
    h = oracle.batch_conv1d(fi.astype(float), gi.astype(float), off, Ls, use_fft=False)
    for o, L in zip(off, Ls):
        exact = scipy.signal.convolve(fi[o:o + L], gi[o:o + L], method="direct")[:L]
        assert np.array_equal(h[o:o + L], exact.astype(float))


def test_planted_batch_offset_mistake_is_caught():
    """A batch whose g is read at the wrong offset (the next item's start, as a
    mistake that applied off[i] to f but not to g would) fails the check."""
    off, Ls, f, g = _uneven_batch()
    shifted = np.roll(g, -int(Ls[0]))  # g_i read from another item's data
    h_bad = oracle.batch_conv1d(f, shifted, off, Ls, use_fft=True)
    assert not _check_batch(h_bad, f, g, off, Ls)
    h_off = oracle.batch_conv1d(f, g, off + 1, Ls, use_fft=True)  # every item one place late
    assert not _check_batch(h_off, f, g, off, Ls)


# --- O1m / O2m: n >= 2 arrays of possibly different lengths (Sec. 4.1; Sec. 7) ---
def _int_multi(rng, lengths):
    return [rng.integers(-8, 9, L) for L in lengths]


def _exact_multi(xs):
    """Repeated exact int64 convolution (SciPy direct method, integer dtype)."""
    acc = xs[0]
    for x in xs[1:]:
        acc = scipy.signal.convolve(acc, x, method="direct")
    return acc


def _multi_matches(h, xs_int, K):
    return np.array_equal(h, _exact_multi(xs_int)[:K].astype(float))


@pytest.mark.parametrize("lengths", [(37, 5), (5, 37), (1, 9), (4096, 64), (300, 300), (17, 1, 9), (64, 33, 7, 12)])
def test_multi_integer_exact(lengths):
    rng = np.random.default_rng(30 + sum(lengths))
    xi = _int_multi(rng, lengths)
    S = sum(lengths) - len(lengths) + 1
    xs = [x.astype(float) for x in xi]
    for K in (max(lengths), S):
        assert _multi_matches(oracle.direct_conv_multi(xs, K), xi, K)
        h2 = oracle.fft_conv_multi(xs, K)
        assert np.abs(h2 - _exact_multi(xi)[:K]).max() < 1e-6
    assert len(oracle.direct_conv_multi(xs)) == max(lengths)  # default K = max L_i


def test_multi_three_geometric_closed_form():
    """x^i_j = a_i^j: for k below every length, the sum over j1 + j2 + j3 = k of
    a^j1 b^j2 c^j3 has the partial-fraction closed form sum_i a_i^{k+2} /
    prod_{l != i} (a_i - a_l)."""
    a, b, c = 0.9995, -0.999, 0.5
    L = (300, 200, 250)
    xs = [r ** np.arange(n, dtype=np.float64) for r, n in zip((a, b, c), L)]
    k = np.arange(200, dtype=np.float64)
    ref = (a ** (k + 2) / ((a - b) * (a - c)) + b ** (k + 2) / ((b - a) * (b - c)) +
           c ** (k + 2) / ((c - a) * (c - b)))
    for fn in (oracle.direct_conv_multi, oracle.fft_conv_multi):
        assert rel_l2(fn(xs, 200), ref) < 1e-12


def test_multi_delta_shifts():
    rng = np.random.default_rng(33)
    f = rng.standard_normal(50)
    d3 = np.zeros(4)
    d3[3] = 1.0
    d5 = np.zeros(6)
    d5[5] = 1.0
    S = 50 + 4 + 6 - 2
    ref = np.zeros(S)
    ref[8:58] = f
    for fn in (oracle.direct_conv_multi, oracle.fft_conv_multi):
        assert np.abs(fn([d3, f, d5], S) - ref).max() < 1e-13


def test_multi_rejects_bad_extent():
    with pytest.raises(ValueError):
        oracle.direct_conv_multi([np.ones(4), np.ones(3)], 7)  # support is 6
    with pytest.raises(ValueError):
        oracle.fft_conv_multi([np.ones(4)], 4)


def test_planted_multi_reversed_operand_is_caught(monkeypatch):
    """An oracle that read one array back to front (a transposed operand)
    fails the integer pin."""
    rng = np.random.default_rng(34)
    xi = _int_multi(rng, (40, 7, 9))
    xs = [x.astype(float) for x in xi]
    orig = oracle._multi
    monkeypatch.setattr(oracle, "_multi", lambda name, ys, K: orig(name, [ys[0], ys[1][::-1]] + list(ys[2:]), K))
    S = 40 + 7 + 9 - 2
    assert not _multi_matches(oracle.direct_conv_multi(xs, S), xi, S)


# --- App. A inner loop (the three-kernel path's arithmetic), pinned against O1 ---
@pytest.mark.parametrize("L,m,q", [(1, 1, 2), (7, 2, 4), (37, 4, 10), (100, 8, 14), (64, 16, 8), (250, 10, 26)])
def test_inner_loop_forward_is_eq_forwardr(L, m, q):
    rng = np.random.default_rng(40 + L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    if L > q * m:
        pytest.skip("more blocks than residues")
    assert np.allclose(steps.inner_loop_forward(x, m, q), steps.hybrid_forward(x, m, q), atol=1e-9)


@pytest.mark.parametrize("L,m,q", [(1, 1, 2), (9, 2, 6), (37, 4, 10), (101, 8, 14), (256, 16, 16), (300, 20, 16)])
def test_inner_loop_rcm_and_cs_match_direct(L, m, q):
    rng = np.random.default_rng(50 + L)
    f, g = rng.standard_normal(L), rng.standard_normal(L)
    for K in (L, 2 * L - 1):
        ref = oracle.direct_conv(f, g, (K,))
        if 2 * q * m >= 2 * L - 1:
            assert rel_l2(steps.conv_rcm_inner_loop([f, g], m, q, K), ref) < 1e-12
        if q * m >= 2 * L - 1:
            assert rel_l2(steps.conv_cs_inner_loop(f, g, m, q, K), ref) < 1e-12


@pytest.mark.parametrize("lengths,m,q", [((50, 7), 8, 8), ((30, 20, 12), 8, 8), ((13, 1, 5, 9), 4, 8), ((64,) * 5, 16, 20)])
def test_inner_loop_n_arrays_unequal_match_direct(lengths, m, q):
    """Sec. 4.1 (R^j = R^{j-1} RCM F^j) and Sec. 7 (separate block counts), the
    reading of Eq. RnMk with conj(A_k)."""
    rng = np.random.default_rng(60 + sum(lengths))
    xs = [rng.standard_normal(L) for L in lengths]
    S = sum(lengths) - len(lengths) + 1
    ref = oracle.direct_conv_multi(xs, S)
    assert rel_l2(steps.conv_rcm_inner_loop(xs, m, q, S), ref) < 1e-12


def test_planted_inner_loop_sign_is_caught(monkeypatch):
    """A q-point DFT over the blocks with the wrong sign fails the pin."""
    rng = np.random.default_rng(70)
    f, g = rng.standard_normal(101), rng.standard_normal(101)
    orig = steps.dft
    monkeypatch.setattr(steps, "dft", lambda x, sign=+1, axis=-1: orig(x, -sign if axis == 0 else sign, axis))
    assert rel_l2(steps.conv_rcm_inner_loop([f, g], 8, 14), oracle.direct_conv(f, g)) > 1e-3
