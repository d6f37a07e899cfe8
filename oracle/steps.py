"""FP64 step oracle: the paper's equations, one step at a time, in NumPy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (Sec. 2): zeta_N = exp(+2 pi i / N); forward transforms use the
plus sign, backward transforms the minus sign and no scaling, except where an
equation carries 1/(qm).  Index splits: j = t m + s (t < p, s < m) for inputs
and k = q l + r (l < m, r < q) for transformed data (Sec. 2).  The library FFT
(numpy.fft) serves only as the plain length-n DFT step
``dft(x, +1) = sum_j x_j zeta_n^{jk}``; every other step is written out as the
equation states it, with no blocking or fusion beyond it.

Readings of places where the paper is silent or garbled:
  * the DFT index range "k = 0..M" before Eq. forwardr is k = 0..qm-1;
  * the packed length written with an undefined macro in Sec. 4 is the packed
    complex length N (real length 2N), i.e. qm in the hybrid setting;
  * the forward r = 0 real FFT returns bins 0..floor(m/2) (Alg. 1's upper
    index is garbled); the backward input for r = q/2 has m/2 entries;
  * outputs are the first L per dimension, normalised by 1/(qm) per dimension;
  * dealiasing needs qm >= 2L-1 for real or complex data of length L and
    qm >= L for packed data (real length 2qm >= 2L-1).
"""
import math

import numpy as np


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------
def zeta(N, k):
    """zeta_N^k = exp(2 pi i k / N)  (Sec. 2)."""
    return np.exp(2j * np.pi * np.asarray(k, dtype=np.float64) / N)


def dft(x, sign=+1, axis=-1):
    """sum_j x_j zeta_n^{sign j k} along ``axis`` (unnormalised)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[axis]
    if sign > 0:
        return np.fft.ifft(x, axis=axis) * n
    return np.fft.fft(x, axis=axis)


def hybrid_params(L, M, m):
    """Sec. 2: p = ceil(L/m), q = ceil(M/m)."""
    return -(-L // m), -(-M // m)


def _pad(f, n):
    out = np.zeros(n, dtype=np.complex128)
    out[: len(f)] = f
    return out


# ---------------------------------------------------------------------------
# Sec. 2: complex hybrid dealiasing, one residue at a time
# ---------------------------------------------------------------------------
def forward_residue(f, m, q, r):
    """Eq. forwardr for one residue: F_{q l + r}, l = 0..m-1.

    y_s = zeta_{qm}^{rs} sum_{t<p} zeta_q^{rt} f_{tm+s}, then a length-m DFT."""
    L = len(f)
    p = -(-L // m)
    x = _pad(f, p * m).reshape(p, m)
    t = np.arange(p)[:, None]
    s = np.arange(m)
    inner = np.sum(zeta(q, r * t) * x, axis=0)
    y = zeta(q * m, r * s) * inner
    return dft(y, +1)


def hybrid_forward(f, m, q):
    """Eq. forwardr for all residues: the DFT of f zero padded to qm."""
    F = np.zeros(q * m, dtype=np.complex128)
    for r in range(q):
        F[r::q] = forward_residue(f, m, q, r)
    return F


def residue_contribution(Fr, m, q, p, r):
    """Eq. accumulator: h_{r, tm+s} = zeta_q^{-tr} zeta_{qm}^{-sr} sum_l zeta_m^{-sl} F_{ql+r}."""
    w = dft(Fr, -1)
    t = np.arange(p)[:, None]
    s = np.arange(m)
    return (zeta(q, -t * r) * zeta(q * m, -s * r) * w).reshape(p * m)


def hybrid_backward(F, m, q, p):
    """Eqs. backwardr / accumulation: f = (1/qm) sum_r h_r (length pm)."""
    acc = np.zeros(p * m, dtype=np.complex128)
    for r in range(q):
        acc += residue_contribution(F[r::q], m, q, p, r)
    return acc / (q * m)


def conv_complex_hybrid(f, g, m, q, K=None):
    """Complex hybrid-dealiased convolution (Sec. 2): F, G, pointwise, backward."""
    L = len(f)
    p = -(-L // m)
    F = hybrid_forward(f, m, q)
    G = hybrid_forward(g, m, q)
    h = hybrid_backward(F * G, m, q, p)
    return h[: (L if K is None else K)]


# ---------------------------------------------------------------------------
# Sec. 3: real hybrid dealiasing via conjugate symmetries (hybridCS)
# ---------------------------------------------------------------------------
def cs_valid(L, m, q):
    """Constraints: qm >= 2L-1 (dealiased) and m even when q is even (Sec. 3.1.3)."""
    return q * m >= 2 * L - 1 and not (q % 2 == 0 and m % 2 == 1)


def cs_forward(f, m, q, r):
    """Forward residue transform for real f, the three cases of Sec. 3.1.

    r = 0: real fold sum_t f_{tm+s}, real-to-complex DFT, bins 0..floor(m/2).
    1 <= r < ceil(q/2): Eq. forwardr (complex, length m).
    r = q/2: Eq. forwardq2 -> the even indices F_{2cq+q/2}, c < m/2."""
    L = len(f)
    p = -(-L // m)
    x = np.zeros(p * m)
    x[:L] = f
    x = x.reshape(p, m)
    if r == 0:
        fold = x.sum(axis=0)
        return dft(fold, +1)[: m // 2 + 1]
    if 2 * r == q:
        e = m // 2
        sgn = (-1.0) ** np.arange(p)[:, None]
        xs = np.sum(sgn * x, axis=0)  # sum_t (-1)^t f_{tm+s}
        b = np.arange(e)
        W = zeta(2 * m, b) * (xs[:e] + 1j * xs[e:])
        return dft(W, +1)
    return forward_residue(f, m, q, r)


def cs_backward(H, m, q, p, r):
    """Residue contribution h_r for the real algorithm (Sec. 3.1).

    r = 0: complex-to-real DFT (the spectrum is Hermitian, bins 0..floor(m/2)).
    1 <= r < ceil(q/2): Eq. accumulator (complex; the caller takes 2 Re).
    r = q/2: Eqs. wb and accumulateq2: w_b, then (-1)^t 2Re w_b, (-1)^t 2Im w_b."""
    t = np.arange(p)[:, None]
    if r == 0:
        full = np.zeros(m, dtype=np.complex128)
        nh = m // 2 + 1
        full[:nh] = H
        for l in range(nh, m):
            full[l] = np.conj(H[m - l])
        w = dft(full, -1).real
        return np.tile(w, p)
    if 2 * r == q:
        e = m // 2
        b = np.arange(e)
        w = zeta(2 * m, -b) * dft(H, -1)
        sgn = (-1.0) ** t
        out = np.zeros((p, m))
        out[:, :e] = sgn * 2.0 * w.real
        out[:, e:] = sgn * 2.0 * w.imag
        return out.reshape(p * m)
    return residue_contribution(H, m, q, p, r)


def conv_hybrid_cs(f, g, m, q, K=None):
    """hybridCS: Eq. real-accumulation,
    f = (1/qm)(h_0 + 2 sum_{r=1}^{ceil(q/2)-1} Re h_r + h_{q/2})."""
    L = len(f)
    if not cs_valid(L, m, q):
        raise ValueError("invalid (m, q) for hybridCS")
    p = -(-L // m)
    acc = np.zeros(p * m)
    for r in range(0, (q + 1) // 2):
        H = cs_forward(f, m, q, r) * cs_forward(g, m, q, r)
        h = cs_backward(H, m, q, p, r)
        acc += h if r == 0 else 2.0 * h.real
    if q % 2 == 0:
        r = q // 2
        H = cs_forward(f, m, q, r) * cs_forward(g, m, q, r)
        acc += cs_backward(H, m, q, p, r)
    return acc[: (L if K is None else K)] / (q * m)


# ---------------------------------------------------------------------------
# Sec. 4: implicit packing and the RCM operator (hybridRCM, explicitRCM)
# ---------------------------------------------------------------------------
def pack(f):
    """Eq. complexPacking: f~_j = f_{2j} + i f_{2j+1} (odd length: one zero)."""
    f = np.asarray(f, dtype=np.float64)
    if len(f) % 2:
        f = np.append(f, 0.0)
    return f[0::2] + 1j * f[1::2]


def unpack_real(ft, L):
    """Inverse of pack: the first L real values."""
    out = np.empty(2 * len(ft))
    out[0::2] = ft.real
    out[1::2] = ft.imag
    return out[:L]


def fourier_unpack(Ft):
    """Eq. fourierUnpack: U maps the DFT of the packing to F_k, k = 0..N."""
    N = len(Ft)
    k = np.arange(N + 1)
    Fk = Ft[k % N]
    Fc = np.conj(Ft[(N - k) % N])
    return 0.5 * (Fk + Fc) - 0.5j * (Fk - Fc) * zeta(2 * N, k)


def fourier_pack(F):
    """Eq. fourierPack: U^{-1} maps F_k (k = 0..N) back to F~_k, k = 0..N-1."""
    N = len(F) - 1
    k = np.arange(N)
    Fk = F[k]
    Fc = np.conj(F[N - k])
    return 0.5 * (Fk + Fc) + 0.5j * (Fk - Fc) * zeta(2 * N, -k)


def rcm_via_U(Ft, Gt):
    """Eq. RCM-U: U^{-1}(U(F~) . U(G~))."""
    return fourier_pack(fourier_unpack(Ft) * fourier_unpack(Gt))


def rcm(Ft, Gt):
    """Eq. RCM: (F~ [.] G~)_k = F~_k G~_k - 1/4 (F~_k - conj F~_{N-k})
    (G~_k - conj G~_{N-k})(1 + zeta_N^k), with F~_N = F~_0."""
    N = len(Ft)
    k = np.arange(N)
    kc = (N - k) % N
    return Ft * Gt - 0.25 * (Ft - np.conj(Ft[kc])) * (Gt - np.conj(Gt[kc])) * (1 + zeta(N, k))


def rcm_W(Ft, Gt, m, q, l, r):
    """W_{l,r} of Sec. 4 (definition before Eq. Hr), with F~ in natural order."""
    k = q * l + r
    kc = (q * m - k) % (q * m)
    return 0.25 * (Ft[k] - np.conj(Ft[kc])) * (Gt[k] - np.conj(Gt[kc])) * (1 + zeta(q * m, k))


def rcm_residue_pairs(Ft, Gt, m, q):
    """Eqs. Hr / Hr-conj: residues r and q-r together (r = 0, q/2 self-paired)."""
    H = np.zeros(q * m, dtype=np.complex128)
    for r in range(0, q // 2 + 1):
        rc = (q - r) % q
        if rc == r:
            for l in range(m):
                k = q * l + r
                H[k] = Ft[k] * Gt[k] - rcm_W(Ft, Gt, m, q, l, r)
        else:
            for l in range(m):
                k = q * l + r
                kc = q * (m - l - 1) + q - r
                Wlr = rcm_W(Ft, Gt, m, q, l, r)
                H[k] = Ft[k] * Gt[k] - Wlr
                H[kc] = Ft[kc] * Gt[kc] - np.conj(Wlr)
    return H


def rcm_valid(L, m, q):
    """Packed data of length ceil(L/2) need qm >= L (real length 2qm >= 2L-1)."""
    return q * m >= L


def conv_hybrid_rcm(f, g, m, q, K=None):
    """hybridRCM in 1D: pack, complex hybrid forward (Eq. forwardr), residue
    pairs by Eqs. Hr / Hr-conj, complex hybrid backward, unpack."""
    L = len(f)
    if not rcm_valid(L, m, q):
        raise ValueError("invalid (m, q) for hybridRCM")
    ft, gt = pack(f), pack(g)
    p = -(-len(ft) // m)
    Ft = hybrid_forward(ft, m, q)
    Gt = hybrid_forward(gt, m, q)
    H = rcm_residue_pairs(Ft, Gt, m, q)
    ht = hybrid_backward(H, m, q, p)
    return unpack_real(ht, L)[: (L if K is None else K)]


def mult_rcm(A, B, C, D, first):
    """Alg. 4 (multRCM): in place on A and C; M = len(A) even;
    Z_k = (1 + zeta_M^k)/4."""
    M = len(A)
    same = (A is C) or (B is D)
    if first:
        alpha = 0.5 * (A[0] - np.conj(C[0])) * (B[0] - np.conj(D[0]))
        A[0] = A[0] * B[0] - alpha
        if not same:
            C[0] = C[0] * D[0] - np.conj(alpha)
    for k in range(1, M // 2):
        Z = (1 + zeta(M, k)) / 4
        alpha = (A[k] - np.conj(C[M - k])) * (B[k] - np.conj(D[M - k])) * Z
        A[k] = A[k] * B[k] - alpha
        C[M - k] = C[M - k] * D[M - k] - np.conj(alpha)
    A[M // 2] = A[M // 2] * B[M // 2]


def conv_explicit(f, g):
    """explicit (Sec. 6): zero pad to M = 2L, real DFT, pointwise, inverse, crop."""
    L = len(f)
    M = 2 * L
    F = dft(np.pad(np.asarray(f, float), (0, M - L)), +1)
    G = dft(np.pad(np.asarray(g, float), (0, M - L)), +1)
    return (dft(F * G, -1).real / M)[:L]


def explicit_rcm_length(L):
    """Packed length of explicitRCM: Alg. 4 needs it even, so the real padded
    length 2L is rounded up to a multiple of 4 (packed length L rounded up to
    even)."""
    return L + (L % 2)


def conv_explicit_rcm(f, g):
    """Alg. 3 (convolveRCM1): zeroPad, complexPack, fft, multRCM, ifft, unpack."""
    L = len(f)
    M = explicit_rcm_length(L)
    ft = pack(np.pad(np.asarray(f, float), (0, 2 * M - L)))
    gt = pack(np.pad(np.asarray(g, float), (0, 2 * M - L)))
    Ft, Gt = dft(ft, +1), dft(gt, +1)
    mult_rcm(Ft, Gt, Ft, Gt, True)
    ht = dft(Ft, -1) / len(Ft)
    return unpack_real(ht, L)


# ---------------------------------------------------------------------------
# Sec. 5: multidimensional forms
# ---------------------------------------------------------------------------
def pack_last(f):
    """Eq. multidimComplexPacking: pack along the last dimension."""
    f = np.asarray(f, dtype=np.float64)
    if f.shape[-1] % 2:
        f = np.concatenate([f, np.zeros(f.shape[:-1] + (1,))], axis=-1)
    return f[..., 0::2] + 1j * f[..., 1::2]


def unpack_last(ht, Ln):
    out = np.empty(ht.shape[:-1] + (2 * ht.shape[-1],))
    out[..., 0::2] = ht.real
    out[..., 1::2] = ht.imag
    return out[..., :Ln]


def rcm_ndim(Ft, Gt):
    """Eq. RCM-ndim: k* = (M - k) mod M in every dimension and the factor
    (1 + zeta_{M_n}^{k_n}) of the last dimension."""
    idx = tuple((-np.arange(n)) % n for n in Ft.shape)
    Fc = np.conj(Ft[np.ix_(*idx)])
    Gc = np.conj(Gt[np.ix_(*idx)])
    Mn = Ft.shape[-1]
    fac = 1 + zeta(Mn, np.arange(Mn))
    return Ft * Gt - 0.25 * (Ft - Fc) * (Gt - Gc) * fac


def C_op(A, B, C, D):
    """The generalised operator C_n(A, B, C, D) of Sec. 5."""
    idx = tuple((-np.arange(n)) % n for n in A.shape)
    Cc = np.conj(C[np.ix_(*idx)])
    Dc = np.conj(D[np.ix_(*idx)])
    Mn = A.shape[-1]
    fac = 1 + zeta(Mn, np.arange(Mn))
    return A * B - 0.25 * (A - Cc) * (B - Dc) * fac


def _hybrid_forward_axis(x, m, q, axis):
    """Eq. forwardr applied along one axis of an array (complex hybrid)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    out = np.apply_along_axis(lambda v: hybrid_forward(v, m, q), -1, x)
    return np.moveaxis(out, -1, axis)


def _hybrid_backward_axis(X, m, q, p, axis):
    X = np.moveaxis(X, axis, -1)
    out = np.apply_along_axis(lambda v: hybrid_backward(v, m, q, p), -1, X)
    return np.moveaxis(out, -1, axis)


def conv_hybrid_rcm_nd(f, g, params, K=None):
    """hybridRCM in nD (Sec. 5): pack along the last dimension, complex hybrid
    forward along every dimension, the operator of Eq. RCM-ndim, hybrid
    backward, unpack.  ``params`` holds (m_i, q_i) per dimension; the last
    dimension is the packed one."""
    f = np.asarray(f, dtype=np.float64)
    d = f.ndim
    Ls = f.shape
    for ax in range(d - 1):
        m, q = params[ax]
        if q * m < 2 * Ls[ax] - 1:
            raise ValueError("outer dimensions need qm >= 2L-1")
    if not rcm_valid(Ls[-1], *params[-1]):
        raise ValueError("the packed dimension needs qm >= L")
    X, Y = pack_last(f), pack_last(g)
    for ax in range(d):
        m, q = params[ax]
        X = _hybrid_forward_axis(X, m, q, ax)
        Y = _hybrid_forward_axis(Y, m, q, ax)
    H = rcm_ndim(X, Y)
    for ax in range(d):
        m, q = params[ax]
        Lax = Ls[ax] if ax < d - 1 else -(-Ls[ax] // 2)
        p = -(-Lax // m)
        H = _hybrid_backward_axis(H, m, q, p, ax)
        H = np.take(H, np.arange(Lax), axis=ax)
    out = unpack_last(H, Ls[-1])
    if K is not None:
        out = out[tuple(slice(0, k) for k in K)]
    return out


def conv_explicit_rcm_2d(f, g):
    """Alg. 5 (convolveRCM2): zeroPad to M1 x 2M2 (M1 = 2L1; M2 = L2 rounded up
    to even for Alg. 4), pack along the last dimension, fftx, per k1 < M1/2 the
    pair (k1, k1*) with ffty, multRCM (Alg. 4), iffty, then ifftx and unpack."""
    f = np.asarray(f, float)
    L1, L2 = f.shape
    M1, M2 = 2 * L1, explicit_rcm_length(L2)
    fp = np.zeros((M1, 2 * M2))
    gp = np.zeros((M1, 2 * M2))
    fp[:L1, :L2] = f
    gp[:L1, :L2] = g
    Ft = dft(pack_last(fp), +1, axis=0)
    Gt = dft(pack_last(gp), +1, axis=0)
    for k1 in range(M1 // 2):
        k1s = M1 // 2 if k1 == 0 else M1 - k1
        for row in {k1, k1s}:
            Ft[row] = dft(Ft[row], +1)
            Gt[row] = dft(Gt[row], +1)
        A, B, C, D = Ft[k1], Gt[k1], Ft[k1s], Gt[k1s]
        if k1 == 0:
            mult_rcm(A, B, A, B, True)
            mult_rcm(C, D, C, D, True)
        else:
            mult_rcm(A, B, C, D, True)
            mult_rcm(C, D, A, B, False)
        Ft[k1], Gt[k1], Ft[k1s], Gt[k1s] = A, B, C, D
        for row in {k1, k1s}:
            Ft[row] = dft(Ft[row], -1) / M2
    ht = dft(Ft, -1, axis=0) / M1
    return unpack_last(ht, 2 * M2)[:L1, :L2]


def conv_hybrid_cs_nd(f, g, params, K=None):
    """hybridCS in nD (Sec. 5): the outermost (first) dimension is transformed
    with the real residues of Sec. 3.1; every inner dimension with complex
    hybrid dealiasing (Sec. 2); pointwise product; inverse in reverse order;
    Eq. real-accumulation along the first dimension."""
    f = np.asarray(f, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    d = f.ndim
    Ls = f.shape
    m0, q0 = params[0]
    if not cs_valid(Ls[0], m0, q0):
        raise ValueError("invalid outer (m, q) for hybridCS")
    p0 = -(-Ls[0] // m0)

    def inner_conv(Fr, Gr):
        X, Y = Fr, Gr
        for ax in range(1, d):
            m, q = params[ax]
            X = _hybrid_forward_axis(X, m, q, ax)
            Y = _hybrid_forward_axis(Y, m, q, ax)
        H = X * Y
        for ax in range(1, d):
            m, q = params[ax]
            p = -(-Ls[ax] // m)
            H = _hybrid_backward_axis(H, m, q, p, ax)
            H = np.take(H, np.arange(Ls[ax]), axis=ax)
        return H

    def fwd(x, r):
        return np.apply_along_axis(lambda v: cs_forward(v, m0, q0, r), 0, x)

    acc = np.zeros((p0 * m0,) + Ls[1:])
    residues = list(range((q0 + 1) // 2)) + ([q0 // 2] if q0 % 2 == 0 else [])
    for r in residues:
        H = inner_conv(fwd(f, r), fwd(g, r))
        if r == 0:
            h = np.apply_along_axis(lambda v: cs_backward(v, m0, q0, p0, 0), 0, H)
            acc += h.real
        elif 2 * r == q0:
            # the inner inverse of a real-input product keeps the half-length
            # packing of Eq. forwardq2 intact, so Eq. accumulateq2 applies
            acc += np.apply_along_axis(lambda v: cs_backward(v, m0, q0, p0, r), 0, H)
        else:
            h = np.apply_along_axis(lambda v: cs_backward(v, m0, q0, p0, r), 0, H)
            acc += 2.0 * h.real
    out = acc[: Ls[0]] / (q0 * m0)
    if K is not None:
        out = out[tuple(slice(0, k) for k in K)]
    return out


# ---------------------------------------------------------------------------
# App. A: the inner loop for many blocks -- the sums over the blocks t of
# Eq. forwardr, and the sum over the residues of Eq. accumulation, as q-point
# DFTs (the blocks t >= p are zero).  Used with the n-array product of Sec.
# 4.1 and the per-array block counts of Sec. 7.
# ---------------------------------------------------------------------------
def inner_loop_forward(x, m, q):
    """F[q l + r] = sum_s zeta_m^{ls} zeta_{qm}^{rs} sum_t zeta_q^{rt} x_{tm+s}:
    the sum over t as one q-point DFT of the q blocks (zero for t >= p)."""
    x = np.asarray(x, dtype=np.complex128)
    if len(x) > q * m:
        raise ValueError("more than q blocks")
    blocks = np.zeros((q, m), dtype=np.complex128)
    blocks.reshape(-1)[: len(x)] = x
    Y = dft(blocks, +1, axis=0)                      # Y[r][s] = sum_t zeta_q^{rt} x_t[s]
    r = np.arange(q)[:, None]
    s = np.arange(m)[None, :]
    Y = Y * zeta(q * m, r * s)                       # pre-twiddle zeta_{qm}^{rs}
    Fr = dft(Y, +1, axis=1)                          # Fr[r][l]
    F = np.empty(q * m, dtype=np.complex128)
    for rr in range(q):
        F[rr::q] = Fr[rr]                            # k = q l + r
    return F


def inner_loop_backward(H, m, q, K):
    """h_{tm+s} = sum_r zeta_q^{-rt} zeta_{qm}^{-rs} sum_l zeta_m^{-ls} H[q l + r]
    (Eqs. accumulator and accumulation, unscaled): the sum over r as one
    backward q-point DFT; the first K entries."""
    Hr = np.stack([H[rr::q] for rr in range(q)])   # Hr[r][l]
    w = dft(Hr, -1, axis=1)                          # w[r][s]
    r = np.arange(q)[:, None]
    s = np.arange(m)[None, :]
    v = w * zeta(q * m, -r * s)
    h = dft(v, -1, axis=0)                           # h[t][s]
    return h.reshape(-1)[:K]


def conv_rcm_inner_loop(xs, m, q, K=None):
    """x^1 * ... * x^n (real 1D arrays of any lengths) by implicit packing with
    the inner loop: pack each array, transform, R^1 = F^1 and R^j = R^{j-1} RCM F^j
    by the residue-pair formulas (Eqs. Akn, Rnk, RnMk: Eqs. Hr/Hr-conj with
    R^{j-1} in F's place), transform back, scale 1/(qm), unpack the first K
    (default max L_i).  Needs 2 q m >= sum L_i - n + 1."""
    Ls = [len(x) for x in xs]
    S = sum(Ls) - len(xs) + 1
    if 2 * q * m < S:
        raise ValueError("does not dealias")
    K = max(Ls) if K is None else K
    R = inner_loop_forward(pack(xs[0]), m, q)
    for x in xs[1:]:
        R = rcm_residue_pairs(R, inner_loop_forward(pack(x), m, q), m, q)
    ht = inner_loop_backward(R, m, q, (K + 1) // 2) / (q * m)
    return unpack_real(ht, K)


def conv_cs_inner_loop(f, g, m, q, K=None):
    """hybridCS with the inner loop for real f, g: the q-point DFT over the
    blocks of real data is Hermitian in r, so residues r <= q/2 are formed,
    multiplied pointwise and transformed back; the sum over r takes
    v_{q-r} = conj v_r (Eq. hrHerm), and the real part is the result (Eq.
    real-accumulation), scaled 1/(qm).  Needs q m >= 2L - 1."""
    L = len(f)
    if q * m < 2 * L - 1:
        raise ValueError("does not dealias")
    K = L if K is None else K
    F = inner_loop_forward(np.asarray(f, dtype=np.float64), m, q)
    G = inner_loop_forward(np.asarray(g, dtype=np.float64), m, q)
    H = np.zeros(q * m, dtype=np.complex128)
    for rr in range(q // 2 + 1):
        H[rr::q] = F[rr::q] * G[rr::q]
    Hr = np.stack([H[rr::q] for rr in range(q)])
    w = dft(Hr, -1, axis=1)
    r = np.arange(q)[:, None]
    s = np.arange(m)[None, :]
    v = w * zeta(q * m, -r * s)
    for rr in range(q // 2 + 1, q):
        v[rr] = np.conj(v[q - rr])                   # Eq. hrHerm
    h = dft(v, -1, axis=0).reshape(-1)[:K]
    return h.real / (q * m)
