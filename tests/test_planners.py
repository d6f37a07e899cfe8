"""Host-only checks of the planners inside libhdconv.so (no GPU): the
three-kernel path's (M, q) rule and the cluster choices for single calls and
for batches, called through their exported C++ entry points."""
import ctypes

import pytest

import paper_2608_14497_b300 as hd
from paper_2608_14497_b300 import build as hdbuild

# residue lengths of stage B and of the cluster kernel (256 R3), per cluster size
STAGE_B_M = (512, 1024, 2048, 4096, 4608)
CLUSTER_R3 = {1: (1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 16, 18), 2: (10, 12, 16, 18), 4: (5, 6, 8, 9, 10, 12, 16, 18),
              8: (5, 6, 8, 9, 10, 12, 16, 18), 16: (5, 6, 8, 9)}


@pytest.fixture(scope="module")
def lib():
    hdbuild.build()
    lb = ctypes.CDLL(hd.LIB_PATH)
    fns = {
        "staged": ("_ZN2hd13staged_paramsElPiS0_", [ctypes.c_int64] + [ctypes.POINTER(ctypes.c_int)] * 2),
        "single": ("_ZN2hd21cluster_params_singleElPiS0_S0_", [ctypes.c_int64] + [ctypes.POINTER(ctypes.c_int)] * 3),
        "instance": ("_ZN2hd16cluster_instanceEii", [ctypes.c_int, ctypes.c_int]),
        "choose_W": ("_ZN2hd8choose_WEmillmbli", [ctypes.c_size_t, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.c_size_t, ctypes.c_bool, ctypes.c_int64, ctypes.c_int]),
    }
    out = {}
    for key, (sym, args) in fns.items():
        f = getattr(lb, sym)
        f.argtypes = args
        f.restype = ctypes.c_int if key == "choose_W" else ctypes.c_bool
        out[key] = f
    return out


def staged(lib, n):
    M, q = ctypes.c_int(), ctypes.c_int()
    ok = lib["staged"](n, ctypes.byref(M), ctypes.byref(q))
    return ok, M.value, q.value


LENGTHS = [1, 2, 100, 2047, 2048, 2049, 5000, 8191, 16383, 16384, 16385, 32767, 32768, 32769, 73729, 100000, (1 << 17) - 1, 1 << 17, (1 << 17) + 1, 200000, 262144, 262145, 500000,
           524288, 1000000, 1048576, 2000000, 3000000, 4000000, 4194304, 4718592]


@pytest.mark.parametrize("n", LENGTHS)
def test_staged_params_rule(lib, n):
    ok, M, q = staged(lib, n)
    assert ok
    assert M in STAGE_B_M and q % 2 == 0 and 2 <= q <= 1024 and M * q >= n
    if n <= 16384:
        assert q == 4 and M == min(mm for mm in (512, 1024, 2048, 4096) if 4 * mm >= n)
    elif n <= 32768:
        assert (M, q) == (4096, 8)
    else:
        # the compile-time q lengths, the smallest N, the larger M on ties
        assert q in (256, 512, 1024)
        Ns = [qq * mm for qq in (256, 512, 1024) for mm in STAGE_B_M if qq * mm >= n]
        assert M * q == min(Ns)
        assert M == max(mm for qq in (256, 512, 1024) for mm in STAGE_B_M if qq * mm == M * q)


def test_staged_params_limit(lib):
    assert staged(lib, 1024 * 4608)[0]
    assert not staged(lib, 1024 * 4608 + 1)[0]


@pytest.mark.parametrize("L", [1, 2, 3, 511, 512, 513, 1000, 4096, 4097, 4608, 4609, 8192, 9000, 16384, 20000,
                               32768, 40000, 65536, 73727, 73728])
def test_single_call_cluster_choice(lib, L):
    C, m, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib["single"](L, ctypes.byref(C), ctypes.byref(m), ctypes.byref(p))
    C, m, p = C.value, m.value, p.value
    assert m % 256 == 0 and m // 256 in CLUSTER_R3[C] and lib["instance"](C, m)
    assert 2 * C * m >= L                        # q = 2C residues of m packed values cover L
    assert p == -(-((L + 1) // 2) // m) and 1 <= p <= C
    if L <= 4608:
        assert C == 1                            # one CTA while it fits: no exchange cost


def test_single_call_beyond_the_cluster_kernel(lib):
    C, m, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert not lib["single"](73729, ctypes.byref(C), ctypes.byref(m), ctypes.byref(p))
    assert not lib["single"](0, ctypes.byref(C), ctypes.byref(m), ctypes.byref(p))


@pytest.mark.parametrize("even", [False, True])
def test_column_strip_width(lib, even):
    """Strip widths of the column passes: a power of two <= 8 for every block
    shape (the strip loops split the element index with a shift and a mask),
    even for the paired real columns, at most B otherwise unless B < 1, and
    within the shared-memory and point limits."""
    smem, pts_max, sms = 232448, 4096, 148
    for per_col in (8 * 400, 8 * 1200, 8 * 4000, 8 * 20000):
        for pts in (16, 192, 384, 1024, 3072):
            for A in (1, 3, 24, 300, 768, 4096):
                for B in (1, 2, 3, 5, 6, 7, 8, 9, 15, 49, 190, 1500, 73728):
                    W = lib["choose_W"](per_col, pts, A, B, smem, even, pts_max, sms)
                    assert W in (1, 2, 4, 8), (per_col, pts, A, B, even, W)
                    if even:
                        assert W >= 2
                    else:
                        assert W <= B
                        if W > 1:
                            assert W * per_col <= smem and W * pts <= pts_max
