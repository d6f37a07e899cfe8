"""GPU parity of the batched 1D path (one launch over uneven lengths)."""
import numpy as np
import pytest

import oracle
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


def flat(Ls, seed):
    off = np.zeros(len(Ls), dtype=np.int64)
    off[1:] = np.cumsum(Ls)[:-1]
    f, g = inputs.normal_pair(int(np.sum(Ls)), seed)
    return off, f, g


@pytest.mark.parametrize("algo", ["hybridRCM", "hybridCS"])
def test_batched_small_every_item(hd, algo):
    rng = np.random.default_rng(40)
    Ls = np.concatenate([[1, 2, 3, 4, 5, 16, 17, 255, 256, 257], rng.integers(1, 20000, 54)]).astype(np.int64)
    off, f, g = flat(Ls, 41)
    plan = hd.BatchPlan(off, Ls, algo=algo)
    h = plan(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    ref = oracle.batch_conv1d(f, g, off, Ls)
    for i in range(len(Ls)):
        a, b = off[i], off[i] + Ls[i]
        assert rel_l2(h[a:b], ref[a:b]) <= TOL, (i, Ls[i])


@pytest.mark.parametrize("algo", ["hybridRCM", "hybridCS"])
def test_batched_equals_single_calls(hd, algo):
    Ls = np.array([700, 4096, 9999, 33333, 70000], dtype=np.int64)
    off, f, g = flat(Ls, 42)
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    hb = hd.BatchPlan(off, Ls, algo=algo)(tf, tg).cpu().numpy()
    for i in range(len(Ls)):
        a, b = off[i], off[i] + Ls[i]
        hs = hd.conv(tf[a:b].contiguous(), tg[a:b].contiguous(), algo=algo).cpu().numpy()
        ref = oracle.fft_conv(f[a:b].astype(np.float64), g[a:b].astype(np.float64))
        assert rel_l2(hb[a:b], ref) <= TOL
        assert rel_l2(hs, ref) <= TOL


def test_batched_full_workload_sampled(hd):
    """The benchmark's configuration (4096 items, L ~ U{500..70000}), sampled items."""
    off, Ls = inputs.batch_lengths(4096, 500, 70000, seed=2)
    f, g = inputs.batch_values(int(Ls.sum()), seed=3)
    plan = hd.BatchPlan(off, Ls, algo="hybridRCM")
    h = plan(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    hh = h.cpu().numpy()
    for i in [0, 1, 777, 2048, 3000, 4095] + list(np.argsort(Ls)[[0, -1]]):
        a, b = off[i], off[i] + Ls[i]
        ref = oracle.fft_conv(f[a:b].astype(np.float64), g[a:b].astype(np.float64))
        assert rel_l2(hh[a:b], ref) <= TOL, (i, Ls[i])
    # untouched gaps: nothing outside the items (there are none here) and no NaN
    assert np.isfinite(hh).all()


def test_autotune_table_matches_direct_timing(hd):
    """The planner's cost table must describe real launches: the entry it picks
    for L = 65536 (64 items, about the tuner's batch size) agrees with a CUDA-event
    timing of the same batch within a factor of two."""
    L, K = 65536, 64
    Ls = np.full(K, L, dtype=np.int64)
    off = np.arange(K, dtype=np.int64) * L
    f = torch.randn(K * L, device="cuda")
    g = torch.randn(K * L, device="cuda")
    h = torch.empty_like(f)
    plan = hd.BatchPlan(off, Ls, algo="hybridRCM")
    tab = hd.hd_tuning_table(hd.context())
    if not tab:
        pytest.skip("autotuner disabled (HD_AUTOTUNE=0)")
    assert all(us > 0 for _, _, us in tab)
    # the planner's rule: the cheapest measured instance whose 2 C m covers L
    best = None
    for C, m, us in tab:
        if 2 * C * m < L:
            continue
        if best is None or us < best[2]:
            best = (C, m, us)
    assert best is not None
    for _ in range(3):
        plan(f, g, out=h)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(10):
        plan(f, g, out=h)
    b.record()
    torch.cuda.synchronize()
    us_direct = 1e3 * a.elapsed_time(b) / (10 * K)
    assert 0.5 <= us_direct / best[2] <= 2.0, (best, us_direct)


@pytest.mark.parametrize("algo", ["hybridRCM", "hybridCS"])
def test_batched_in_place(hd, algo):
    """h may alias f: every item reads its inputs before writing its outputs."""
    rng = np.random.default_rng(43)
    Ls = rng.integers(300, 40000, 48).astype(np.int64)
    off, f, g = flat(Ls, 44)
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    plan = hd.BatchPlan(off, Ls, algo=algo)
    plan(tf, tg, out=tf)
    h = tf.cpu().numpy()
    ref = oracle.batch_conv1d(f, g, off, Ls, use_fft=True)
    for i in range(len(Ls)):
        a, b = off[i], off[i] + Ls[i]
        assert rel_l2(h[a:b], ref[a:b]) <= TOL, (i, Ls[i])


def test_batched_graph_replay_matches_eager(hd):
    """A plan whose items span several cluster sizes launches one kernel per size
    on streams forked from the caller's stream; captured in a CUDA graph and
    replayed, it must give the eager result bit for bit."""
    Ls = np.array([600, 1500, 9000, 17000, 30000, 52000, 69000, 2500, 40000, 12000] * 6, dtype=np.int64)
    off, f, g = flat(Ls, 45)
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    plan = hd.BatchPlan(off, Ls, algo="hybridRCM")
    assert 1 <= plan.launches <= 25  # one per (cluster size, residue length) class, plus the one-CTA kernel
    h_eager = plan(tf, tg).clone()
    h = torch.zeros_like(tf)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan(tf, tg, out=h)  # warm-up on the capture stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            plan(tf, tg, out=h)
    h.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(h, h_eager)
    ref = oracle.batch_conv1d(f, g, off, Ls, use_fft=True)
    hh = h.cpu().numpy()
    for i in range(0, len(Ls), 7):
        a, b = off[i], off[i] + Ls[i]
        assert rel_l2(hh[a:b], ref[a:b]) <= TOL, (i, Ls[i])


def test_batched_explicit_rcm_every_item(hd):
    """The explicit-padding baseline as a batched plan (padded copies in the plan)."""
    rng = np.random.default_rng(46)
    Ls = np.concatenate([[1, 2, 3, 500, 9216, 9217, 73728], rng.integers(1, 70000, 40)]).astype(np.int64)
    off, f, g = flat(Ls, 47)
    plan = hd.BatchPlan(off, Ls, algo="explicitRCM")
    tf, tg = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    h = plan(tf, tg).cpu().numpy()
    ref = oracle.batch_conv1d(f, g, off, Ls, use_fft=True)
    for i in range(len(Ls)):
        a, b = off[i], off[i] + Ls[i]
        assert rel_l2(h[a:b], ref[a:b]) <= TOL, (i, Ls[i])
    # graph replay gives the eager result
    h2 = torch.zeros_like(tf)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        plan(tf, tg, out=h2)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            plan(tf, tg, out=h2)
    h2.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(h2.cpu().numpy(), h)
