"""Batched solve (one block per LP, condensed tableau in shared memory) vs the
oracle, LP by LP.  The batch runs the same FP64 method with the same tie rules,
so every LP's status, pivot count, objective, x and y -- and its full tableau
rebuilt from the condensed one -- equal the oracle's (tolerance 0).
"""
import numpy as np
import pytest

import lpgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tsx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10979_gb300 import build
    build.build()
    import paper_2211_10979_gb300 as mod
    mod.use_torch_allocator()
    return mod


def _problems(shapes, seed0):
    return [lpgen.dense_lp(m, n, seed0 + k) for k, (m, n) in enumerate(shapes)]


def _check(batch_sol, problems, refs, idx=None):
    for k in (range(len(problems)) if idx is None else idx):
        ref = refs[k]
        assert batch_sol.status[k] == ref.status, k
        assert batch_sol.iters[k] == ref.iters, k
        assert batch_sol.obj[k] == ref.obj, k
        np.testing.assert_array_equal(batch_sol.x[k], ref.x)
        np.testing.assert_array_equal(batch_sol.y[k], ref.y)


MIXED = [(1, 1), (1, 9), (9, 1), (3, 4), (16, 16), (17, 31), (31, 17), (40, 64), (64, 40),
         (100, 128), (128, 100), (128, 128), (77, 91), (5, 120), (120, 5)]


@pytest.mark.parametrize("threads", [0, 32, 64, 128, 256, 512])
def test_mixed_batch_equals_oracle(tsx, threads):
    problems = _problems(MIXED, 500)
    refs = [oracle.solve(*p) for p in problems]
    with tsx.Batch(problems) as bt:
        bt.solve(tsx.batch_options(threads=threads, keep_tableaux=1))
        sol = bt.results()
        _check(sol, problems, refs)
        for k in (0, 4, 9, 11):
            np.testing.assert_array_equal(bt.tableau(k), refs[k].T)
        assert sol.stats["total_pivots"] == sum(r.iters for r in refs)


def test_graph_replay_and_direct_launch_agree(tsx):
    shapes = lpgen.batch_shapes(200, 16, 128, 3)
    problems = _problems(shapes, 900)
    refs = [oracle.solve(*p) for p in problems]
    with tsx.Batch(problems) as bt:
        for rep in range(4):   # the first solve launches directly, the second captures, later ones replay
            bt.solve(tsx.batch_options(threads=64))
            sol = bt.results()
            assert sol.stats["graph"] == (0 if rep == 0 else 1)
            _check(sol, problems, refs)
        bt.solve(tsx.batch_options(threads=64, use_graph=0))
        _check(bt.results(), problems, refs)


def test_config_4096_small_lps(tsx):
    # the batching workload: 4096 LPs, m and n uniform in [16, 128], FP64
    shapes = lpgen.batch_shapes(4096, 16, 128, 1)
    problems = _problems(shapes, 10_000)
    refs = [oracle.solve(*p) for p in problems]
    with tsx.Batch(problems) as bt:
        bt.solve()                     # autotuned threads per size class
        sol = bt.results()
    _check(sol, problems, refs)
    st = sol.stats
    assert sum(st["lps_per_class"]) == 4096
    assert all(t in (0, 32, 64, 128, 256, 512) for t in st["threads"])


def test_special_lps_inside_a_batch(tsx):
    cyc = (np.array([[0.5, -5.5, -2.5, 9.0], [0.5, -1.5, -0.5, 1.0], [1.0, 0.0, 0.0, 0.0]]),
           np.array([0.0, 0.0, 1.0]), np.array([10.0, -57.0, -9.0, -24.0]))
    unb = (np.array([[1.0, -2.0], [1.0, 0.0]]), np.array([4.0, 3.0]), np.array([0.0, 1.0]))
    zero = (np.ones((3, 2)), np.array([1.0, 2.0, 3.0]), np.array([-1.0, -1.0]))
    A0, b0, c0 = lpgen.dense_lp(20, 15, 7)
    bad = (A0, b0.copy(), c0)
    bad[1][3] = -1.0
    ok = lpgen.dense_lp(30, 25, 8)
    problems = [cyc, unb, zero, bad, ok]
    with tsx.Batch(problems) as bt:
        for kw in ({"k_cyc": 3}, {"rule": 1}, {}):
            bt.solve(tsx.batch_options(**kw))
            sol = bt.results()
            for k in (0, 1, 2, 4):
                ref = oracle.solve(*problems[k], oracle.Options(**kw))
                assert sol.status[k] == ref.status and sol.iters[k] == ref.iters and sol.obj[k] == ref.obj
            assert sol.status[3] == tsx.LP_ERR_INVALID


def test_device_inputs(tsx):
    import torch
    problems = _problems([(20, 30), (50, 10), (64, 64)], 77)
    refs = [oracle.solve(*p) for p in problems]
    m = np.array([p[0].shape[0] for p in problems], dtype=np.int32)
    n = np.array([p[0].shape[1] for p in problems], dtype=np.int32)
    dA = torch.from_numpy(np.concatenate([p[0].ravel() for p in problems])).cuda()
    db = torch.from_numpy(np.concatenate([p[1] for p in problems])).cuda()
    dc = torch.from_numpy(np.concatenate([p[2] for p in problems])).cuda()
    s = torch.cuda.current_stream().cuda_stream
    with tsx.Batch(m=m, n=n, A=dA, b=db, c=dc, device=True, stream=s) as bt:
        bt.solve(tsx.batch_options(stream=s))
        _check(bt.results(), problems, refs)


def test_page_locked_inputs(tsx):
    # page-locked packed inputs are read by one kernel over the host link; an
    # invalid LP in them is still reported per LP by the solve
    import torch
    problems = _problems([(20, 30), (50, 10), (64, 64), (7, 9)], 91)
    bad = list(problems[3])
    bad[1] = bad[1].copy()
    bad[1][2] = -1.0
    problems[3] = tuple(bad)
    refs = [oracle.solve(*p) for p in problems[:3]]
    m = np.array([p[0].shape[0] for p in problems], dtype=np.int32)
    n = np.array([p[0].shape[1] for p in problems], dtype=np.int32)
    pA, pb, pc = (torch.from_numpy(np.concatenate([np.ravel(p[k]) for p in problems])).pin_memory() for k in range(3))
    with tsx.Batch(m=m, n=n, A=pA, b=pb, c=pc) as bt:
        bt.solve(tsx.batch_options())
        sol = bt.results()
        _check(sol, problems[:3], refs)
        assert sol.status[3] == tsx.LP_ERR_INVALID


@pytest.mark.parametrize("threads", [0, 64, 256, 512])
def test_lps_beyond_shared_memory_use_global_workspace(tsx, threads):
    # condensed tableaux above the shared-memory limit (m = n = 200: 323 KB)
    # are solved from a global workspace slice, mixed with shared-memory ones
    problems = _problems([(200, 200), (40, 50), (300, 120), (129, 400), (64, 64), (500, 90)], 321)
    refs = [oracle.solve(*p) for p in problems]
    with tsx.Batch(problems) as bt:
        bt.solve(tsx.batch_options(threads=threads, keep_tableaux=1))
        sol = bt.results()
        _check(sol, problems, refs)
        np.testing.assert_array_equal(bt.tableau(0), refs[0].T)
        assert sol.stats["lps_per_class"][4] == 4


def test_invalid_sizes_refused(tsx):
    with pytest.raises(ValueError, match="m > 0"):
        tsx.Batch(m=np.array([0], np.int32), n=np.array([3], np.int32), A=np.zeros(0), b=np.zeros(0),
                  c=np.zeros(3))


def _tie_lps():
    """LPs whose Step 1 and Step 2 comparisons meet exact ties, signed zeros
    and zero ratios: duplicated rows and columns of a small integer matrix,
    equal costs, and two unit rows with right-hand sides -0.0 and +0.0."""
    rng = np.random.default_rng(77)
    out = []
    for h, n in ((3, 6), (6, 9), (20, 33), (35, 64)):
        A0 = rng.integers(1, 4, size=(h, n - 2)).astype(np.float64)
        A = np.vstack([A0, A0])                                  # every ratio appears twice
        A = np.hstack([A, A[:, 2:4]])                            # duplicated columns
        units = np.zeros((2, n))
        units[0, 0] = 1.0
        units[1, 1] = 2.0
        A = np.vstack([A, units])
        b = np.concatenate([np.tile(rng.integers(1, 5, size=h).astype(np.float64) * 4.0, 2), [-0.0, 0.0]])
        c = rng.integers(1, 3, size=n).astype(np.float64)       # equal reduced costs
        out.append((A, b, c))
    return out


@pytest.mark.parametrize("rule", [0, 1])
def test_ties_and_signed_zeros_inside_a_batch(tsx, rule):
    problems = _tie_lps()
    kw = {"rule": rule} if rule else {"k_cyc": 5}
    refs = [oracle.solve(*p, oracle.Options(**kw)) for p in problems]
    with tsx.Batch(problems) as bt:
        bt.solve(tsx.batch_options(keep_tableaux=1, **kw))
        sol = bt.results()
        _check(sol, problems, refs)
        for k in range(len(problems)):
            np.testing.assert_array_equal(bt.tableau(k), refs[k].T)


def _screen_lps():
    """LPs aimed at the single-precision screen of the ratio test: exact ties
    among more rows than a warp holds, ratios one ulp apart (inside the screen's
    band, so the exact division decides), and rows whose entries lie outside
    float's exponent range (they bypass the screen)."""
    out = []
    # 100 identical constraint rows in column 0: 100 tied candidates per pivot
    A = np.ones((100, 5))
    A[:, 1:] = np.linspace(0.5, 2.0, 4)
    out.append((A, np.full(100, 100.0), np.array([9.0, 1.0, 2.0, 3.0, 4.0])))
    # ratios b_i / A_i0 = 7 (1 + d_i 2^-50), d_i in 0..5: all within the band
    rng = np.random.default_rng(11)
    m, n = 60, 8
    A = rng.integers(1, 9, size=(m, n)).astype(np.float64) / 4.0
    d = rng.integers(0, 6, size=m)
    b = A[:, 0] * 7.0 * (1.0 + d * 2.0 ** -50)
    c = np.concatenate([[10.0], np.ones(n - 1)])
    out.append((A, b, c))
    # rows scaled by 2^300 and 2^-300 (ratios unchanged; no float estimate)
    A, b, c = lpgen.dense_lp(40, 30, 21)
    A, b = A.copy(), b.copy()
    A[:10] *= 2.0 ** 300
    b[:10] *= 2.0 ** 300
    A[10:20] *= 2.0 ** -300
    b[10:20] *= 2.0 ** -300
    out.append((A, b, c))
    # a zero right-hand side (ratio 0, degenerate) next to ordinary rows
    A, b, c = lpgen.dense_lp(50, 50, 22)
    b = b.copy()
    b[[3, 17, 40]] = 0.0
    out.append((A, b, c))
    return out


@pytest.mark.parametrize("threads", [32, 128, 512])
@pytest.mark.parametrize("rule", [0, 1])
def test_ratio_screen_edge_cases(tsx, threads, rule):
    problems = _screen_lps()
    kw = {"rule": rule} if rule else {"k_cyc": 5}
    refs = [oracle.solve(*p, oracle.Options(**kw)) for p in problems]
    with tsx.Batch(problems) as bt:
        bt.solve(tsx.batch_options(threads=threads, keep_tableaux=1, **kw))
        sol = bt.results()
        _check(sol, problems, refs)
        for k in range(len(problems)):
            np.testing.assert_array_equal(bt.tableau(k), refs[k].T)
