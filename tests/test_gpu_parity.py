"""CUDA path vs the CPU oracle, through the C ABI (needs a GPU).

FP64 parity bar (from the arithmetic both sides share: IEEE division for the
pivot row and ratios, one fused multiply-add per updated entry, comparisons
only in the reductions): the pivot sequence, the final basis and every entry
of the tableau are EQUAL to the oracle's (tolerance 0); x, y and the objective
are copies of tableau entries and are equal too.
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


def _gpu_run(tsx, A, b, c, **kw):
    kw.setdefault("log_capacity", 100000)
    with tsx.Problem(A, b, c) as pr:
        st = pr.solve(tsx.options(**kw))
        sol = pr.solution()
        T = pr.tableau()
        q, p = pr.pivot_log(kw["log_capacity"])
        return st, sol, T, q, p, pr.stats()


def _oracle_run(A, b, c, **kw):
    return oracle.solve(A, b, c, oracle.Options(**kw))


def _assert_same(gpu, ref):
    st, sol, T, q, p, _ = gpu
    assert st == ref.status, (st, ref.status)
    assert sol.iters == ref.iters
    np.testing.assert_array_equal(q, ref.qlog[:len(q)])
    np.testing.assert_array_equal(p, ref.plog[:len(p)])
    np.testing.assert_array_equal(sol.basis, ref.basis)
    np.testing.assert_array_equal(T, ref.T)
    np.testing.assert_array_equal(sol.x, ref.x)
    np.testing.assert_array_equal(sol.y, ref.y)
    assert sol.obj == ref.obj


SHAPES = [(1, 1), (1, 7), (7, 1), (3, 4), (16, 16), (37, 53), (64, 64), (100, 300),
          (300, 100), (129, 257), (256, 256), (1024, 1024), (512, 2048)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("layout", [0, 1])
def test_full_solve_bit_exact(tsx, m, n, path, layout):
    # layout 0: condensed device tableau (nonbasic columns + RHS), 1: Table I itself
    A, b, c = lpgen.dense_lp(m, n, 1 + m + n)
    ref = _oracle_run(A, b, c)
    _assert_same(_gpu_run(tsx, A, b, c, path=path, layout=layout), ref)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6, 7, 8])
def test_config_256_seeds(tsx, seed):
    A, b, c = lpgen.dense_lp(256, 256, seed)
    ref = _oracle_run(A, b, c)
    assert ref.status == oracle.OPTIMAL
    _assert_same(_gpu_run(tsx, A, b, c), ref)


@pytest.mark.parametrize("layout,skip", [(0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("threads,blocks", [(128, 1), (256, 2), (512, 3), (256, 7), (256, 0)])
def test_launch_shapes_agree(tsx, layout, skip, threads, blocks):
    A, b, c = lpgen.dense_lp(300, 200, 11)
    ref = _oracle_run(A, b, c)
    _assert_same(_gpu_run(tsx, A, b, c, layout=layout, skip_zero_columns=skip, threads=threads, blocks=blocks),
                 ref)


@pytest.mark.parametrize("k", [0, 1, 2, 5, 17])
@pytest.mark.parametrize("layout", [0, 1])
def test_tableau_after_k_pivots(tsx, k, layout):
    A, b, c = lpgen.dense_lp(200, 150, 21)
    ref = _oracle_run(A, b, c, max_iters=k)
    st, sol, T, q, p, _ = _gpu_run(tsx, A, b, c, max_iters=k, layout=layout)
    assert st == ref.status == oracle.ITER_LIMIT
    assert sol.iters == k
    np.testing.assert_array_equal(T, ref.T)


def test_golden_hand_traces(tsx, golden_dir):
    import json
    import os
    for name in ("two_pivots_dyadic.json", "one_pivot.json", "unbounded_after_one.json"):
        g = json.load(open(os.path.join(golden_dir, name)))
        A = np.array(g["A"], dtype=np.float64)
        b = np.array(g["b"], dtype=np.float64)
        c = np.array(g["c"], dtype=np.float64)
        for path, layout in ((1, 0), (2, 0), (4, 0), (1, 1), (2, 1)):
            st, sol, T, q, p, _ = _gpu_run(tsx, A, b, c, path=path, layout=layout)
            assert tsx.STATUS_NAMES[st] == g["status"]
            assert q.tolist() == [s["q"] for s in g["steps"]]
            assert p.tolist() == [s["p"] for s in g["steps"]]
            np.testing.assert_array_equal(T, np.array(g["steps"][-1]["T"], dtype=np.float64))
            assert sol.obj == g["obj"]


def test_cycling_lp_bland_fallback(tsx):
    A = np.array([[0.5, -5.5, -2.5, 9.0], [0.5, -1.5, -0.5, 1.0], [1.0, 0.0, 0.0, 0.0]])
    b = np.array([0.0, 0.0, 1.0])
    c = np.array([10.0, -57.0, -9.0, -24.0])
    for kw in ({"k_cyc": 3}, {"k_cyc": 50}, {"rule": 1}, {"k_cyc": 0, "max_iters": 200}):
        ref = _oracle_run(A, b, c, **kw)
        for path, layout in ((1, 0), (1, 1), (2, 0), (2, 1), (4, 0)):
            _assert_same(_gpu_run(tsx, A, b, c, path=path, layout=layout, **kw), ref)


def test_unbounded_and_zero_objective(tsx):
    A = np.array([[1.0, -2.0], [1.0, 0.0]])
    b = np.array([4.0, 3.0])
    c = np.array([0.0, 1.0])
    _assert_same(_gpu_run(tsx, A, b, c), _oracle_run(A, b, c))
    A, b, _ = lpgen.dense_lp(5, 4, 3)
    c = -np.ones(4)
    _assert_same(_gpu_run(tsx, A, b, c), _oracle_run(A, b, c))


def test_degenerate_duplicate_rows(tsx):
    A0, b0, c = lpgen.dense_lp(40, 30, 11)
    A = np.vstack([A0, A0[:10], np.ones((3, 30))])
    b = np.concatenate([b0, b0[:10], np.full(3, 50.0)])
    _assert_same(_gpu_run(tsx, A, b, c), _oracle_run(A, b, c))


def test_device_inputs_match_host_inputs(tsx):
    import torch
    A, b, c = lpgen.dense_lp(120, 90, 5)
    ref = _oracle_run(A, b, c)
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    s = torch.cuda.current_stream().cuda_stream
    with tsx.Problem(dA, db, dc, device=True, stream=s) as pr:
        assert pr.solve(tsx.options(stream=s)) == tsx.LP_OPTIMAL
        sol = pr.solution()
        np.testing.assert_array_equal(pr.tableau(), ref.T)
        np.testing.assert_array_equal(sol.x, ref.x)
        # a second solve on the same handle starts over and repeats the result
        assert pr.solve() == tsx.LP_OPTIMAL
        np.testing.assert_array_equal(pr.tableau(), ref.T)


def test_invalid_inputs_rejected_on_device(tsx):
    A, b, c = lpgen.dense_lp(4, 3, 1)
    bad_b = b.copy()
    bad_b[2] = -1.0
    with pytest.raises(ValueError, match="b >= 0"):
        tsx.Problem(A, bad_b, c)
    bad_A = A.copy()
    bad_A[1, 1] = np.nan
    with pytest.raises(ValueError, match="finite"):
        tsx.Problem(bad_A, b, c)
    with pytest.raises(ValueError, match="finite"):
        tsx.Problem(A, b, np.array([1.0, np.inf, 2.0]))


@pytest.mark.parametrize("m,n,offset", [(37, 53, 0), (37, 53, 1), (64, 64, 0), (1, 1, 0)])
def test_page_locked_inputs_read_by_the_gpu(tsx, m, n, offset):
    # page-locked A, b, c: one kernel reads them over the host link and checks
    # them (odd m*n: the 16-byte loop's tail; offset 1: 8-byte aligned A, the
    # element-wise loop); the solve equals the oracle's exactly
    import torch
    A, b, c = lpgen.dense_lp(m, n, 11 + m + n)
    buf = torch.empty(m * n + offset, dtype=torch.float64).pin_memory()
    buf[offset:] = torch.from_numpy(A.ravel())
    pA = buf[offset:]
    pb, pc = torch.from_numpy(b).pin_memory(), torch.from_numpy(c).pin_memory()
    ref = _oracle_run(A, b, c)
    h = tsx.lp_create(m, n, pA, pb, pc)
    try:
        assert tsx.lp_solve(h, tsx.options()) == ref.status
        s = tsx.lp_get_stats(h)
        assert s.create_copy_ms > 0 and s.create_check_ms == 0.0
        T = np.empty_like(ref.T)
        assert tsx.lp_get_tableau(h, T) == 0
        np.testing.assert_array_equal(T, ref.T)
    finally:
        tsx.lp_destroy(h)
    # b page-locked, A pageable: the copy-and-check path
    h = tsx.lp_create(m, n, A, pb, pc)
    try:
        tsx.lp_solve(h, tsx.options())
        assert tsx.lp_get_stats(h).create_check_ms > 0
    finally:
        tsx.lp_destroy(h)


def test_page_locked_inputs_checked(tsx):
    import torch
    A, b, c = lpgen.dense_lp(5, 4, 3)
    pin = lambda v: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
    bad_b = b.copy()
    bad_b[4] = -1e-300
    with pytest.raises(ValueError, match="b >= 0"):
        tsx.lp_create(5, 4, pin(A), pin(bad_b), pin(c))
    zero_b = b.copy()
    zero_b[0] = -0.0   # -0 >= 0
    h = tsx.lp_create(5, 4, pin(A), pin(zero_b), pin(c))
    tsx.lp_destroy(h)
    for k, v in [(0, np.nan), (19, np.inf), (7, -np.inf)]:
        bad_A = A.copy().ravel()
        bad_A[k] = v
        with pytest.raises(ValueError, match="finite"):
            tsx.lp_create(5, 4, pin(bad_A), pin(b), pin(c))
    bad_c = c.copy()
    bad_c[3] = np.nan
    with pytest.raises(ValueError, match="finite"):
        tsx.lp_create(5, 4, pin(A), pin(b), pin(bad_c))


def test_state_errors(tsx):
    A, b, c = lpgen.dense_lp(4, 3, 1)
    with tsx.Problem(A, b, c) as pr:
        assert tsx.lp_get_solution(pr.h)[0] == tsx.LP_ERR_STATE
        assert tsx.lp_solve(pr.h, tsx.options(threads=96)) == tsx.LP_ERR_INVALID
        assert tsx.lp_solve(pr.h, tsx.options(eps_d=-1.0)) == tsx.LP_ERR_INVALID


def test_barrier_timeout_reports_and_context_survives(tsx):
    # a zero wait budget makes every barrier wait expire at once: the kernel
    # must report LP_ERR_TIMEOUT (no trap, no hang) and later solves still work
    A, b, c = lpgen.dense_lp(256, 256, 1)
    with tsx.Problem(A, b, c) as pr:
        st = tsx.lp_solve(pr.h, tsx.options(path=1, blocks=8, barrier_timeout_ns=0))
        assert st == tsx.LP_ERR_TIMEOUT
        assert "barrier" in tsx.lp_last_error()
        assert pr.solve() == tsx.LP_OPTIMAL
        np.testing.assert_array_equal(pr.tableau(), _oracle_run(A, b, c).T)


@pytest.mark.parametrize("layout", [0, 1])
def test_stats_account_for_the_update(tsx, layout):
    A, b, c = lpgen.dense_lp(256, 256, 2)
    st, sol, T, q, p, stats = _gpu_run(tsx, A, b, c, layout=layout)
    m, n = 256, 256
    W = n + m + 1
    ld, it = stats["ld"], sol.iters
    assert stats["layout"] == layout
    assert stats["iters"] == it > 0
    assert stats["dense_update_bytes"] == 2.0 * (m + 1) * W * 8 * it
    side = (64.0 * (m + 1) + 24.0 * ld) * it
    if layout == 0:
        # condensed: every 32-byte group of the (n + 1)-wide rows is updated
        assert ld == -(-(n + 1) // 16) * 16
        assert stats["update_bytes"] == (64.0 * (m - 1) + 96.0) * (ld // 4) * it + side
    else:
        assert ld == -(-W // 16) * 16
        assert 0 < stats["update_bytes"] <= 2.0 * (m + 1) * ld * 8 * it + side
    assert stats["pivot_ms"] > 0 and stats["kernel_launches"] >= 3


def test_create_timings(tsx):
    # lp_create times its own copy and input check (device) and the whole
    # call (host); a handle over device inputs copies nothing
    import torch
    A, b, c = lpgen.dense_lp(512, 384, 5)
    h = tsx.lp_create(512, 384, A, b, c)
    try:
        assert tsx.lp_solve(h, tsx.options(max_iters=3)) in (tsx.LP_OPTIMAL, tsx.LP_ITER_LIMIT)
        s = tsx.lp_get_stats(h)
        assert s.create_copy_ms > 0 and s.create_check_ms > 0
        assert s.create_wall_ms >= s.create_copy_ms + s.create_check_ms
    finally:
        tsx.lp_destroy(h)
    dev = [torch.from_numpy(v).cuda() for v in (A, b, c)]
    h = tsx.lp_create_device(512, 384, *dev)
    try:
        tsx.lp_solve(h, tsx.options(max_iters=3))
        s = tsx.lp_get_stats(h)
        assert s.create_copy_ms == s.create_check_ms == s.create_wall_ms == 0.0
    finally:
        tsx.lp_destroy(h)


# the cluster path (LP_PATH_CLUSTER, chosen by default for FP64 condensed LPs
# that fit one cluster's shared memory): shapes around the row split (16 rows
# per block, clusters of 1-16 blocks) and the largest that fit
CLUSTER_SHAPES = [(1, 1), (1, 7), (7, 1), (3, 4), (16, 16), (17, 33), (33, 17), (37, 53), (64, 64),
                  (100, 300), (300, 100), (129, 257), (256, 256), (255, 511), (511, 255), (600, 600)]


@pytest.mark.parametrize("m,n", CLUSTER_SHAPES)
def test_cluster_path_bit_exact(tsx, m, n):
    A, b, c = lpgen.dense_lp(m, n, 7 + m + 3 * n)
    ref = _oracle_run(A, b, c)
    run = _gpu_run(tsx, A, b, c, path=tsx.LP_PATH_CLUSTER)
    _assert_same(run, ref)
    stats = run[5]
    assert stats["path"] == tsx.LP_PATH_CLUSTER and 1 <= stats["grid"] <= 16
    # the default path picks the cluster for these sizes
    assert _gpu_run(tsx, A, b, c)[5]["path"] == tsx.LP_PATH_CLUSTER


@pytest.mark.parametrize("kw", [{"k_cyc": 3}, {"rule": 1}, {"max_iters": 7}, {"eps_p": 0.0, "eps_d": 0.0}])
def test_cluster_path_options(tsx, kw):
    A, b, c = lpgen.dense_lp(200, 150, 31)
    ref = _oracle_run(A, b, c, **kw)
    _assert_same(_gpu_run(tsx, A, b, c, path=tsx.LP_PATH_CLUSTER, **kw), ref)
    A0, b0, c0 = lpgen.dense_lp(40, 30, 11)
    A = np.vstack([A0, A0[:10], np.ones((3, 30))])
    b = np.concatenate([b0, b0[:10], np.full(3, 50.0)])
    _assert_same(_gpu_run(tsx, A, b, c0, path=tsx.LP_PATH_CLUSTER, **kw), _oracle_run(A, b, c0, **kw))


def test_cluster_path_unbounded_zero_and_refusals(tsx):
    A = np.array([[1.0, -2.0], [1.0, 0.0]])
    b = np.array([4.0, 3.0])
    c = np.array([0.0, 1.0])
    _assert_same(_gpu_run(tsx, A, b, c, path=tsx.LP_PATH_CLUSTER), _oracle_run(A, b, c))
    A, b, _ = lpgen.dense_lp(5, 4, 3)
    _assert_same(_gpu_run(tsx, A, b, -np.ones(4), path=tsx.LP_PATH_CLUSTER), _oracle_run(A, b, -np.ones(4)))
    # refused: the Table I layout, a float tableau, an LP too large for a cluster
    A, b, c = lpgen.dense_lp(64, 64, 3)
    with tsx.Problem(A, b, c) as pr:
        for kw in ({"layout": tsx.LP_LAYOUT_FULL}, {"precision": tsx.LP_PREC_FP32}):
            assert tsx.lp_solve(pr.h, tsx.options(path=tsx.LP_PATH_CLUSTER, **kw)) == tsx.LP_ERR_INVALID
            assert "cluster" in tsx.lp_last_error()
    A, b, c = lpgen.dense_lp(1024, 1024, 3)
    with tsx.Problem(A, b, c) as pr:
        assert tsx.lp_solve(pr.h, tsx.options(path=tsx.LP_PATH_CLUSTER)) == tsx.LP_ERR_INVALID
        assert pr.solve() == tsx.LP_OPTIMAL
        assert pr.stats()["path"] == tsx.LP_PATH_PERSISTENT
