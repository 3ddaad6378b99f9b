"""lp_solve_many: several LPs in one launch, a team of blocks per LP.

The team path runs the same Steps with the same arithmetic and tie rules as
lp_solve, so every LP's status, pivot count, x, y, objective and tableau equal
the oracle's (FP64, tolerance 0), and an FP32 solve equals lp_solve's FP32
solve of the same LP entry for entry.
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


SHAPES = [(1, 1), (1, 9), (9, 1), (3, 4), (37, 53), (64, 64), (200, 150), (150, 200), (300, 700),
          (700, 300), (1024, 512), (129, 257), (16, 2000), (2000, 16), (600, 1100)]


def _check(tsx, pr, ref, tableau=True):
    sol = pr.solution()
    assert sol.status == ref.status
    assert sol.iters == ref.iters
    assert sol.obj == ref.obj
    np.testing.assert_array_equal(sol.x, ref.x)
    np.testing.assert_array_equal(sol.y, ref.y)
    np.testing.assert_array_equal(sol.basis, ref.basis)
    if tableau:
        np.testing.assert_array_equal(pr.tableau(), ref.T)
    assert pr.stats()["path"] == tsx.LP_PATH_TEAM


@pytest.mark.parametrize("blocks", [0, 1, 2, 7, 64])
def test_mixed_lps_equal_the_oracle(tsx, blocks):
    problems = [lpgen.dense_lp(m, n, 70 + k) for k, (m, n) in enumerate(SHAPES)]
    refs = [oracle.solve(*p) for p in problems]
    prs = [tsx.Problem(*p) for p in problems]
    try:
        st = tsx.solve_many(prs, tsx.options(blocks=blocks))
        assert st == [r.status for r in refs]
        for pr, ref in zip(prs, refs):
            _check(tsx, pr, ref)
    finally:
        for pr in prs:
            pr.close()


def test_special_lps_and_rules(tsx):
    cyc = (np.array([[0.5, -5.5, -2.5, 9.0], [0.5, -1.5, -0.5, 1.0], [1.0, 0.0, 0.0, 0.0]]),
           np.array([0.0, 0.0, 1.0]), np.array([10.0, -57.0, -9.0, -24.0]))
    unb = (np.array([[1.0, -2.0], [1.0, 0.0]]), np.array([4.0, 3.0]), np.array([0.0, 1.0]))
    zero = (np.ones((3, 2)), np.array([1.0, 2.0, 3.0]), np.array([-1.0, -1.0]))
    A0, b0, c0 = lpgen.dense_lp(40, 30, 11)
    dup = (np.vstack([A0, A0[:10]]), np.concatenate([b0, b0[:10]]), c0)
    problems = [cyc, unb, zero, dup, lpgen.dense_lp(90, 60, 5)]
    for kw in ({"k_cyc": 3}, {"rule": 1}, {"max_iters": 4}, {}):
        refs = [oracle.solve(*p, oracle.Options(**kw)) for p in problems]
        prs = [tsx.Problem(*p) for p in problems]
        try:
            st = tsx.solve_many(prs, tsx.options(blocks=3, **kw))
            assert st == [r.status for r in refs], kw
            for pr, ref in zip(prs, refs):
                _check(tsx, pr, ref)
        finally:
            for pr in prs:
                pr.close()


def test_fp32_equals_single_lp_fp32(tsx):
    shapes = [(300, 200), (512, 512), (64, 700), (900, 400)]
    problems = [lpgen.dense_lp(m, n, 300 + k) for k, (m, n) in enumerate(shapes)]
    alone = []
    for p in problems:
        with tsx.Problem(*p) as pr:
            assert pr.solve(tsx.options(precision=tsx.LP_PREC_FP32)) == tsx.LP_OPTIMAL
            alone.append((pr.solution(), pr.tableau()))
    prs = [tsx.Problem(*p) for p in problems]
    try:
        st = tsx.solve_many(prs, tsx.options(precision=tsx.LP_PREC_FP32))
        assert st == [tsx.LP_OPTIMAL] * len(problems)
        for pr, (sol1, T1), p in zip(prs, alone, problems):
            sol = pr.solution()
            assert sol.obj == sol1.obj and sol.iters == sol1.iters
            np.testing.assert_array_equal(sol.x, sol1.x)
            np.testing.assert_array_equal(sol.y, sol1.y)
            np.testing.assert_array_equal(pr.tableau(), T1)
            ref = oracle.solve(*p)
            assert abs(sol.obj - ref.obj) <= 1e-9 * abs(ref.obj)
    finally:
        for pr in prs:
            pr.close()


def test_lp_beyond_team_shared_memory_falls_back(tsx):
    # n = 40000: the pivot row alone needs 320 KB, more than a block's shared memory
    problems = [lpgen.dense_lp(3, 40000, 1), lpgen.dense_lp(50, 40, 2)]
    refs = [oracle.solve(*p) for p in problems]
    prs = [tsx.Problem(*p) for p in problems]
    try:
        st = tsx.solve_many(prs)
        assert st == [r.status for r in refs]
        for pr, ref in zip(prs, refs):
            sol = pr.solution()
            assert sol.iters == ref.iters and sol.obj == ref.obj
            np.testing.assert_array_equal(sol.x, ref.x)
        assert prs[0].stats()["path"] != tsx.LP_PATH_TEAM
        assert prs[1].stats()["path"] == tsx.LP_PATH_TEAM
    finally:
        for pr in prs:
            pr.close()


def test_invalid_calls(tsx):
    p = tsx.Problem(*lpgen.dense_lp(5, 5, 1))
    try:
        rc, _ = tsx.lp_solve_many([p.h, p.h])
        assert rc == tsx.LP_ERR_INVALID and "twice" in tsx.lp_last_error()
        rc, _ = tsx.lp_solve_many([p.h], tsx.options(layout=tsx.LP_LAYOUT_FULL))
        assert rc == tsx.LP_ERR_INVALID
        rc, _ = tsx.lp_solve_many([p.h], tsx.options(log_capacity=10))
        assert rc == tsx.LP_ERR_INVALID
        rc, st = tsx.lp_solve_many([])
        assert rc == tsx.LP_OPTIMAL and st == []
    finally:
        p.close()


def test_team_barrier_timeout_reports_and_context_survives(tsx):
    # a zero wait budget: the teams give up at their first barrier (no hang);
    # every LP reports LP_ERR_TIMEOUT, and the next call on the same context is exact
    problems = [lpgen.dense_lp(m, n, 40 + k) for k, (m, n) in enumerate([(300, 200), (120, 500), (64, 900)])]
    refs = [oracle.solve(*p) for p in problems]
    prs = [tsx.Problem(*p) for p in problems]
    try:
        st = tsx.solve_many(prs, tsx.options(blocks=4, barrier_timeout_ns=0))
        assert all(s in (tsx.LP_ERR_TIMEOUT, tsx.LP_OPTIMAL) for s in st)
        assert tsx.LP_ERR_TIMEOUT in st
        st = tsx.solve_many(prs, tsx.options(blocks=4))
        assert st == [r.status for r in refs]
        for pr, ref in zip(prs, refs):
            _check(tsx, pr, ref)
    finally:
        for pr in prs:
            pr.close()


def test_device_inputs(tsx):
    import torch
    shapes = [(250, 300), (400, 180)]
    problems = [lpgen.dense_lp(m, n, 60 + k) for k, (m, n) in enumerate(shapes)]
    refs = [oracle.solve(*p) for p in problems]
    s = torch.cuda.current_stream().cuda_stream
    dev = [tuple(torch.from_numpy(v).cuda() for v in p) for p in problems]
    prs = [tsx.Problem(A, b, c, device=True, stream=s) for A, b, c in dev]
    try:
        st = tsx.solve_many(prs, tsx.options(stream=s))
        assert st == [r.status for r in refs]
        for pr, ref in zip(prs, refs):
            _check(tsx, pr, ref)
    finally:
        for pr in prs:
            pr.close()
