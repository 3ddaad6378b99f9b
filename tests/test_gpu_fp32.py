"""The FP32 path (float tableau for every pivot, FP64 recovery on the GPU).

Two bars:
  - the float pivots equal the float variant of the oracle step by step
    (tableau entries and (q, p) pairs identical: same operations, same order);
  - the recovered result equals the FP64 oracle's: objective within 1e-9
    relative, x and y within 1e-9 relative to their scale, and primal/dual
    feasibility violations at most 1e-9 (times 1 + |b| or 1 + |c|).
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


def _run(tsx, A, b, c, **kw):
    kw.setdefault("log_capacity", 100000)
    kw.setdefault("precision", tsx.LP_PREC_FP32)
    with tsx.Problem(A, b, c) as pr:
        st = pr.solve(tsx.options(**kw))
        sol = pr.solution()
        T = pr.tableau()
        q, p = pr.pivot_log(kw["log_capacity"])
        return st, sol, T, q, p, pr.stats()


def _violations(A, b, c, x, y):
    pv = max(0.0, float(np.max((A @ x - b) / (1.0 + np.abs(b)))), float(-x.min()))
    dv = max(0.0, float(np.max((c - A.T @ y) / (1.0 + np.abs(c)))), float(-y.min()))
    return pv, dv


def _assert_matches_fp64(A, b, c, sol, ref, tol=1e-9):
    assert abs(sol.obj - ref.obj) <= tol * abs(ref.obj)
    scale_x = max(1.0, float(np.abs(ref.x).max()))
    scale_y = max(1.0, float(np.abs(ref.y).max()))
    assert np.abs(sol.x - ref.x).max() <= tol * scale_x
    assert np.abs(sol.y - ref.y).max() <= tol * scale_y
    pv, dv = _violations(A, b, c, sol.x, sol.y)
    assert pv <= tol and dv <= tol
    assert abs(c @ sol.x - b @ sol.y) <= tol * abs(ref.obj)


@pytest.mark.parametrize("m,n", [(1, 5), (7, 3), (37, 53), (100, 300), (256, 256), (300, 100)])
def test_float_pivots_equal_float_oracle(tsx, m, n):
    A, b, c = lpgen.dense_lp(m, n, 100 + m + n)
    st32, it32, qref, pref, Tref, bref = oracle.solve32(A, b, c)
    st, sol, T, q, p, stats = _run(tsx, A, b, c)
    assert stats["pivot_status"] == st32 and stats["iters"] == it32
    np.testing.assert_array_equal(q, qref)
    np.testing.assert_array_equal(p, pref)
    np.testing.assert_array_equal(T, Tref.astype(np.float64))


@pytest.mark.parametrize("k", [1, 3, 11])
def test_float_tableau_after_k_pivots(tsx, k):
    A, b, c = lpgen.dense_lp(200, 150, 21)
    st32, it32, qref, pref, Tref, bref = oracle.solve32(A, b, c, oracle.Options(eps_d=1e-5, eps_p=1e-6,
                                                                                 max_iters=k))
    st, sol, T, q, p, stats = _run(tsx, A, b, c, max_iters=k)
    assert stats["pivot_status"] == oracle.ITER_LIMIT == st32
    np.testing.assert_array_equal(T, Tref.astype(np.float64))


@pytest.mark.parametrize("m,n,seed", [(16, 16, 1), (64, 64, 2), (256, 256, 1), (256, 256, 3),
                                      (1024, 1024, 1), (512, 2048, 2), (2048, 512, 3)])
def test_recovered_result_equals_fp64_oracle(tsx, m, n, seed):
    A, b, c = lpgen.dense_lp(m, n, seed)
    ref = oracle.solve(A, b, c)
    st, sol, T, q, p, stats = _run(tsx, A, b, c)
    assert st == tsx.LP_OPTIMAL == ref.status
    _assert_matches_fp64(A, b, c, sol, ref)
    assert stats["k"] == int((ref.basis < n).sum())
    assert sorted(sol.basis.tolist()) == sorted(ref.basis.tolist())
    assert stats["primal_violation"] <= 1e-9 and stats["dual_violation"] <= 1e-9
    assert stats["recover_ms"] > 0


@pytest.mark.parametrize("k", [0, 2, 7])
def test_primal_cleanup_finishes_a_stopped_float_phase(tsx, k):
    # the float phase stops after k pivots; FP64 cleanup pivots (revised form)
    # must carry the basis to the optimum
    A, b, c = lpgen.dense_lp(120, 90, 7)
    ref = oracle.solve(A, b, c)
    st, sol, T, q, p, stats = _run(tsx, A, b, c, max_iters=k)
    assert stats["pivot_status"] == tsx.LP_ITER_LIMIT
    assert st == tsx.LP_OPTIMAL
    assert stats["cleanup_pivots"] > 0
    _assert_matches_fp64(A, b, c, sol, ref)


def test_dual_cleanup_repairs_an_infeasible_basis(tsx):
    # a float ratio test that ignores entries below 3 picks wrong leaving rows,
    # so the float basis is primal infeasible; dual cleanup pivots repair it
    A, b, c = lpgen.dense_lp(80, 60, 9)
    ref = oracle.solve(A, b, c)
    st, sol, T, q, p, stats = _run(tsx, A, b, c, eps_p_fp32=3.0)
    assert st == tsx.LP_OPTIMAL
    assert stats["cleanup_pivots"] > 0
    _assert_matches_fp64(A, b, c, sol, ref)


def test_golden_traces_and_special_cases(tsx, golden_dir):
    import json
    import os
    for name in ("two_pivots_dyadic.json", "one_pivot.json", "unbounded_after_one.json"):
        g = json.load(open(os.path.join(golden_dir, name)))
        A = np.array(g["A"], dtype=np.float64)
        b = np.array(g["b"], dtype=np.float64)
        c = np.array(g["c"], dtype=np.float64)
        st, sol, T, q, p, stats = _run(tsx, A, b, c)
        assert tsx.STATUS_NAMES[st] == g["status"]
        if g["status"] == "OPTIMAL":
            assert sol.obj == g["obj"]
            np.testing.assert_array_equal(sol.x, np.array(g["x"], dtype=np.float64))
    # nothing to improve: x = 0 from the start
    A, b, _ = lpgen.dense_lp(6, 4, 2)
    st, sol, T, q, p, stats = _run(tsx, A, b, -np.ones(4))
    assert st == tsx.LP_OPTIMAL and sol.obj == 0.0 and stats["k"] == 0
    assert not sol.x.any() and not sol.y.any()


def test_fp32_full_size_16384(tsx):
    # the precision workload: m = n = 16384, float tableau (2.1 GB) for every
    # pivot, FP64 recovery; checked against the FP64 oracle's whole solve
    # (tests/golden/full_size, written by the oracle alone) and by certificates.
    # The FP64 path on the same LP must equal that oracle run exactly.
    import torch
    from test_gpu_full_size import load_golden
    m = n = 16384
    g = load_golden(m, n, 1)
    A, b, c = lpgen.dense_lp(m, n, 1)
    assert lpgen.lp_digest(A, b, c) == g["lp_sha256"]
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    s = torch.cuda.current_stream().cuda_stream
    with tsx.Problem(dA, db, dc, device=True, stream=s) as pr:
        assert pr.solve(tsx.options(stream=s, precision=tsx.LP_PREC_FP32)) == tsx.LP_OPTIMAL
        sol32 = pr.solution()
        st32 = pr.stats()
        assert pr.solve(tsx.options(stream=s, log_capacity=1 << 16)) == tsx.LP_OPTIMAL
        sol64 = pr.solution()
        q, p = (v.tolist() for v in pr.pivot_log(1 << 16))
    ref_obj = g["obj_value"]
    assert abs(sol32.obj - ref_obj) <= 1e-9 * abs(ref_obj)
    assert np.abs(sol32.x - g["x"]).max() <= 1e-9 * max(1.0, float(np.abs(g["x"]).max()))
    assert np.abs(sol32.y - g["y"]).max() <= 1e-9 * max(1.0, float(np.abs(g["y"]).max()))
    pv, dv = _violations(A, b, c, sol32.x, sol32.y)
    assert pv <= 1e-9 and dv <= 1e-9
    assert abs(c @ sol32.x - b @ sol32.y) <= 1e-9 * abs(ref_obj)
    assert st32["primal_violation"] <= 1e-9 and st32["dual_violation"] <= 1e-9
    # the FP64 path: the oracle's run, pivot for pivot
    assert sol64.iters == g["iters"] and q == g["qlog"] and p == g["plog"]
    assert sol64.obj == ref_obj
    np.testing.assert_array_equal(sol64.x, g["x"])
    np.testing.assert_array_equal(sol64.y, g["y"])


@pytest.mark.parametrize("m", [2048, 4096])
def test_fp32_recovery_of_a_large_basis(tsx, m):
    # every structural variable ends basic (k = m): the FP64 recovery factors
    # an m x m block; its result is checked against the FP64 oracle's whole
    # solve (tests/golden/full_size, written by the oracle alone)
    import torch
    from test_gpu_full_size import load_golden
    g = load_golden(m, m, 1, gen="diag_dominant_lp")
    A, b, c = lpgen.diag_dominant_lp(m, m, 1)
    assert lpgen.lp_digest(A, b, c) == g["lp_sha256"]
    assert len(g["x_nonzero"]) == m   # the oracle's basis: k = m
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    s = torch.cuda.current_stream().cuda_stream
    with tsx.Problem(dA, db, dc, device=True, stream=s) as pr:
        assert pr.solve(tsx.options(stream=s, precision=tsx.LP_PREC_FP32)) == tsx.LP_OPTIMAL
        sol = pr.solution()
        st = pr.stats()
    assert st["k"] == m and st["recover_ms"] > 0
    ref_obj = g["obj_value"]
    assert abs(sol.obj - ref_obj) <= 1e-9 * abs(ref_obj)
    assert np.abs(sol.x - g["x"]).max() <= 1e-9 * max(1.0, float(np.abs(g["x"]).max()))
    assert np.abs(sol.y - g["y"]).max() <= 1e-9 * max(1.0, float(np.abs(g["y"]).max()))
    pv, dv = _violations(A, b, c, sol.x, sol.y)
    assert pv <= 1e-9 and dv <= 1e-9
    assert st["primal_violation"] <= 1e-9 and st["dual_violation"] <= 1e-9


@pytest.mark.parametrize("path", [1, 2])
def test_concurrent_solves_equal_their_solo_runs(tsx, path):
    # eight host threads solve medium LPs at once on full grids, so the
    # refactorisation's blocks run interleaved with other solves' kernels;
    # every result must equal the same solve run alone
    import threading
    shapes = [(300, 500), (640, 410), (512, 512), (800, 350)] * 6
    problems = [lpgen.dense_lp(m, n, 600 + k) for k, (m, n) in enumerate(shapes)]
    opts = dict(precision=tsx.LP_PREC_FP32, path=path, blocks=304)

    def solve(k):
        with tsx.Problem(*problems[k]) as pr:
            st = pr.solve(tsx.options(**opts))
            return st, pr.solution()

    alone = [solve(k) for k in range(len(problems))]
    together = [None] * len(problems)

    def worker(idx):
        for k in idx:
            together[k] = solve(k)

    th = [threading.Thread(target=worker, args=(range(j, len(problems), 8),)) for j in range(8)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for k in range(len(problems)):
        (st1, s1), (st2, s2) = alone[k], together[k]
        assert st1 == st2 == tsx.LP_OPTIMAL, k
        assert s1.obj == s2.obj and s1.iters == s2.iters, k
        np.testing.assert_array_equal(s1.x, s2.x)
        np.testing.assert_array_equal(s1.y, s2.y)
