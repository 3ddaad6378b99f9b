"""The paper's CPU+GPU column split (Section IV) vs the oracle (needs a GPU).

LP_PATH_HYBRID keeps a fraction gpu_share of the nonbasic column slots on the
GPU and the rest on host threads, and exchanges the Step 1 candidates, the
owner's Step 2 result and column q every pivot.  Both sides do the method's
arithmetic (IEEE division, one fused multiply-add per entry, the same tie
rules), so the pivot sequence, basis, tableau, x, y and objective equal the
oracle's at tolerance 0, whatever the split.
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
    with tsx.Problem(A, b, c) as pr:
        st = pr.solve(tsx.options(path=tsx.LP_PATH_HYBRID, **kw))
        sol = pr.solution()
        T = pr.tableau()
        q, p = pr.pivot_log(kw["log_capacity"])
        return st, sol, T, q, p, pr.stats()


def _same(run, ref):
    st, sol, T, q, p, stats = run
    assert st == ref.status, tsx_name(st)
    assert sol.iters == ref.iters
    np.testing.assert_array_equal(q, ref.qlog[:len(q)])
    np.testing.assert_array_equal(p, ref.plog[:len(p)])
    np.testing.assert_array_equal(sol.basis, ref.basis)
    np.testing.assert_array_equal(T, ref.T)
    np.testing.assert_array_equal(sol.x, ref.x)
    np.testing.assert_array_equal(sol.y, ref.y)
    assert sol.obj == ref.obj
    assert stats["path"] == 5


def tsx_name(st):
    return {0: "OPTIMAL", 1: "UNBOUNDED", 2: "ITER_LIMIT", -4: "TIMEOUT", -3: "CUDA"}.get(st, st)


@pytest.mark.parametrize("m,n", [(1, 1), (3, 4), (37, 53), (200, 150), (150, 400), (600, 500)])
@pytest.mark.parametrize("share", [0.0, 0.3, 0.95, 1.0])
@pytest.mark.parametrize("threads", [1, 4])
def test_hybrid_equals_oracle(tsx, m, n, share, threads):
    A, b, c = lpgen.dense_lp(m, n, 70 + m + n)
    _same(_run(tsx, A, b, c, gpu_share=share, cpu_threads=threads), oracle.solve(A, b, c))


@pytest.mark.parametrize("kw", [{"k_cyc": 3}, {"rule": 1}, {"max_iters": 9}])
def test_hybrid_rules_and_degenerate_lps(tsx, kw):
    A = np.array([[0.5, -5.5, -2.5, 9.0], [0.5, -1.5, -0.5, 1.0], [1.0, 0.0, 0.0, 0.0]])
    b = np.array([0.0, 0.0, 1.0])
    c = np.array([10.0, -57.0, -9.0, -24.0])
    for share in (0.0, 0.5, 1.0):
        _same(_run(tsx, A, b, c, gpu_share=share, cpu_threads=2, **kw), oracle.solve(A, b, c, oracle.Options(**kw)))
    A0, b0, c0 = lpgen.dense_lp(40, 30, 11)
    A = np.vstack([A0, A0[:10], np.ones((3, 30))])
    b = np.concatenate([b0, b0[:10], np.full(3, 50.0)])
    _same(_run(tsx, A, b, c0, gpu_share=0.5, cpu_threads=3, **kw), oracle.solve(A, b, c0, oracle.Options(**kw)))


def test_hybrid_unbounded_on_either_side(tsx):
    # column 1 has no positive entry and enters first: unbounded, whichever
    # side holds it
    A = np.array([[1.0, -2.0, 1.0], [1.0, 0.0, 2.0]])
    b = np.array([4.0, 3.0])
    c = np.array([0.0, 5.0, 1.0])
    ref = oracle.solve(A, b, c)
    assert ref.status == oracle.UNBOUNDED
    for share in (0.0, 1.0, 0.34, 0.67):
        _same(_run(tsx, A, b, c, gpu_share=share, cpu_threads=2), ref)


def test_hybrid_wait_limit_reports_and_context_survives(tsx):
    # a zero wait budget: both sides give up at their first exchange; the
    # solve ends LP_ERR_TIMEOUT and the next solve on the context is exact
    A, b, c = lpgen.dense_lp(120, 100, 5)
    with tsx.Problem(A, b, c) as pr:
        st = tsx.lp_solve(pr.h, tsx.options(path=tsx.LP_PATH_HYBRID, gpu_share=0.5, cpu_threads=2,
                                            barrier_timeout_ns=0))
        assert st == tsx.LP_ERR_TIMEOUT
        assert pr.solve(tsx.options(path=tsx.LP_PATH_HYBRID, gpu_share=0.5, cpu_threads=2)) == tsx.LP_OPTIMAL
        np.testing.assert_array_equal(pr.tableau(), oracle.solve(A, b, c).T)


def test_hybrid_refusals(tsx):
    A, b, c = lpgen.dense_lp(30, 20, 3)
    with tsx.Problem(A, b, c) as pr:
        for kw in ({"layout": tsx.LP_LAYOUT_FULL}, {"precision": tsx.LP_PREC_FP32}):
            assert tsx.lp_solve(pr.h, tsx.options(path=tsx.LP_PATH_HYBRID, **kw)) == tsx.LP_ERR_INVALID
        assert tsx.lp_solve(pr.h, tsx.options(path=tsx.LP_PATH_HYBRID, gpu_share=1.5)) == tsx.LP_ERR_INVALID


def test_hybrid_full_size_equals_oracle_golden(tsx):
    # the benchmark's 8192^2 LP with 5 % of the columns on the host: the whole
    # pivot sequence and the solution equal the oracle's whole solve
    import torch
    from test_gpu_full_size import load_golden
    m = n = 8192
    g = load_golden(m, n, 1)
    A, b, c = lpgen.dense_lp(m, n, 1)
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    s = torch.cuda.current_stream().cuda_stream
    with tsx.Problem(dA, db, dc, device=True, stream=s) as pr:
        st = pr.solve(tsx.options(stream=s, path=tsx.LP_PATH_HYBRID, gpu_share=0.95, log_capacity=1 << 16))
        assert tsx.STATUS_NAMES[st] == g["status"]
        sol = pr.solution()
        q, p = (v.tolist() for v in pr.pivot_log(1 << 16))
    assert sol.iters == g["iters"] and q == g["qlog"] and p == g["plog"]
    assert sol.obj == g["obj_value"]
    np.testing.assert_array_equal(sol.x, g["x"])
    np.testing.assert_array_equal(sol.y, g["y"])
