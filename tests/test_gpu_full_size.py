"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (persistent kernel, default grid and block, zero-column skipping on).

The oracle cannot finish a whole 8192 x 8192 solve in test time (~2800 pivots
at ~15 pivots/s), so the checks are:
  - the first K pivots: the GPU tableau after K pivots equals the oracle's
    after K pivots, entry by entry (tolerance 0), and so do the (q, p) pairs;
  - the full solve: properties that hold at any size -- the basic columns are
    exact unit vectors, x and y satisfy primal and dual feasibility and strong
    duality in FP64 within 1e-9 (relative), and the pivot log starts with the
    oracle's K pivots.
"""
import numpy as np
import pytest

import lpgen
import oracle

pytestmark = pytest.mark.gpu

K = 3


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


def _certificate(A, b, c, x, y, obj, tol=1e-9):
    scale = max(1.0, abs(obj))
    assert np.all(x >= -tol)
    assert np.all(A @ x <= b + tol * (1.0 + np.abs(b)))
    assert np.all(y >= -tol)
    assert np.all(A.T @ y >= c - tol * (1.0 + np.abs(c)))
    assert abs(c @ x - obj) <= tol * scale
    assert abs(b @ y - obj) <= tol * scale


@pytest.mark.parametrize("m,n,layout", [(8192, 8192, 0), (4096, 16384, 0), (8192, 8192, 1)])
def test_full_size_first_pivots_and_certificates(tsx, m, n, layout):
    # layout 0 (the bench's): condensed device tableau, expanded to Table I on
    # read-out, so the unit-column check below holds by construction there and
    # is the real check for layout 1
    import torch
    A, b, c = lpgen.dense_lp(m, n, 1)
    ref = oracle.solve(A, b, c, oracle.Options(max_iters=K))
    assert ref.status == oracle.ITER_LIMIT and ref.iters == K
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    s = torch.cuda.current_stream().cuda_stream
    with tsx.Problem(dA, db, dc, device=True, stream=s) as pr:
        # the first K pivots, compared entry by entry
        assert pr.solve(tsx.options(stream=s, max_iters=K, log_capacity=K, layout=layout)) == tsx.LP_ITER_LIMIT
        q, p = pr.pivot_log(K)
        assert q.tolist() == ref.qlog.tolist() and p.tolist() == ref.plog.tolist()
        T = pr.tableau()
        np.testing.assert_array_equal(T, ref.T)
        del T
        # the whole solve, checked by properties that hold at any size
        assert pr.solve(tsx.options(stream=s, log_capacity=1 << 16, layout=layout)) == tsx.LP_OPTIMAL
        sol = pr.solution()
        q, p = pr.pivot_log(K)
        assert q.tolist() == ref.qlog.tolist() and p.tolist() == ref.plog.tolist()
        stats = pr.stats()
        assert stats["path"] == tsx.LP_PATH_PERSISTENT and stats["iters"] == sol.iters
        assert stats["layout"] == layout
        T = pr.tableau()
    rows = np.arange(1, m + 1)
    basic = sol.basis.astype(np.int64)
    assert len(set(basic.tolist())) == m
    np.testing.assert_array_equal(T[rows, basic], 1.0)
    sub = T[:, basic]
    sub[rows, np.arange(m)] = 0.0
    assert not np.any(sub)
    _certificate(A, b, c, sol.x, sol.y, sol.obj)
