"""lp_solve_noalloc: the solve for callers that cannot allocate device memory.

Some callers cannot let a library call cudaMalloc/cudaFree: a plugin inside a
host application whose memory pool already holds the GPU's memory, or a
latency-bound loop where an allocation may block on other device work.
lp_solve_noalloc takes every input and output buffer from the caller and keeps
its work buffers in one fixed array inside the library.  These tests call it
through the C ABI and compare it with the allocating entry points
(lp_create_device + lp_solve), with the tolerance of the other FP64 parity
tests: equal tableau, basis, status and pivot count.  This file sorts last so a
first-failure run has already run every other test.
"""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_10979_gb300 import build
    build.build()
    import paper_2211_10979_gb300 as tsx
    return torch, tsx


def _reference(tsx, torch, dA, db, dc, m, n, stream):
    with tsx.Problem(dA, db, dc, device=True, stream=stream) as pr:
        st = pr.solve(tsx.options(stream=stream))
        sol = pr.solution()
        return st, sol.iters, pr.tableau(), sol.basis


def test_noalloc_matches_allocating_path_twice_in_a_row(env):
    torch, tsx = env
    stream = torch.cuda.current_stream().cuda_stream
    # two different LPs back to back: the second call must not see the first
    # call's leftovers in the shared work array
    for (m, n, seed) in ((300, 200, 5), (257, 129, 6), (300, 200, 5)):
        A, b, c = lpgen.dense_lp(m, n, seed)
        dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
        ld = (n + m + 1 + 3) // 4 * 4
        dT = torch.full(((m + 1) * ld,), float("nan"), dtype=torch.float64, device="cuda")
        dbasis = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        st, iters = tsx.lp_solve_noalloc(m, n, dA, db, dc, dT, ld, dbasis,
                                         tsx.options(stream=stream))
        assert st == tsx.LP_OPTIMAL, tsx.lp_last_error()
        rst, riters, rT, rbasis = _reference(tsx, torch, dA, db, dc, m, n, stream)
        assert st == rst and iters == riters
        T = dT.view(m + 1, ld).cpu().numpy()
        np.testing.assert_array_equal(T[:, :n + m + 1], rT)
        np.testing.assert_array_equal(T[:, n + m + 1:], 0.0)
        np.testing.assert_array_equal(dbasis.cpu().numpy(), rbasis)


def test_noalloc_call_allocates_nothing(env):
    # the property the entry point exists for: after a first call (which looks
    # up the fixed array's address once), a call leaves the device's free
    # memory unchanged and never reaches the library's allocator
    import ctypes
    torch, tsx = env
    stream = torch.cuda.current_stream().cuda_stream
    m, n = 300, 200
    A, b, c = lpgen.dense_lp(m, n, 7)
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    ld = (n + m + 1 + 3) // 4 * 4
    dT = torch.zeros((m + 1) * ld, dtype=torch.float64, device="cuda")
    dbasis = torch.zeros(m, dtype=torch.int32, device="cuda")
    opts = tsx.options(stream=stream)
    assert tsx.lp_solve_noalloc(m, n, dA, db, dc, dT, ld, dbasis, opts)[0] == tsx.LP_OPTIMAL
    calls = [0]

    def count_alloc(nbytes, strm, ctx):
        calls[0] += 1
        return None

    def count_free(ptr, nbytes, strm, ctx):
        calls[0] += 1

    alloc_cb, free_cb = tsx.abi.ALLOC_FN(count_alloc), tsx.abi.FREE_FN(count_free)
    assert tsx.abi.lp_set_allocator(alloc_cb, free_cb) == 0
    try:
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st, _ = tsx.lp_solve_noalloc(m, n, dA, db, dc, dT, ld, dbasis, opts)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
    finally:
        # put back whatever was installed before (torch's hooks if an earlier
        # test routed the library through torch, else the library default)
        prev = tsx._torch_hooks
        if prev is not None:
            tsx.abi.lp_set_allocator(prev[0], prev[1])
        else:
            tsx.abi.lp_set_allocator(ctypes.cast(None, tsx.abi.ALLOC_FN),
                                     ctypes.cast(None, tsx.abi.FREE_FN))
    assert st == tsx.LP_OPTIMAL
    assert calls[0] == 0
    assert free_after == free_before


def test_noalloc_binding_checks_tensors(env):
    torch, tsx = env
    m, n, ld = 4, 3, 8
    ok = dict(dA=torch.zeros(m * n, dtype=torch.float64, device="cuda"),
              db=torch.zeros(m, dtype=torch.float64, device="cuda"),
              dc=torch.zeros(n, dtype=torch.float64, device="cuda"),
              dT=torch.zeros((m + 1) * ld, dtype=torch.float64, device="cuda"),
              dbasis=torch.zeros(m, dtype=torch.int32, device="cuda"))
    bad = [("dT", torch.zeros((m + 1) * ld - 1, dtype=torch.float64, device="cuda")),
           ("dbasis", torch.zeros(m, dtype=torch.int64, device="cuda")),
           ("dA", torch.zeros(m * n, dtype=torch.float64)),
           ("dc", torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2])]
    for name, t in bad:
        args = dict(ok, **{name: t})
        with pytest.raises(ValueError, match=name):
            tsx.lp_solve_noalloc(m, n, args["dA"], args["db"], args["dc"], args["dT"], ld,
                                 args["dbasis"])


def test_noalloc_per_phase_path_and_bland(env):
    torch, tsx = env
    A = np.array([[0.5, -5.5, -2.5, 9.0], [0.5, -1.5, -0.5, 1.0], [1.0, 0.0, 0.0, 0.0]])
    b = np.array([0.0, 0.0, 1.0])
    c = np.array([10.0, -57.0, -9.0, -24.0])
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    m, n, ld = 3, 4, 8
    stream = torch.cuda.current_stream().cuda_stream
    for path in (1, 2):
        dT = torch.zeros((m + 1) * ld, dtype=torch.float64, device="cuda")
        dbasis = torch.zeros(m, dtype=torch.int32, device="cuda")
        st, iters = tsx.lp_solve_noalloc(m, n, dA, db, dc, dT, ld, dbasis,
                                         tsx.options(stream=stream, path=path, k_cyc=3))
        ref = tsx.Problem(dA, db, dc, device=True, stream=stream)
        ref_st = ref.solve(tsx.options(stream=stream, path=path, k_cyc=3))
        assert st == ref_st == tsx.LP_OPTIMAL
        np.testing.assert_array_equal(dT.view(m + 1, ld).cpu().numpy()[:, :n + m + 1], ref.tableau())
        ref.close()


def test_noalloc_rejects_sizes_beyond_the_array(env):
    torch, tsx = env
    # sizes only: the call must refuse before touching any pointer
    fake = 1 << 20
    m, n = 150000, 150000
    st, _ = tsx.lp_solve_noalloc(m, n, fake, fake, fake, fake, n + m + 4, fake)
    assert st == tsx.LP_ERR_INVALID
    msg = tsx.lp_last_error()
    assert "fixed array" in msg and str(tsx.abi.LP_NOALLOC_SCRATCH_BYTES) in msg
    st, _ = tsx.lp_solve_noalloc(4, 3, fake, fake, fake, fake, 7, fake)   # ld not a multiple of 4
    assert st == tsx.LP_ERR_INVALID and "multiple of 4" in tsx.lp_last_error()
    st, _ = tsx.lp_solve_noalloc(4, 3, fake, fake, fake, fake, 8, fake,
                                 tsx.options(log_capacity=10))
    assert st == tsx.LP_ERR_INVALID


def test_noalloc_refuses_a_capturing_stream(env):
    # the call reads status words back and waits for the device, so it cannot
    # be recorded into a graph: on a capturing stream it returns LP_ERR_STATE
    # before any device work, and the capture itself completes
    torch, tsx = env
    m, n = 6, 5
    A, b, c = lpgen.dense_lp(m, n, 3)
    dA, db, dc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    ld = (n + m + 1 + 3) // 4 * 4
    dT = torch.zeros((m + 1) * ld, dtype=torch.float64, device="cuda")
    dbasis = torch.zeros(m, dtype=torch.int32, device="cuda")
    x = torch.zeros(4, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        st, iters = tsx.lp_solve_noalloc(m, n, dA, db, dc, dT, ld, dbasis, tsx.options(stream=s.cuda_stream))
    assert st == tsx.LP_ERR_STATE and iters == 0
    assert "captured" in tsx.lp_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert x.tolist() == [1.0] * 4
    # outside the capture the same call solves
    st, _ = tsx.lp_solve_noalloc(m, n, dA, db, dc, dT, ld, dbasis, tsx.options(stream=s.cuda_stream))
    assert st == tsx.LP_OPTIMAL
