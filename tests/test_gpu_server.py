"""The request server (continuous batching) and the device input generator.

Each served result must be the same in the mix as alone: the server runs the
library's deterministic solves, so a small LP (micro-batched, FP64) equals the
oracle exactly, and a larger LP (FP32 tableau + FP64 recovery) equals the same
solve run alone, entry for entry, and the FP64 oracle's objective within 1e-9.
"""
import threading
import time

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


@pytest.mark.parametrize("m,n,seed", [(1, 1, 1), (5, 3, 2), (37, 53, 3), (300, 200, 4), (1000, 999, 5)])
def test_device_generator_equals_lpgen(tsx, m, n, seed):
    import torch
    A, b, c = lpgen.dense_lp(m, n, seed)
    dA = torch.empty(m * n, dtype=torch.float64, device="cuda")
    db = torch.empty(m, dtype=torch.float64, device="cuda")
    dc = torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert tsx.lp_generate_dense(m, n, seed, dA, db, dc, s) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dA.cpu().numpy().reshape(m, n), A)
    np.testing.assert_array_equal(db.cpu().numpy(), b)
    np.testing.assert_array_equal(dc.cpu().numpy(), c)


def _alone_fp32(tsx, A, b, c):
    with tsx.Problem(A, b, c) as pr:
        st = pr.solve(tsx.options(precision=tsx.LP_PREC_FP32))
        return st, pr.solution()


@pytest.mark.parametrize("continuous", [1, 0])
def test_results_same_alone_and_in_the_mix(tsx, continuous):
    # a mix of small (micro-batched) and larger (team-solved) LPs submitted
    # from two client threads while earlier ones are being solved; the large
    # ones go to the continuous team launch (1) or to lp_solve_many waves (0)
    shapes = [(20, 30), (64, 64), (300, 250), (16, 128), (128, 16), (700, 400), (50, 50),
              (256, 1024), (90, 120), (33, 77), (1500, 600), (128, 128), (1200, 1100)] * 3
    problems = [lpgen.dense_lp(m, n, 4000 + k) for k, (m, n) in enumerate(shapes)]
    tickets = [None] * len(problems)
    with tsx.Server(workers=4, continuous=continuous) as sv:
        def client(idx):
            for k in idx:
                tickets[k] = sv.submit(*problems[k])
                time.sleep(0.001)
        th = [threading.Thread(target=client, args=(range(j, len(problems), 2),)) for j in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        results = []
        for k, t in enumerate(tickets):
            assert sv.wait(t, 120.0) == tsx.LP_OPTIMAL
            results.append(sv.result(t))
        st = sv.stats()
    assert st["completed"] == len(problems) and st["batched_lps"] > 0
    if continuous:
        assert st["waves"] == 0 and st["lane_launches"] >= 1
        assert st["lane_lps"] + st["batched_lps"] == len(problems)
    else:
        assert st["lane_lps"] == 0 and st["waves"] > 0
        assert st["wave_lps"] + st["batched_lps"] == len(problems)
    for k, ((m, n), (A, b, c), r) in enumerate(zip(shapes, problems, results)):
        ref = oracle.solve(A, b, c)
        if (m + 1) * (n + 2) * 8 < 200_000:
            # micro-batched: the FP64 method, equal to the oracle
            assert r.iters == ref.iters and r.obj == ref.obj
            np.testing.assert_array_equal(r.x, ref.x)
            np.testing.assert_array_equal(r.y, ref.y)
        else:
            st1, alone = _alone_fp32(tsx, A, b, c)
            assert st1 == tsx.LP_OPTIMAL
            assert r.obj == alone.obj and r.iters == alone.iters
            np.testing.assert_array_equal(r.x, alone.x)
            np.testing.assert_array_equal(r.y, alone.y)
            assert abs(r.obj - ref.obj) <= 1e-9 * abs(ref.obj)
        assert r.t_submit <= r.t_admit <= r.t_done


def test_budget_admission_and_device_inputs(tsx):
    # a budget that fits one larger request at a time: admission waits for
    # memory; device-resident inputs are referenced until their request ends
    import torch
    shapes = [(400, 300), (350, 420), (30, 40), (500, 200)]
    reqs = []
    s = torch.cuda.current_stream().cuda_stream
    for k, (m, n) in enumerate(shapes):
        dA = torch.empty(m * n, dtype=torch.float64, device="cuda")
        db = torch.empty(m, dtype=torch.float64, device="cuda")
        dc = torch.empty(n, dtype=torch.float64, device="cuda")
        tsx.lp_generate_dense(m, n, 700 + k, dA, db, dc, s)
        reqs.append((m, n, dA, db, dc))
    torch.cuda.synchronize()
    budget = 12 << 20
    with tsx.Server(workers=3, budget_bytes=budget) as sv:
        tickets = [sv.submit_device(m, n, dA, db, dc) for (m, n, dA, db, dc) in reqs]
        res = [(sv.wait(t, 120.0), sv.result(t)) for t in tickets]
        st = sv.stats()
    assert st["peak_bytes"] <= budget
    for k, ((m, n), (code, r)) in enumerate(zip(shapes, res)):
        A, b, c = lpgen.dense_lp(m, n, 700 + k)
        ref = oracle.solve(A, b, c)
        assert code == tsx.LP_OPTIMAL
        assert abs(r.obj - ref.obj) <= 1e-9 * abs(ref.obj)


def test_global_memory_micro_batches(tsx):
    # with batch_max_bytes set, medium LPs join the micro-batches too (solved
    # from global memory one block per LP): still the FP64 method, oracle-exact
    shapes = [(200, 200), (300, 150), (60, 60), (400, 90)] * 2
    problems = [lpgen.dense_lp(m, n, 800 + k) for k, (m, n) in enumerate(shapes)]
    with tsx.Server(workers=2, batch_max_bytes=8 << 20) as sv:
        tickets = [sv.submit(*p) for p in problems]
        res = [(sv.wait(t, 120.0), sv.result(t)) for t in tickets]
        assert sv.stats()["batched_lps"] == len(problems)
    for (A, b, c), (code, r) in zip(problems, res):
        ref = oracle.solve(A, b, c)
        assert code == tsx.LP_OPTIMAL and r.obj == ref.obj and r.iters == ref.iters
        np.testing.assert_array_equal(r.x, ref.x)


def test_one_per_worker_without_waves(tsx):
    # team_blocks < 0: the large requests are solved one per worker by lp_solve
    shapes = [(300, 250), (256, 700), (600, 300)] * 2
    problems = [lpgen.dense_lp(m, n, 900 + k) for k, (m, n) in enumerate(shapes)]
    with tsx.Server(workers=3, team_blocks=-1) as sv:
        tickets = [sv.submit(*p) for p in problems]
        res = [(sv.wait(t, 120.0), sv.result(t)) for t in tickets]
        st = sv.stats()
    assert st["waves"] == 0 and st["completed"] == len(problems)
    for (A, b, c), (code, r) in zip(problems, res):
        st1, alone = _alone_fp32(tsx, A, b, c)
        assert code == st1 == tsx.LP_OPTIMAL
        assert r.obj == alone.obj and r.iters == alone.iters
        np.testing.assert_array_equal(r.x, alone.x)


def test_plain_mode_and_stats(tsx):
    problems = [lpgen.dense_lp(m, n, 90 + m) for m, n in [(40, 40), (200, 150), (64, 32)]]
    with tsx.Server(workers=1, batch_small=0) as sv:
        tickets = [sv.submit(*p) for p in problems]
        for t in tickets:
            assert sv.wait(t, 60.0) == tsx.LP_OPTIMAL
        st = sv.stats()
        assert st["batches"] == 0 and st["completed"] == 3
        assert 0 < st["lat_p50_ms"] <= st["lat_p99_ms"] <= st["lat_max_ms"]
        assert sv.wait(10**9, 0.0) == tsx.LP_ERR_INVALID
    with pytest.raises(ValueError, match="budget"):
        with tsx.Server(budget_bytes=1 << 20) as sv:
            sv.submit(*lpgen.dense_lp(500, 500, 1))


def test_request_admitted_into_running_work_finishes_first(tsx):
    # a large LP is being solved by the continuous team launch when a medium
    # one arrives: the medium one is taken by another team at once and its
    # result comes back before the large one's (no wave boundary to wait for)
    big = lpgen.dense_lp(4000, 4000, 31)
    mid = lpgen.dense_lp(400, 300, 32)
    with tsx.Server(workers=2) as sv:
        tb = sv.submit(*big)
        time.sleep(0.005)
        tm = sv.submit(*mid)
        assert sv.wait(tm, 120.0) == tsx.LP_OPTIMAL
        assert sv.wait(tb, 0.0) == tsx.LP_PENDING      # the large one is still running
        rm = sv.result(tm)
        assert sv.wait(tb, 120.0) == tsx.LP_OPTIMAL
        rb = sv.result(tb)
        st = sv.stats()
    assert rm.t_done < rb.t_done and st["lane_lps"] == 2
    for (A, b, c), r in ((mid, rm), (big, rb)):
        st1, alone = _alone_fp32(tsx, A, b, c)
        assert st1 == tsx.LP_OPTIMAL and r.obj == alone.obj and r.iters == alone.iters
        np.testing.assert_array_equal(r.x, alone.x)
        np.testing.assert_array_equal(r.y, alone.y)


@pytest.mark.parametrize("continuous", [1, 0])
def test_invalid_device_request_in_a_wave(tsx, continuous):
    # device inputs are checked in the team kernel's build: a request with
    # b_i < 0 ends LP_ERR_INVALID, the others of its wave are unaffected
    import torch
    shapes = [(400, 300), (350, 420), (500, 250)]
    reqs = []
    s = torch.cuda.current_stream().cuda_stream
    for k, (m, n) in enumerate(shapes):
        A, b, c = lpgen.dense_lp(m, n, 910 + k)
        if k == 1:
            b = b.copy()
            b[7] = -1.0
        reqs.append((m, n, *(torch.from_numpy(v).cuda() for v in (A.ravel(), b, c))))
    torch.cuda.synchronize()
    with tsx.Server(workers=2, continuous=continuous) as sv:
        tickets = [sv.submit_device(m, n, dA, db, dc) for (m, n, dA, db, dc) in reqs]
        codes = [sv.wait(t, 120.0) for t in tickets]
        res = [sv.result(t) for t in tickets]
    assert codes[1] == tsx.LP_ERR_INVALID
    for k in (0, 2):
        A, b, c = lpgen.dense_lp(*shapes[k], 910 + k)
        ref = oracle.solve(A, b, c)
        assert codes[k] == tsx.LP_OPTIMAL
        assert abs(res[k].obj - ref.obj) <= 1e-9 * abs(ref.obj)
