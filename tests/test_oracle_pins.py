"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Each test checks the oracle (a plain C tableau simplex following Section III of
arXiv 2211.10979) against something other than itself: hand-derived exact
traces, brute-force vertex enumeration, closed forms, LP duality, and an
independent solver (HiGHS through scipy).
"""
import itertools
import json
import os

import numpy as np
import pytest

import lpgen
import oracle


def _load_golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- exact traces
@pytest.mark.parametrize("name", ["two_pivots_dyadic.json", "one_pivot.json",
                                  "unbounded_after_one.json"])
def test_hand_derived_trace_is_exact(golden_dir, name):
    g = _load_golden(golden_dir, name)
    A = np.array(g["A"], dtype=np.float64)
    b = np.array(g["b"], dtype=np.float64)
    c = np.array(g["c"], dtype=np.float64)
    m, n = A.shape
    T, basis = oracle.build_tableau(A, b, c)
    np.testing.assert_array_equal(T, np.array(g["T0"], dtype=np.float64))
    for st in g["steps"]:
        q = oracle.entering(T, m, n)
        assert q == st["q"]
        p, ratio = oracle.leaving(T, basis, m, n, q)
        assert p == st["p"] and ratio == st["ratio"]
        oracle.pivot(T, m, n, p, q)
        basis[p - 1] = q
        np.testing.assert_array_equal(T, np.array(st["T"], dtype=np.float64))
    # the full solve reproduces the same run and outcome
    r = oracle.solve(A, b, c)
    assert oracle.STATUS_NAMES[r.status] == g["status"]
    assert r.iters == len(g["steps"])
    assert r.qlog.tolist() == [s["q"] for s in g["steps"]]
    assert r.plog.tolist() == [s["p"] for s in g["steps"]]
    np.testing.assert_array_equal(r.T, np.array(g["steps"][-1]["T"], dtype=np.float64))
    assert r.obj == g["obj"]
    np.testing.assert_array_equal(r.x, np.array(g["x"], dtype=np.float64))
    np.testing.assert_array_equal(r.y, np.array(g["y"], dtype=np.float64))
    assert r.basis.tolist() == g["basis"]


def test_step1_rules_on_hand_made_row():
    # m = 1, n = 4: objective row [-1, -3, -3, 2, 0 | 0]
    T = np.array([[-1.0, -3.0, -3.0, 2.0, 0.0, 0.0],
                  [1.0, 1.0, 1.0, 1.0, 1.0, 1.0]])
    assert oracle.entering(T, 1, 4, bland=False) == 1     # most negative, lowest index on tie
    assert oracle.entering(T, 1, 4, bland=True) == 0      # lowest index below -eps
    T[0, :4] = [-1e-10, 0.0, 1.0, 2.0]
    assert oracle.entering(T, 1, 4) == -1                 # within eps_d: optimal
    assert oracle.entering(T, 1, 4, eps_d=1e-11) == 0


def test_step2_rules_on_hand_made_column():
    # m = 3, n = 1, W = 5: column 0 entries 2, 4, 1 with rhs 4, 8, 3 -> ratios 2, 2, 3
    T = np.zeros((4, 5))
    T[1:, 0] = [2.0, 4.0, 1.0]
    T[1:, 4] = [4.0, 8.0, 3.0]
    basis = np.array([3, 1, 2], dtype=np.int32)   # row 2's basic variable has the lower index
    assert oracle.leaving(T, basis, 3, 1, 0, bland=False) == (1, 2.0)  # lowest row on tie
    assert oracle.leaving(T, basis, 3, 1, 0, bland=True) == (2, 2.0)   # lowest basic index on tie
    T[1:, 0] = [0.0, -1.0, 1e-12]                                       # none above eps_p
    assert oracle.leaving(T, basis, 3, 1, 0)[0] == -1


def test_pivot_gaps_on_hand_made_tableau():
    # objective row [-1, -3, -2.5, 2 | 0] (m = 3, n = 1 plus slacks is not needed:
    # the gaps only read row 0 and column q): Step 1 picks column 1 (-3); the
    # next candidate is -2.5 -> gap 0.5.  Column 1 entries 2, 4, 1 with rhs
    # 4, 10, 3 -> ratios 2, 2.5, 3: row 1 leaves, next ratio 2.5 -> gap 0.5.
    T = np.zeros((4, 5))
    T[0, :4] = [-1.0, -3.0, -2.5, 2.0]
    T[1:, 1] = [2.0, 4.0, 1.0]
    T[1:, 4] = [4.0, 10.0, 3.0]
    assert oracle.entering(T, 3, 1) == 1
    assert oracle.leaving(T, np.array([1, 2, 3], dtype=np.int32), 3, 1, 1) == (1, 2.0)
    assert oracle.pivot_gaps(T, 3, 1, 1, 1) == (0.5, 0.5)
    # a tie shows as a zero gap; a lone candidate as an infinite one
    T[0, 2] = -3.0
    T[2, 4] = 8.0
    assert oracle.pivot_gaps(T, 3, 1, 1, 1) == (0.0, 0.0)
    T[0, :4] = [0.0, -3.0, 0.0, 2.0]
    T[2:, 1] = [0.0, -1.0]
    assert oracle.pivot_gaps(T, 3, 1, 1, 1) == (np.inf, np.inf)


def test_traced_solve_is_the_plain_solve_with_its_gaps():
    A, b, c = lpgen.dense_lp(48, 40, 5)
    r = oracle.solve(A, b, c)
    rt, tr = oracle.solve_traced(A, b, c)
    assert (rt.status, rt.iters, rt.obj) == (r.status, r.iters, r.obj)
    assert rt.qlog.tolist() == r.qlog.tolist() and rt.plog.tolist() == r.plog.tolist()
    np.testing.assert_array_equal(rt.T, r.T)
    # replay pivot by pivot: each recorded gap, ratio and entry is the one of
    # that pivot's tableau
    m, n = A.shape
    T, basis = oracle.build_tableau(A, b, c)
    for k, (q, p) in enumerate(zip(r.qlog.tolist(), r.plog.tolist())):
        assert tr.dval[k] == T[0, q]
        assert tr.theta[k] == oracle.leaving(T, basis, m, n, q)[1]
        assert (tr.dgap[k], tr.rgap[k]) == oracle.pivot_gaps(T, m, n, q, p)
        assert tr.dgap[k] > 0 and tr.rgap[k] > 0
        oracle.pivot(T, m, n, p, q)
        basis[p - 1] = q


# ------------------------------------------------------------- brute force
def _vertex_max(A, b, c):
    """max c.x over {Ax <= b, x >= 0} by enumerating every choice of n tight
    constraints among the m + n (rows of A, then the bounds x_j >= 0)."""
    m, n = A.shape
    G = np.vstack([A, -np.eye(n)])
    h = np.concatenate([b, np.zeros(n)])
    best, arg = -np.inf, None
    for rows in itertools.combinations(range(m + n), n):
        M = G[list(rows)]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, h[list(rows)])
        if np.all(G @ x <= h + 1e-9):
            v = float(c @ x)
            if v > best:
                best, arg = v, x
    return best, arg


def _small_lp(rng, m, n, mixed):
    if mixed:
        A = rng.integers(-4, 9, size=(m, n)).astype(np.float64)
        A[0] = np.abs(A[0]) + 1.0          # one all-positive row keeps it bounded
    else:
        A = rng.uniform(1.0, 10.0, size=(m, n))
    b = rng.uniform(1.0, 20.0, size=m)
    c = rng.uniform(-2.0, 10.0, size=n)
    return A, b, c


@pytest.mark.parametrize("mixed", [False, True])
def test_brute_force_vertex_enumeration(mixed):
    rng = np.random.default_rng(20221119 + int(mixed))
    for _ in range(100):
        m, n = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        A, b, c = _small_lp(rng, m, n, mixed)
        r = oracle.solve(A, b, c)
        assert r.status == oracle.OPTIMAL
        best, _ = _vertex_max(A, b, c)
        best = max(best, 0.0) if np.all(b >= 0) else best
        assert abs(r.obj - best) <= 1e-12 * max(1.0, abs(best)), (A, b, c, r.obj, best)
        # the reported x attains the reported objective and is feasible
        assert np.all(r.x >= 0)
        assert np.all(A @ r.x <= b + 1e-9 * (1 + np.abs(b)))
        assert abs(c @ r.x - r.obj) <= 1e-9 * max(1.0, abs(r.obj))


# ------------------------------------------------------------- closed forms
def test_single_variable_closed_form():
    # n = 1: x = min_i b_i / a_i, reached in exactly one pivot
    rng = np.random.default_rng(7)
    for m in (1, 2, 5, 17, 64):
        a = rng.uniform(1.0, 10.0, size=m)
        b = rng.uniform(100.0, 1000.0, size=m)
        r = oracle.solve(a.reshape(m, 1), b, np.array([3.0]))
        i = int(np.argmin(b / a))
        assert r.status == oracle.OPTIMAL and r.iters == 1
        assert r.x[0] == b[i] / a[i]
        assert r.plog.tolist() == [i + 1]
        assert r.obj == pytest.approx(3.0 * b[i] / a[i], rel=1e-15)


def test_single_constraint_closed_form():
    # m = 1: z* = b * max_j c_j / a_j; the optimum has one basic x_j
    rng = np.random.default_rng(8)
    for n in (1, 2, 3, 9, 50):
        a = rng.uniform(1.0, 10.0, size=n)
        c = rng.uniform(1.0, 10.0, size=n)
        b = np.array([rng.uniform(100.0, 1000.0)])
        r = oracle.solve(a.reshape(1, n), b, c)
        assert r.status == oracle.OPTIMAL
        k = int(np.argmax(c / a))
        assert r.obj == pytest.approx(b[0] * c[k] / a[k], rel=1e-13)
        assert r.basis.tolist() == [k]
        # Dantzig enters the largest c_j first; when that is also the best
        # ratio c_j / a_j it is the only pivot
        if int(np.argmax(c)) == k:
            assert r.iters == 1


def test_diagonal_closed_form():
    # A diagonal, c > 0: x_j = b_j / a_jj; Dantzig enters in decreasing order of
    # c_j (each pivot leaves the other reduced costs untouched)
    rng = np.random.default_rng(9)
    n = 12
    d = rng.uniform(1.0, 10.0, size=n)
    b = rng.uniform(100.0, 1000.0, size=n)
    c = rng.permutation(np.arange(1, n + 1)).astype(np.float64)
    r = oracle.solve(np.diag(d), b, c)
    assert r.status == oracle.OPTIMAL and r.iters == n
    np.testing.assert_array_equal(r.x, b / d)
    assert r.qlog.tolist() == list(np.argsort(-c))
    np.testing.assert_allclose(r.y, c / d, rtol=1e-15)


def test_unbounded_status():
    A = np.array([[1.0, -2.0], [1.0, 0.0]])
    r = oracle.solve(A, np.array([4.0, 3.0]), np.array([0.0, 1.0]))
    assert r.status == oracle.UNBOUNDED


def test_zero_objective_is_optimal_at_start():
    A, b, _ = lpgen.dense_lp(5, 4, 3)
    r = oracle.solve(A, b, -np.ones(4))
    assert r.status == oracle.OPTIMAL and r.iters == 0 and r.obj == 0.0
    assert r.basis.tolist() == [4, 5, 6, 7, 8]


def test_iteration_cap_stops_after_k_pivots():
    A, b, c = lpgen.dense_lp(64, 64, 1)
    full = oracle.solve(A, b, c)
    k = 5
    part = oracle.solve(A, b, c, oracle.Options(max_iters=k))
    assert part.status == oracle.ITER_LIMIT and part.iters == k
    assert part.qlog.tolist() == full.qlog[:k].tolist()
    # resuming from the stopped tableau finishes the same run
    T, basis = part.T.copy(), part.basis.copy()
    st, it, qlog, plog = oracle.solve_tableau(T, basis, 64, 64)
    assert st == oracle.OPTIMAL and k + it == full.iters
    np.testing.assert_array_equal(T, full.T)


def test_invalid_inputs_rejected():
    with pytest.raises(ValueError):
        oracle.build_tableau(np.ones((2, 2)), np.array([1.0, -1.0]), np.ones(2))
    with pytest.raises(ValueError):
        oracle.build_tableau(np.ones((2, 2)), np.array([1.0, np.nan]), np.ones(2))


# ------------------------------------------------------------- duality
def _certificate(A, b, c, x, y, obj, tol=1e-9):
    scale = max(1.0, abs(obj))
    assert np.all(x >= -tol)
    assert np.all(A @ x <= b + tol * (1 + np.abs(b)))
    assert np.all(y >= -tol)
    assert np.all(A.T @ y >= c - tol * (1 + np.abs(c)))
    assert abs(c @ x - obj) <= tol * scale
    assert abs(b @ y - obj) <= tol * scale
    # complementary slackness
    assert np.all(np.abs(y * (b - A @ x)) <= tol * scale * 10)
    assert np.all(np.abs(x * (A.T @ y - c)) <= tol * scale * 10)


@pytest.mark.parametrize("m,n,seed", [(16, 16, 1), (64, 48, 2), (256, 256, 1), (128, 512, 3),
                                      (512, 128, 4)])
def test_duality_certificate_generated(m, n, seed):
    A, b, c = lpgen.dense_lp(m, n, seed)
    r = oracle.solve(A, b, c)
    assert r.status == oracle.OPTIMAL
    _certificate(A, b, c, r.x, r.y, r.obj)


# ------------------------------------------------------------- independent solver
@pytest.mark.parametrize("m,n,seed", [(16, 16, 1), (64, 64, 2), (256, 256, 1), (256, 256, 2),
                                      (100, 300, 5), (300, 100, 6), (512, 512, 1)])
def test_objective_matches_highs(m, n, seed):
    linprog = pytest.importorskip("scipy.optimize").linprog
    A, b, c = lpgen.dense_lp(m, n, seed)
    r = oracle.solve(A, b, c)
    res = linprog(-c, A_ub=A, b_ub=b, bounds=(0, None), method="highs")
    assert res.status == 0
    assert abs(r.obj - (-res.fun)) <= 1e-9 * abs(res.fun)


# ------------------------------------------------------------- degeneracy
def test_cycling_example_terminates_with_bland_fallback():
    # A classic degenerate LP on which the largest-coefficient rule cycles
    # (Chvatal, Linear Programming, 1983, Ch. 3).  Its optimum is 1.
    A = np.array([[0.5, -5.5, -2.5, 9.0],
                  [0.5, -1.5, -0.5, 1.0],
                  [1.0, 0.0, 0.0, 0.0]])
    b = np.array([0.0, 0.0, 1.0])
    c = np.array([10.0, -57.0, -9.0, -24.0])
    pure = oracle.solve(A, b, c, oracle.Options(k_cyc=0, max_iters=200))
    assert pure.status == oracle.ITER_LIMIT          # Dantzig alone cycles
    for k in (1, 3, 6, 50):
        r = oracle.solve(A, b, c, oracle.Options(k_cyc=k))
        assert r.status == oracle.OPTIMAL
        assert r.obj == pytest.approx(1.0, abs=1e-12)
        _certificate(A, b, c, r.x, r.y, r.obj)
    r = oracle.solve(A, b, c, oracle.Options(rule=1))
    assert r.status == oracle.OPTIMAL and r.obj == pytest.approx(1.0, abs=1e-12)


def test_degenerate_duplicate_rows():
    A0, b0, c = lpgen.dense_lp(6, 5, 11)
    A = np.vstack([A0, A0[:3], np.ones((2, 5))])
    b = np.concatenate([b0, b0[:3], np.zeros(2)])
    r = oracle.solve(A, b, c)
    assert r.status == oracle.OPTIMAL and r.obj == 0.0      # the zero rows pin x = 0
    b[-2:] = 1e6
    r = oracle.solve(A, b, c)
    best, _ = _vertex_max(A, b, c)
    assert r.status == oracle.OPTIMAL and abs(r.obj - best) <= 1e-9 * best


# ------------------------------------------------------------- float variant
@pytest.mark.parametrize("name", ["two_pivots_dyadic.json", "one_pivot.json",
                                  "unbounded_after_one.json"])
def test_float_variant_hand_derived_trace_is_exact(golden_dir, name):
    # every value of these traces is a float as well: the float steps must
    # reproduce them exactly
    g = _load_golden(golden_dir, name)
    A = np.array(g["A"], dtype=np.float64)
    b = np.array(g["b"], dtype=np.float64)
    c = np.array(g["c"], dtype=np.float64)
    m, n = A.shape
    T, basis = oracle.build_tableau32(A, b, c)
    np.testing.assert_array_equal(T, np.array(g["T0"], dtype=np.float32))
    for st in g["steps"]:
        q = oracle.entering32(T, m, n)
        assert q == st["q"]
        p, ratio = oracle.leaving32(T, basis, m, n, q)
        assert p == st["p"] and ratio == st["ratio"]
        oracle.pivot32(T, m, n, p, q)
        basis[p - 1] = q
        np.testing.assert_array_equal(T, np.array(st["T"], dtype=np.float32))
    status, iters, qlog, plog, T, basis = oracle.solve32(A, b, c)
    assert oracle.STATUS_NAMES[status] == g["status"]
    assert qlog.tolist() == [s["q"] for s in g["steps"]]


def test_float_variant_brute_force_objective():
    rng = np.random.default_rng(31)
    for _ in range(60):
        m, n = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        A, b, c = _small_lp(rng, m, n, False)
        status, iters, qlog, plog, T, basis = oracle.solve32(A, b, c)
        assert status == oracle.OPTIMAL
        best, _ = _vertex_max(A, b, c)
        best = max(best, 0.0)
        assert abs(float(T[0, -1]) - best) <= 2e-5 * max(1.0, abs(best))


def test_float_variant_follows_double_run_on_generated_lp():
    # both precisions choose the same pivots here (gaps between candidates are
    # far above float rounding); the objectives agree to float accuracy
    A, b, c = lpgen.dense_lp(96, 80, 4)
    ref = oracle.solve(A, b, c)
    status, iters, qlog, plog, T, basis = oracle.solve32(A, b, c)
    assert status == oracle.OPTIMAL and iters == ref.iters
    assert qlog.tolist() == ref.qlog.tolist()
    assert abs(float(T[0, -1]) - ref.obj) <= 1e-5 * abs(ref.obj)
