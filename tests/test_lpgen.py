"""The seeded input generator (no GPU)."""
import numpy as np

import lpgen


def test_splitmix64_published_vector():
    # first outputs of the SplitMix64 reference generator for seed 1234567
    # (a widely reproduced known-answer vector of Vigna's splitmix64.c)
    assert lpgen.splitmix64_stream(1234567, 0, 5).tolist() == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_stream_is_counter_based():
    whole = lpgen.splitmix64_stream(99, 0, 1000)
    part = lpgen.splitmix64_stream(99, 500, 500)
    np.testing.assert_array_equal(whole[500:], part)


def test_dense_lp_ranges_and_order():
    A, b, c = lpgen.dense_lp(40, 30, 5)
    assert A.shape == (40, 30) and b.shape == (40,) and c.shape == (30,)
    assert A.min() >= 1.0 and A.max() < 10.0
    assert b.min() >= 100.0 and b.max() < 1000.0
    assert c.min() >= 1.0 and c.max() < 10.0
    u = lpgen.uniform01(5, 0, 40 * 30 + 40 + 30)
    np.testing.assert_array_equal(A.ravel(), 1.0 + u[:1200] * 9.0)
    np.testing.assert_array_equal(b, 100.0 + 900.0 * u[1200:1240])
    np.testing.assert_array_equal(c, 1.0 + 9.0 * u[1240:])


def test_dense_lp_deterministic():
    d1 = lpgen.lp_digest(*lpgen.dense_lp(256, 256, 1))
    d2 = lpgen.lp_digest(*lpgen.dense_lp(256, 256, 1))
    d3 = lpgen.lp_digest(*lpgen.dense_lp(256, 256, 2))
    assert d1 == d2 != d3
    # regression value: changing the generator changes every stored case
    assert d1 == "c1b3d07caffc0501adf062f00226ba14127d469d2a0fbb4c55c61f6cea145408"


def test_batch_and_stream_shapes():
    sh = lpgen.batch_shapes(4096, 16, 128, 1)
    ms = np.array([s[0] for s in sh])
    ns = np.array([s[1] for s in sh])
    assert ms.min() == 16 and ms.max() == 128 and ns.min() == 16 and ns.max() == 128
    assert abs(ms.mean() - 72) < 2 and abs(ns.mean() - 72) < 2
    ls = lpgen.loguniform_shapes(2000, 32, 4096, 3)
    assert min(min(s) for s in ls) >= 32 and max(max(s) for s in ls) <= 4096
    t = lpgen.poisson_arrivals(20000, 2000.0, 4)
    assert np.all(np.diff(t) > 0)
    assert abs(20000 / t[-1] - 2000.0) < 60.0
