"""Seeded synthetic LP generator (inputs only; no simplex arithmetic here).

This module is shared by the tests, the benchmark and the oracle's callers.  It
holds none of the method's arithmetic: it only draws the data (A, b, c) of a
dense LP  maximize c^T x  s.t.  A x <= b, x >= 0  (the problem statement of
Section III, Table I of arXiv 2211.10979).  The paper's own generator for its
25000 x 25000 random dense LP is unspecified ("similar to" its refs [19, 33]),
so the distributions below stand in for it:

    A_ij ~ U[1, 10),   b_i ~ U[100, 1000),   c_j ~ U[1, 10)

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the k-th
draw (k = 0, 1, ...) of seed s is  mix64(s + (k + 1) * GAMMA)  with
GAMMA = 0x9E3779B97F4A7C15 and mix64 the published 64-bit finaliser.  Draws are
consumed in the order A (row-major, i then j), then b, then c, and a draw x maps
to u = (x >> 11) * 2**-53 in [0, 1).
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# chunk size for the vectorised stream (bounds temporary memory)
_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function, applied elementwise (uint64, wrapping)."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_stream(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream of `seed`."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, count, _CHUNK):
            hi = min(count, lo + _CHUNK)
            k = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            out[lo:hi] = _mix64(s + k * GAMMA)
    return out


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """u = (x >> 11) * 2^-53 for the SplitMix64 draws start .. start+count-1."""
    x = splitmix64_stream(seed, start, count)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def dense_lp(m: int, n: int, seed: int):
    """The seeded dense LP (A m x n row-major float64, b m, c n).

    A_ij = 1 + 9u, b_i = 100 + 900u, c_j = 1 + 9u, drawn in the order A, b, c.
    """
    if m <= 0 or n <= 0:
        raise ValueError("m and n must be positive")
    A = uniform01(seed, 0, m * n)
    A *= 9.0
    A += 1.0
    A = A.reshape(m, n)
    b = 100.0 + 900.0 * uniform01(seed, m * n, m)
    c = 1.0 + 9.0 * uniform01(seed, m * n + m, n)
    return A, b, c


def diag_dominant_lp(m: int, n: int, seed: int):
    """A dense LP whose optimal basis holds min(m, n) structural variables:
    A_ij = u (i != j), A_ii = 4 max(m, n) + u, b_i = 100 + 900u, c_j = 1 + 9u
    (draws in the order A row-major, b, c).  The strong diagonal makes
    x = A^-1 b and y = A^-T c positive at m = n, so every structural variable
    ends basic (k = m): the workload of an FP64 recovery of a large basis.
    """
    if m <= 0 or n <= 0:
        raise ValueError("m and n must be positive")
    A = uniform01(seed, 0, m * n).reshape(m, n)
    d = np.arange(min(m, n))
    A[d, d] += 4.0 * max(m, n)
    b = 100.0 + 900.0 * uniform01(seed, m * n, m)
    c = 1.0 + 9.0 * uniform01(seed, m * n + m, n)
    return A, b, c


def lp_digest(A, b, c) -> str:
    """SHA-256 of the little-endian float64 bytes of A, then b, then c."""
    h = hashlib.sha256()
    for a in (A, b, c):
        h.update(np.ascontiguousarray(a, dtype="<f8").tobytes())
    return h.hexdigest()


def batch_shapes(count: int, lo: int, hi: int, seed: int):
    """Shapes (m_k, n_k) of a batch: m and n each uniform integers in [lo, hi].

    Drawn from the SplitMix64 stream of `seed`: draw 2k gives m_k, draw 2k+1
    gives n_k, via floor(u * (hi - lo + 1)) + lo.
    """
    u = uniform01(seed, 0, 2 * count)
    span = hi - lo + 1
    v = np.minimum(np.floor(u * span).astype(np.int64), span - 1) + lo
    return [(int(v[2 * k]), int(v[2 * k + 1])) for k in range(count)]


def loguniform_shapes(count: int, lo: int, hi: int, seed: int):
    """Shapes with m and n each log-uniform in [lo, hi], rounded down."""
    u = uniform01(seed, 0, 2 * count)
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    v = np.clip(v, lo, hi)
    return [(int(v[2 * k]), int(v[2 * k + 1])) for k in range(count)]


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps -ln(1-u)/rate."""
    u = uniform01(seed, 0, count)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)
