"""CPU oracle for the dense full-tableau simplex (arXiv 2211.10979, Section III).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library's product
path never does.  The arithmetic lives in ``simplex_oracle.c`` (plain C, FP64,
single-threaded); this module only compiles it with gcc and marshals arrays.

Every step follows the paper's Section III in order: the Initialization Step
(Table I tableau with the slack basis), Step 1 (Dantzig entering column),
Step 2 (minimum-ratio leaving row), Step 3 (pivoting) and the
Iterate/Finalization Step.  The readings taken where the paper is silent are
listed in the C file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simplex_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_simplex.so")
_lock = threading.Lock()
_lib = None

OPTIMAL, UNBOUNDED, ITER_LIMIT, NUMERIC, INVALID = 0, 1, 2, 3, -1
STATUS_NAMES = {0: "OPTIMAL", 1: "UNBOUNDED", 2: "ITER_LIMIT", 3: "NUMERIC", -1: "INVALID"}


class _Opts(ctypes.Structure):
    _fields_ = [
        ("rule", ctypes.c_int),
        ("eps_d", ctypes.c_double),
        ("eps_p", ctypes.c_double),
        ("max_iters", ctypes.c_long),
        ("k_cyc", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile simplex_oracle.c into a shared library next to it (gcc)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_build.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ip]
        lib.orc_build.restype = ctypes.c_int
        lib.orc_entering.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double]
        lib.orc_entering.restype = ctypes.c_int
        lib.orc_leaving.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, dp]
        lib.orc_leaving.restype = ctypes.c_int
        lib.orc_pivot.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_pivot.restype = None
        lib.orc_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, ctypes.POINTER(_Opts),
                                  ctypes.POINTER(ctypes.c_long), ip, ip, ctypes.c_long]
        lib.orc_solve.restype = ctypes.c_int
        lib.orc_solve_traced.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, ctypes.POINTER(_Opts),
                                         ctypes.POINTER(ctypes.c_long), ip, ip, ctypes.c_long,
                                         dp, dp, dp, dp]
        lib.orc_solve_traced.restype = ctypes.c_int
        lib.orc_pivot_gaps.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_pivot_gaps.restype = None
        lib.orc_extract.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, dp, dp, dp]
        lib.orc_extract.restype = None
        fp = ctypes.POINTER(ctypes.c_float)
        lib.orc32_build.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, fp, ip]
        lib.orc32_build.restype = ctypes.c_int
        lib.orc32_entering.argtypes = [ctypes.c_int, ctypes.c_int, fp, ctypes.c_int, ctypes.c_double]
        lib.orc32_entering.restype = ctypes.c_int
        lib.orc32_leaving.argtypes = [ctypes.c_int, ctypes.c_int, fp, ip, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_double, fp]
        lib.orc32_leaving.restype = ctypes.c_int
        lib.orc32_pivot.argtypes = [ctypes.c_int, ctypes.c_int, fp, ctypes.c_int, ctypes.c_int, fp, fp]
        lib.orc32_pivot.restype = None
        lib.orc32_solve.argtypes = [ctypes.c_int, ctypes.c_int, fp, ip, ctypes.POINTER(_Opts),
                                    ctypes.POINTER(ctypes.c_long), ip, ip, ctypes.c_long]
        lib.orc32_solve.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@dataclass
class Options:
    rule: int = 0            # 0 = Dantzig + Bland fallback, 1 = Bland
    eps_d: float = 1e-9
    eps_p: float = 1e-9
    max_iters: int = -1      # -1 = 50 (m + n)
    k_cyc: int = 50

    def c(self) -> _Opts:
        return _Opts(self.rule, self.eps_d, self.eps_p, self.max_iters, self.k_cyc)


@dataclass
class Result:
    status: int
    iters: int
    x: np.ndarray
    y: np.ndarray
    obj: float
    basis: np.ndarray
    qlog: np.ndarray
    plog: np.ndarray
    T: np.ndarray


def build_tableau(A, b, c):
    """Initialization Step: returns (T (m+1) x (n+m+1), basis[m])."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m, n = A.shape
    T = np.empty((m + 1, n + m + 1), dtype=np.float64)
    basis = np.empty(m, dtype=np.int32)
    rc = _load().orc_build(m, n, _dp(A), _dp(b), _dp(c), _dp(T), _ip(basis))
    if rc != 0:
        raise ValueError("invalid LP (need m, n > 0 and finite b >= 0)")
    return T, basis


def entering(T, m, n, bland=False, eps_d=1e-9) -> int:
    """Step 1 on tableau T; -1 if optimal."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    return int(_load().orc_entering(m, n, _dp(T), int(bland), eps_d))


def leaving(T, basis, m, n, q, bland=False, eps_p=1e-9):
    """Step 2 on tableau T and column q; returns (p, min ratio), p = -1 if unbounded."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    basis = np.ascontiguousarray(basis, dtype=np.int32)
    ratio = ctypes.c_double(0.0)
    p = _load().orc_leaving(m, n, _dp(T), _ip(basis), q, int(bland), eps_p, ctypes.byref(ratio))
    return int(p), ratio.value


def pivot(T, m, n, p, q):
    """Step 3 in place on a C-contiguous float64 tableau."""
    assert T.flags.c_contiguous and T.dtype == np.float64
    r = np.empty(T.shape[1], dtype=np.float64)
    f = np.empty(T.shape[0], dtype=np.float64)
    _load().orc_pivot(m, n, _dp(T), p, q, _dp(r), _dp(f))


def solve_tableau(T, basis, m, n, opts: Options | None = None, log_cap: int = 1 << 20):
    """Iterate Steps 1-3 in place on (T, basis); returns (status, iters, qlog, plog)."""
    opts = opts or Options()
    assert T.flags.c_contiguous and T.dtype == np.float64
    assert basis.flags.c_contiguous and basis.dtype == np.int32
    cap = int(log_cap)
    qlog = np.full(cap, -1, dtype=np.int32)
    plog = np.full(cap, -1, dtype=np.int32)
    it = ctypes.c_long(0)
    o = opts.c()
    st = _load().orc_solve(m, n, _dp(T), _ip(basis), ctypes.byref(o), ctypes.byref(it),
                           _ip(qlog), _ip(plog), cap)
    k = min(it.value, cap)
    return int(st), int(it.value), qlog[:k].copy(), plog[:k].copy()


def pivot_gaps(T, m, n, q, p, eps_d=1e-9, eps_p=1e-9):
    """Separation of the Step 1 and Step 2 decisions (q, p) on tableau T:
    (second most negative candidate - T[0][q], second smallest eligible ratio -
    ratio of row p), +inf where there is no second candidate."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    dg, rg = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _load().orc_pivot_gaps(m, n, _dp(T), q, p, eps_d, eps_p, ctypes.byref(dg), ctypes.byref(rg))
    return dg.value, rg.value


@dataclass
class Trace:
    """Per-pivot record of a traced solve: minimum ratio of Step 2, the
    entering column's objective-row entry T[0][q], and the gaps of pivot_gaps
    (NaN for pivots taken under Bland's rule)."""
    theta: np.ndarray
    dval: np.ndarray
    dgap: np.ndarray
    rgap: np.ndarray


def solve_traced(A, b, c, opts: Options | None = None, log_cap: int = 1 << 20):
    """solve() that also records, for every pivot, its minimum ratio and the
    separation of its Step 1 and Step 2 decisions.  Returns (Result, Trace)."""
    opts = opts or Options()
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    T, basis = build_tableau(A, b, c)
    cap = int(log_cap)
    qlog = np.full(cap, -1, dtype=np.int32)
    plog = np.full(cap, -1, dtype=np.int32)
    theta = np.full(cap, np.nan)
    dgap = np.full(cap, np.nan)
    rgap = np.full(cap, np.nan)
    dval = np.full(cap, np.nan)
    it = ctypes.c_long(0)
    o = opts.c()
    st = _load().orc_solve_traced(m, n, _dp(T), _ip(basis), ctypes.byref(o), ctypes.byref(it),
                                  _ip(qlog), _ip(plog), cap, _dp(dgap), _dp(rgap), _dp(theta),
                                  _dp(dval))
    k = min(it.value, cap)
    x, y, obj = extract(T, basis, m, n)
    res = Result(int(st), int(it.value), x, y, obj, basis, qlog[:k].copy(), plog[:k].copy(), T)
    return res, Trace(theta[:k].copy(), dval[:k].copy(), dgap[:k].copy(), rgap[:k].copy())


def extract(T, basis, m, n):
    """x (n), y (m), objective from a tableau."""
    x = np.empty(n, dtype=np.float64)
    y = np.empty(m, dtype=np.float64)
    obj = ctypes.c_double(0.0)
    T = np.ascontiguousarray(T, dtype=np.float64)
    basis = np.ascontiguousarray(basis, dtype=np.int32)
    _load().orc_extract(m, n, _dp(T), _ip(basis), _dp(x), _dp(y), ctypes.byref(obj))
    return x, y, obj.value


def solve(A, b, c, opts: Options | None = None, log_cap: int = 1 << 20) -> Result:
    """Full solve: Initialization Step, then Steps 1-3 until termination."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    T, basis = build_tableau(A, b, c)
    st, it, qlog, plog = solve_tableau(T, basis, m, n, opts, log_cap)
    x, y, obj = extract(T, basis, m, n)
    return Result(st, it, x, y, obj, basis, qlog, plog, T)


# ---------------------------------------------------------------- float variant
def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def build_tableau32(A, b, c):
    """Initialization Step on a float tableau (inputs rounded to float)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    m, n = A.shape
    T = np.empty((m + 1, n + m + 1), dtype=np.float32)
    basis = np.empty(m, dtype=np.int32)
    if _load().orc32_build(m, n, _dp(A), _dp(b), _dp(c), _fp(T), _ip(basis)) != 0:
        raise ValueError("invalid LP (need m, n > 0 and finite b >= 0)")
    return T, basis


def entering32(T, m, n, bland=False, eps_d=1e-5) -> int:
    T = np.ascontiguousarray(T, dtype=np.float32)
    return int(_load().orc32_entering(m, n, _fp(T), int(bland), eps_d))


def leaving32(T, basis, m, n, q, bland=False, eps_p=1e-6):
    T = np.ascontiguousarray(T, dtype=np.float32)
    basis = np.ascontiguousarray(basis, dtype=np.int32)
    ratio = ctypes.c_float(0.0)
    p = _load().orc32_leaving(m, n, _fp(T), _ip(basis), q, int(bland), eps_p, ctypes.byref(ratio))
    return int(p), ratio.value


def pivot32(T, m, n, p, q):
    assert T.flags.c_contiguous and T.dtype == np.float32
    r = np.empty(T.shape[1], dtype=np.float32)
    f = np.empty(T.shape[0], dtype=np.float32)
    _load().orc32_pivot(m, n, _fp(T), p, q, _fp(r), _fp(f))


def solve32(A, b, c, opts: Options | None = None, log_cap: int = 1 << 20):
    """Steps 1-3 on a float tableau from the slack basis (default tolerances
    eps_d = 1e-5, eps_p = 1e-6).  Returns (status, iters, qlog, plog, T, basis)."""
    opts = opts or Options(eps_d=1e-5, eps_p=1e-6)
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    T, basis = build_tableau32(A, b, c)
    cap = int(log_cap)
    qlog = np.full(cap, -1, dtype=np.int32)
    plog = np.full(cap, -1, dtype=np.int32)
    it = ctypes.c_long(0)
    o = opts.c()
    st = _load().orc32_solve(m, n, _fp(T), _ip(basis), ctypes.byref(o), ctypes.byref(it),
                             _ip(qlog), _ip(plog), cap)
    k = min(it.value, cap)
    return int(st), int(it.value), qlog[:k].copy(), plog[:k].copy(), T, basis
